"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol include/svt.h declares, and its host arithmetic (status names, options,
workspace sizes, the polynomial schedule) is right."""
import ctypes
import re
import os

import numpy as np
import pytest

import paper_2607_22484_gb300 as pkg
from oracle import schedule as osch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "svt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(svt_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    decl = _declared()
    assert decl == sorted(pkg.EXPORTS)
    lib = pkg.lib()
    for name in decl:
        assert hasattr(lib, name), name


def test_status_strings():
    assert pkg.status_str(0) == "SVT_OK"
    assert pkg.status_str(4) == "SVT_ERR_NONFINITE"
    assert pkg.status_str(99) == "SVT_ERR_UNKNOWN"


def test_workspace_bytes():
    small = pkg.workspace_bytes(64, 64, prec="bf16")
    big = pkg.workspace_bytes(4096, 4096, prec="bf16")
    assert 0 < small < big
    # wide and tall give the same (the wide case is the tall case of A^T)
    assert pkg.workspace_bytes(300, 100) == pkg.workspace_bytes(100, 300)
    # FP32 tier carries hi/lo pairs: more than BF16
    assert pkg.workspace_bytes(512, 512, prec="fp32") > pkg.workspace_bytes(512, 512, prec="bf16")
    with pytest.raises(pkg.SVTError):
        pkg.workspace_bytes(0, 5)


def test_reserved_fp8_tier_is_unsupported():
    """SVT_FP8_EXPERIMENTAL is reserved: rejected as unsupported, not as invalid."""
    with pytest.raises(pkg.SVTError) as e:
        pkg.workspace_bytes(64, 64, prec="fp8_experimental")
    assert e.value.status == pkg.binding.ERR_UNSUPPORTED
    with pytest.raises(pkg.SVTError) as e:
        pkg.workspace_bytes(64, 64, prec=7)
    assert e.value.status == pkg.binding.ERR_INVALID


def test_fp8_experiment_workspace():
    """svt_workspace_bytes_fp8: the BF16 tier's workspace plus one e4m3 k x k copy for a
    P-chain policy and four for an S-chain policy; other tiers are rejected."""
    m, n = 700, 300
    base = pkg.workspace_bytes(m, n, prec="bf16")
    assert pkg.workspace_bytes_fp8(m, n) == base
    p = pkg.workspace_bytes_fp8(m, n, p_steps=[1, 2])
    s = pkg.workspace_bytes_fp8(m, n, s_steps=[15, 16], s_y2_only=True)
    both = pkg.workspace_bytes_fp8(m, n, p_steps=[1], s_steps=[15])
    k = min(m, n)
    assert k * k <= p - base <= k * (k + 64) + (1 << 20)
    assert 4 * k * k <= s - base <= 4 * k * (k + 64) + (4 << 20)
    assert both - base == (p - base) + (s - base)
    for bad in ("fp32", "fp64"):
        with pytest.raises(pkg.SVTError) as e:
            pkg.workspace_bytes_fp8(m, n, p_steps=[1], prec=bad)
        assert e.value.status == pkg.binding.ERR_INVALID
    with pytest.raises(ValueError):
        pkg.fp8_policy(p_steps=[64])
    out = ctypes.c_size_t(0)
    o = pkg.make_options(prec="bf16")
    bad = pkg.fp8_policy(s_steps=[3])
    bad.reserved = 1
    assert pkg.lib().svt_workspace_bytes_fp8(m, n, ctypes.byref(o), ctypes.byref(bad),
                                             ctypes.byref(out)) == pkg.binding.ERR_INVALID
    assert pkg.lib().svt_workspace_bytes_fp8(m, n, ctypes.byref(o), None,
                                             ctypes.byref(out)) == pkg.binding.ERR_INVALID


@pytest.mark.parametrize("delta", [0.0, 0.01, 1e-4])
@pytest.mark.parametrize("ell0", [1e-3, 1e-2])
def test_schedule_matches_oracle(delta, ell0):
    """The library's C++ Remez and the oracle's NumPy Remez (independent code) agree."""
    lib_c = pkg.schedule_coeffs("pe5", 20, ell0, delta)
    ora_c, _ = osch.pe5_schedule(20, ell0, delta)
    np.testing.assert_allclose(lib_c, np.array(ora_c), rtol=1e-9, atol=1e-12)


def test_schedule_ns3_and_errors():
    c = pkg.schedule_coeffs("ns3", 4)
    np.testing.assert_array_equal(c, [[1.5, -0.5, 0.0]] * 4)
    with pytest.raises(pkg.SVTError):
        pkg.schedule_coeffs("pe5", 3, ell0=0.0)
    with pytest.raises(pkg.SVTError):
        pkg.schedule_coeffs("pe5", -1)


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the header's sizes and field offsets
    (a C program compiled against include/svt.h prints them)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {
        "svt_options": (pkg.Options, ["iters", "prec", "schedule", "norm", "ell0", "delta",
                                      "polish", "mode", "fuse", "hp_steps", "tile"]),
        "svt_matrix": (pkg.Matrix, ["A", "m", "n", "lda", "tau", "Y", "ldy", "opt", "d_status"]),
        "svt_completion_params": (pkg.binding.CompletionParams,
                                  ["lambda", "lambda0", "eta", "step", "tol", "max_steps",
                                   "stage_steps"]),
        "svt_completion_stats": (pkg.binding.CompletionStats,
                                 ["steps", "stages", "stage_steps", "status", "solve_status",
                                  "reserved", "lambda", "rel_change", "diff2", "data2"]),
    }
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "svt.h"', "int main(void) {"]
    for name, (_, fields) in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run(
        [str(exe)], check=True, capture_output=True, text=True).stdout.splitlines())
    for name, (cls, fields) in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, (pyname, _) in zip(fields, cls._fields_):
            assert int(got[f"{name}.{f}"]) == getattr(cls, pyname).offset, (name, f)


def test_complete_rejects_null_arguments_on_the_host():
    """svt_complete validates its arguments before touching the device."""
    import ctypes
    lib = pkg.lib()
    prm = pkg.binding.CompletionParams(0.1, 0.1, 0.5, 1.0, 0.0, 5, 0)
    st = lib.svt_complete(None, None, 4, None, 4, None, 4, None, 4, None, 4, 4, 4,
                          ctypes.byref(prm), None, None, None)
    assert pkg.status_str(st) == "SVT_ERR_INVALID"


@pytest.mark.parametrize("bad", [
    {"iters": -1}, {"iters": 1001}, {"prec": 9}, {"schedule": 7}, {"norm": 5},
    {"ell0": 1.0}, {"ell0": float("nan")}, {"delta": float("inf")}, {"mode": 2},
    {"hp_steps": -2}, {"tile": 300}, {"tile": 64},
])
def test_option_validation_on_the_host(bad):
    """Options outside their ranges are rejected before any device work (the sizing
    call runs the same resolution as every entry point)."""
    with pytest.raises(pkg.SVTError) as e:
        pkg.workspace_bytes(256, 256, **bad)
    assert e.value.status == pkg.binding.ERR_INVALID


def test_valid_option_corners_on_the_host():
    for ok in ({"iters": 0}, {"iters": 1000}, {"tile": 128}, {"tile": 256}, {"tile": 512},
               {"ell0": 0.0}, {"delta": 0.0}, {"hp_steps": -1}, {"schedule": "ns3"},
               {"prec": "fp64", "tile": 512}):
        assert pkg.workspace_bytes(256, 256, **ok) > 0
