"""Host-side checks of the C ABI (no GPU): the library loads, exports every
symbol include/svt.h declares, and its host arithmetic (status names, options,
workspace sizes, the polynomial schedule) is right."""
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
