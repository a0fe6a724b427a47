"""The fused solve's dependency derivation (csrc/fused_deps.h), checked on the host.

tests/fused_deps_check.cpp compiles against the library's own header and simulates
fused launches at block granularity under random interleavings of all tiles whose
conditions hold: every read must see the version program order implies, no write may
clobber a block an earlier reader still needs, norms must be complete before scales
read them, and no launch may stall. It runs the solve's own product sequence (chain
and strip modes, square and tall, one and two CTAs per tile, with and without the P
chain of Corollary 1's mode) and random product sequences in strip mode. Planting a mistake in the header (dropping the WAR
conditions, letting the combine ignore one chain, a strip target one tile short)
makes it fail by the thousands.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2607_22484_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("fused_deps") / "check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-I", CSRC,
                    os.path.join(HERE, "fused_deps_check.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fused_dependencies_are_race_free(checker, seed):
    r = subprocess.run([checker, str(seed), "20"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert " 0 failures" in r.stdout, r.stdout
