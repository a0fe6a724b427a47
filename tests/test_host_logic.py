"""Host logic of the library checked on the CPU (tests/host_logic_check.cpp, compiled
against the library's own headers): how serving's large lane splits a solve's product
work into launches (segments.h), the autotune cache's JSON writer and strict reader
(tuning_json.h), and the serving loop's first-fit workspace placement (arena.h) against
a brute-force model. Planting a mistake in any of them (no part limit, no format check,
no merge with the previous free range) makes it fail."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2607_22484_gb300", "csrc")


def _cuda_include():
    root = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(root, "include")
    return path if os.path.exists(os.path.join(path, "cuda_runtime.h")) else None


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("no C++ compiler or CUDA headers")
    exe = str(tmp_path_factory.mktemp("host_logic") / "check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-I", CSRC, "-I", inc,
                    os.path.join(HERE, "host_logic_check.cpp"), "-o", exe],
                   check=True, capture_output=True, text=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_segments_tuning_json_and_arena(checker, seed):
    r = subprocess.run([checker, str(seed)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("0 failures"), r.stdout
