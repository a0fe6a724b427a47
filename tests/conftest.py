import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU test")


def pytest_sessionstart(session):
    """Build libsvt.so in-tree when it is missing or older than its sources (nvcc
    cross-compiles without a GPU); a failed build leaves the tests that load the
    library to fail loudly."""
    try:
        from paper_2607_22484_gb300 import build as _build
        _build.build()
    except Exception as e:  # noqa: BLE001 - reported, not hidden: library tests then fail
        sys.stderr.write(f"libsvt.so build failed: {e}\n")


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")


def _block_spread(err, b):
    """max / RMS over the b x b blocks of `err` of each block's root-mean-square entry
    (ragged edge blocks included, weighted by their own size).

    Rounding errors of a correct solve spread evenly over the matrix: a CPU emulation
    of the BF16 tier at 1024^2 gives 1.11 for 32 x 32 blocks and 1.05 for 128 x 128,
    and low-rank errors with Haar singular vectors (rank 64 at 8192 x 2048, rank 300 at
    4096^2) give 1.03-1.13. A tile, a 32-column epilogue chunk or a ragged tail that the
    kernel got partly wrong stands out of that by far more than the factor 2 the tests
    allow, even where it hides under the Frobenius aggregate."""
    import numpy as np
    e = np.asarray(err, np.float64)
    m, n = e.shape
    r0, c0 = np.arange(0, m, b), np.arange(0, n, b)
    s = np.add.reduceat(np.add.reduceat(e * e, r0, axis=0), c0, axis=1)
    cnt = np.outer(np.diff(np.append(r0, m)), np.diff(np.append(c0, n)))
    ms = s / cnt
    return float(np.sqrt(ms.max() / ms.mean())) if ms.mean() > 0 else 0.0


@pytest.fixture(scope="session")
def block_spread():
    return _block_spread
