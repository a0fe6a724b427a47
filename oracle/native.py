"""Build and load the C part of the oracle (``jacobi_svd.c``).

TEST INFRASTRUCTURE ONLY: see the package docstring. The shared object is built
in-tree next to its source with the host C compiler and OpenMP; nothing here is
shared with the GPU library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi_svd.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``jacobi_svd.c`` into ``_liboracle.so`` (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    cc = os.environ.get("CC", "gcc")
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_jacobi_svd.argtypes = [
                ctypes.c_int64, ctypes.c_int64, dp, dp, dp, dp, ctypes.c_double,
                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp]
            lib.oracle_jacobi_svd.restype = ctypes.c_int
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the oracle's parallel sweeps use."""
    return int(_load().oracle_num_threads())


def jacobi_svd(a: np.ndarray, eps: float = 0.0, max_sweeps: int = 60, nthreads: int = 0,
               return_info: bool = False, max_rounds: int = 0, want_off: bool = True):
    """Thin SVD ``a = U diag(sigma) V^T`` of a real matrix by one-sided Jacobi in FP64.

    ``max_rounds`` bounds the work (a timing sample); ``want_off`` = False skips the
    final all-pairs orthogonality diagnostic (reported as NaN then).

    Works on ``a`` when m >= n and on ``a.T`` otherwise (then U and V swap), so U
    is m x k, V is n x k with k = min(m, n), sigma descending.
    """
    a = np.asarray(a, dtype=np.float64)
    if a.ndim != 2:
        raise ValueError("input must be 2-D")
    m, n = a.shape
    wide = n > m
    w = np.ascontiguousarray(a.T if wide else a)
    mm, nn = w.shape
    sigma = np.zeros(nn)
    u = np.zeros((mm, nn))
    v = np.zeros((nn, nn))
    sweeps = ctypes.c_int(0)
    off = ctypes.c_double(0.0)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = _load().oracle_jacobi_svd(
        mm, nn, w.ctypes.data_as(dp), sigma.ctypes.data_as(dp), u.ctypes.data_as(dp),
        v.ctypes.data_as(dp), float(eps), int(max_sweeps), int(max_rounds), int(nthreads),
        ctypes.byref(sweeps), ctypes.byref(off) if want_off else None)
    if not want_off:
        off = ctypes.c_double(float("nan"))
    if rc < 0:
        raise ValueError("oracle_jacobi_svd: bad arguments")
    if wide:
        u, v = v, u
    if return_info:
        return u, sigma, v, {"converged": rc == 0, "sweeps": sweeps.value, "off": off.value}
    return u, sigma, v
