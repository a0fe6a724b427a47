"""ctypes binding of libsvt (include/svt.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module turns
torch tensors into device pointers and the current torch stream into a
cudaStream_t, and raises on error statuses. PyTorch is used only for device
memory (the workspace, outputs) and streams. If libsvt.so is missing the import
fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsvt.so")

# svt_status
OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_DIVERGED, ERR_TIMEOUT, \
    ERR_NOT_READY, ERR_BUSY, ERR_UNSUPPORTED, ERR_CANCELLED = range(11)
# svt_debug_flag
DEBUG = {"fail_plan": 1, "admit_delay_us": 2, "wait_limit_ns": 3}
# svt_precision
FP64, FP32, BF16, FP8_EXPERIMENTAL = 0, 1, 2, 3
PREC = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "fp8_experimental": FP8_EXPERIMENTAL}
# svt_schedule_kind / svt_norm_kind / svt_mode
SCHED_AUTO, SCHED_PE5, SCHED_NS3 = 0, 1, 2
SCHED = {"auto": SCHED_AUTO, "pe5": SCHED_PE5, "ns3": SCHED_NS3}
NORM_AUTO, NORM_FRO, NORM_GRAM = 0, 1, 2
NORM = {"auto": NORM_AUTO, "fro": NORM_FRO, "gram": NORM_GRAM}
MODE_SVT, MODE_RANK_R = 0, 1
MODE = {"svt": MODE_SVT, "rank_r": MODE_RANK_R}

# Every symbol include/svt.h declares.
EXPORTS = [
    "svt_status_str", "svt_options_default", "svt_workspace_bytes_ex", "svt_workspace_bytes",
    "svt_ctx_create", "svt_ctx_destroy", "svt_polar", "svt_polar_ex", "svt_batch",
    "svt_batch_workspace_bytes", "svt_serve_submit", "svt_serve_poll", "svt_serve_release",
    "svt_ctx_sync", "svt_schedule_coeffs", "svt_debug_gemm_bf16", "svt_debug_gemm_bf16_ex",
    "svt_ctx_launch_count",
    "svt_ctx_profile", "svt_ctx_profile_read", "svt_polar_noalloc", "svt_autotune",
    "svt_prox_grad_step", "svt_complete", "svt_autotune_schedule", "svt_autotune_batch",
    "svt_ctx_profile_read_ex", "svt_debug_wait_timeout", "svt_polar_f64", "svt_serve_cancel",
    "svt_serve_metrics", "svt_ctx_debug", "svt_tuning_export", "svt_tuning_import",
    "svt_polar_fp8", "svt_workspace_bytes_fp8", "svt_debug_gemm_e4m3",
]
NOALLOC_SCRATCH_BYTES = 32 << 20


class Options(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("prec", ctypes.c_int), ("schedule", ctypes.c_int),
                ("norm", ctypes.c_int), ("ell0", ctypes.c_double), ("delta", ctypes.c_double),
                ("polish", ctypes.c_int), ("mode", ctypes.c_int), ("fuse", ctypes.c_int),
                ("hp_steps", ctypes.c_int), ("tile", ctypes.c_int)]


class Fp8Policy(ctypes.Structure):
    _fields_ = [("p_steps", ctypes.c_uint64), ("s_steps", ctypes.c_uint64),
                ("s_y2_only", ctypes.c_int), ("reserved", ctypes.c_int)]


class Matrix(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("tau", ctypes.c_float), ("Y", ctypes.c_void_p),
                ("ldy", ctypes.c_int64), ("opt", Options), ("d_status", ctypes.c_void_p)]


class CompletionParams(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_float), ("lam0", ctypes.c_float), ("eta", ctypes.c_float),
                ("step", ctypes.c_float), ("tol", ctypes.c_float), ("max_steps", ctypes.c_int),
                ("stage_steps", ctypes.c_int)]


class CompletionStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("stages", ctypes.c_int), ("stage_steps", ctypes.c_int),
                ("status", ctypes.c_int), ("solve_status", ctypes.c_int), ("reserved", ctypes.c_int),
                ("lam", ctypes.c_double), ("rel_change", ctypes.c_double),
                ("diff2", ctypes.c_double), ("data2", ctypes.c_double)]


COMPLETION_STATS_BYTES = ctypes.sizeof(CompletionStats)


def read_completion_stats(stats) -> dict:
    """The svt_completion_stats a run wrote into the CUDA byte tensor `stats` (copies it
    to the host, which waits for the run)."""
    raw = bytes(stats.cpu().numpy().tobytes())[:COMPLETION_STATS_BYTES]
    c = CompletionStats.from_buffer_copy(raw)
    return {"steps": c.steps, "stages": c.stages, "stage_steps": c.stage_steps,
            "status": c.status, "lam": c.lam, "rel_change": c.rel_change,
            "data_norm": c.data2 ** 0.5}


class SVTError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_str(status)}")


_lib = None
_lock = threading.Lock()


def lib():
    """Load libsvt.so (built by ``build.build()``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsvt.so not built at {LIB_PATH}: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.svt_status_str.argtypes = [i32]
        L.svt_status_str.restype = ctypes.c_char_p
        L.svt_options_default.argtypes = [ctypes.POINTER(Options)]
        L.svt_options_default.restype = None
        L.svt_workspace_bytes_ex.argtypes = [i64, i64, ctypes.POINTER(Options),
                                             ctypes.POINTER(ctypes.c_size_t)]
        L.svt_workspace_bytes.argtypes = [i64, i64, i32, ctypes.POINTER(ctypes.c_size_t)]
        L.svt_ctx_create.argtypes = [i32, vp, ctypes.c_size_t, ctypes.POINTER(vp)]
        L.svt_ctx_destroy.argtypes = [vp]
        L.svt_polar.argtypes = [vp, vp, i64, i64, i64, ctypes.c_float, i32, i32, vp, i64, vp, vp]
        L.svt_polar_ex.argtypes = [vp, vp, i64, i64, i64, ctypes.c_float, ctypes.POINTER(Options),
                                   vp, i64, vp, vp]
        L.svt_polar_f64.argtypes = [vp, vp, i64, i64, i64, ctypes.c_float,
                                    ctypes.POINTER(Options), vp, i64, vp, vp]
        L.svt_batch.argtypes = [vp, ctypes.POINTER(Matrix), i32, vp]
        L.svt_batch_workspace_bytes.argtypes = [ctypes.POINTER(Matrix), i32,
                                                ctypes.POINTER(ctypes.c_size_t)]
        L.svt_serve_submit.argtypes = [vp, ctypes.POINTER(Matrix), ctypes.POINTER(ctypes.c_uint64)]
        L.svt_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
        L.svt_serve_release.argtypes = [vp, ctypes.c_uint64]
        L.svt_serve_cancel.argtypes = [vp, ctypes.c_uint64]
        L.svt_polar_fp8.argtypes = [vp, vp, i64, i64, i64, ctypes.c_float, ctypes.POINTER(Options),
                                    ctypes.POINTER(Fp8Policy), vp, i64, vp, vp]
        L.svt_workspace_bytes_fp8.argtypes = [i64, i64, ctypes.POINTER(Options),
                                              ctypes.POINTER(Fp8Policy), ctypes.POINTER(ctypes.c_size_t)]
        L.svt_debug_gemm_e4m3.argtypes = [vp, vp, vp, i64, i64, i64, i64, i64, vp, i64, i32, vp]
        L.svt_serve_metrics.argtypes = [vp, ctypes.c_char_p]
        L.svt_ctx_debug.argtypes = [vp, i32, i64]
        L.svt_tuning_export.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t,
                                        ctypes.POINTER(ctypes.c_size_t)]
        L.svt_tuning_import.argtypes = [vp, ctypes.c_char_p]
        L.svt_ctx_sync.argtypes = [vp, vp]
        L.svt_schedule_coeffs.argtypes = [i32, i32, ctypes.c_double, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_double)]
        L.svt_debug_gemm_bf16.argtypes = [vp, i32, vp, vp, vp, vp, i64, i64, i64, i64, i64, vp,
                                          i64, i32, vp]
        L.svt_debug_gemm_bf16_ex.argtypes = [vp, i32, vp, vp, vp, vp, i64, i64, i64, i64, i64,
                                             vp, i64, i32, i32, vp]
        L.svt_prox_grad_step.argtypes = [vp, vp, i64, vp, i64, vp, i64, vp, i64, i64, i64,
                                         ctypes.c_float, ctypes.c_float, ctypes.POINTER(Options),
                                         vp, vp]
        L.svt_complete.argtypes = [vp, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, i64, i64,
                                   ctypes.POINTER(CompletionParams), ctypes.POINTER(Options), vp,
                                   vp]
        L.svt_autotune_schedule.argtypes = [vp, vp, i64, i64, i64, ctypes.c_float,
                                            ctypes.POINTER(Options), ctypes.c_double, i32, vp,
                                            i64, vp, i64, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double), vp]
        L.svt_autotune_batch.argtypes = [vp, ctypes.POINTER(Matrix), i32, i32, vp,
                                         ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double)]
        L.svt_debug_wait_timeout.argtypes = [vp, vp, vp]
        L.svt_ctx_launch_count.argtypes = [vp]
        L.svt_ctx_launch_count.restype = ctypes.c_uint64
        L.svt_ctx_profile.argtypes = [vp, i32]
        L.svt_autotune.argtypes = [vp, vp, i64, i64, i64, ctypes.c_float, ctypes.POINTER(Options),
                                   vp, i64, i32, vp]
        L.svt_polar_noalloc.argtypes = [i32, vp, i64, i64, i64, ctypes.c_float,
                                        ctypes.POINTER(Options), vp, i64, vp, vp]
        L.svt_ctx_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_uint64)]
        L.svt_ctx_profile_read_ex.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_uint64)]
        for name in EXPORTS:
            if name not in ("svt_status_str", "svt_options_default", "svt_ctx_launch_count"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def status_str(s: int) -> str:
    return lib().svt_status_str(int(s)).decode()


def _check(st: int, where: str):
    if st != OK:
        raise SVTError(st, where)


def make_options(iters: int = 20, prec="bf16", schedule="auto", norm="auto", ell0: float = 1e-3,
                 delta: float = -1.0, polish: bool = True, mode="svt", hp_steps: int = -1,
                 fuse: bool = True, tile: int = 0) -> Options:
    o = Options()
    lib().svt_options_default(ctypes.byref(o))
    o.iters = int(iters)
    o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    o.schedule = SCHED[schedule] if isinstance(schedule, str) else int(schedule)
    o.norm = NORM[norm] if isinstance(norm, str) else int(norm)
    o.ell0 = float(ell0)
    o.delta = float(delta)
    o.polish = 1 if polish else 0
    o.mode = MODE[mode] if isinstance(mode, str) else int(mode)
    o.hp_steps = int(hp_steps)
    o.fuse = 1 if fuse else 0
    o.tile = int(tile)
    return o


def workspace_bytes(m: int, n: int, **opts) -> int:
    out = ctypes.c_size_t(0)
    o = make_options(**opts)
    _check(lib().svt_workspace_bytes_ex(int(m), int(n), ctypes.byref(o), ctypes.byref(out)),
           "svt_workspace_bytes_ex")
    return int(out.value)


def fp8_policy(p_steps=(), s_steps=(), s_y2_only=False) -> Fp8Policy:
    """svt_fp8_policy from step lists (bit t of p_steps / s_steps: step t on e4m3)."""
    def bits(steps):
        v = 0
        for t in steps:
            if not 0 <= int(t) < 64:
                raise ValueError("FP8 policy steps are 0..63")
            v |= 1 << int(t)
        return v
    return Fp8Policy(bits(p_steps), bits(s_steps), 1 if s_y2_only else 0, 0)


def workspace_bytes_fp8(m: int, n: int, p_steps=(), s_steps=(), s_y2_only=False, **opts) -> int:
    out = ctypes.c_size_t(0)
    o = make_options(**dict({"prec": "bf16"}, **opts))
    pol = fp8_policy(p_steps, s_steps, s_y2_only)
    _check(lib().svt_workspace_bytes_fp8(int(m), int(n), ctypes.byref(o), ctypes.byref(pol),
                                         ctypes.byref(out)), "svt_workspace_bytes_fp8")
    return int(out.value)


def schedule_coeffs(kind="pe5", iters: int = 20, ell0: float = 1e-3, delta: float = 0.0) -> np.ndarray:
    """The library's own polynomial schedule, (iters, 3) array of (a, b, c)."""
    buf = (ctypes.c_double * max(1, 3 * iters))()
    k = SCHED[kind] if isinstance(kind, str) else int(kind)
    _check(lib().svt_schedule_coeffs(k, int(iters), float(ell0), float(delta), buf),
           "svt_schedule_coeffs")
    return np.array(buf[: 3 * iters], dtype=np.float64).reshape(iters, 3)


def polar_noalloc(A, tau: float, out=None, status=None, stream=None, **opts):
    """Y = A_tau through svt_polar_noalloc: no workspace, no device allocation by
    the library (scratch is a fixed 32 MiB device array shared by all calls).
    ``out`` should be preallocated by callers that cannot allocate."""
    import torch
    a_ptr, m, n, lda = _f32_matrix(A, "A")  # rejects host tensors
    if out is None:
        out = torch.empty((m, n), dtype=torch.float32, device=A.device)
    y_ptr, ym, yn, ldy = _f32_matrix(out, "out")
    if (ym, yn) != (m, n):
        raise ValueError("out has the wrong shape")
    if out.device != A.device:
        raise ValueError("out must be on A's device")
    o = make_options(**opts)
    st_ptr = status.data_ptr() if status is not None else None
    # The library runs on A's device: the default stream is that device's current one.
    s = torch.cuda.current_stream(A.device) if stream is None else stream
    _check(lib().svt_polar_noalloc(A.device.index, ctypes.c_void_p(a_ptr), m, n, lda,
                                   ctypes.c_float(tau), ctypes.byref(o), ctypes.c_void_p(y_ptr),
                                   ldy, ctypes.c_void_p(st_ptr),
                                   ctypes.c_void_p(int(s.cuda_stream))), "svt_polar_noalloc")
    return out


def _stream_ptr(stream) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _f32_matrix(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dim() != 2:
        raise ValueError(f"{name} must be a 2-D tensor")
    if t.dtype != torch.float32 or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA float32 tensor")
    if t.stride(1) != 1:
        raise ValueError(f"{name} must be row-major (unit column stride)")
    return t.data_ptr(), t.size(0), t.size(1), t.stride(0)


class Context:
    """A libsvt context with a torch-allocated device workspace."""

    def __init__(self, device: int = 0, workspace_bytes: int = 1 << 28):
        import torch
        self.device = int(device)
        self.workspace = torch.empty(max(256, int(workspace_bytes)), dtype=torch.uint8,
                                     device=f"cuda:{self.device}")
        h = ctypes.c_void_p()
        _check(lib().svt_ctx_create(self.device, ctypes.c_void_p(self.workspace.data_ptr()),
                                    self.workspace.numel(), ctypes.byref(h)), "svt_ctx_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().svt_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ensure_workspace(self, nbytes: int):
        """Grow the workspace (re-creating the context) if it is smaller than nbytes.
        The autotune results and debug settings carry over to the new context."""
        import torch
        if nbytes <= self.workspace.numel():
            return
        torch.cuda.synchronize(self.device)
        tuning = self.tuning_export()
        self.close()
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=f"cuda:{self.device}")
        h = ctypes.c_void_p()
        _check(lib().svt_ctx_create(self.device, ctypes.c_void_p(self.workspace.data_ptr()),
                                    self.workspace.numel(), ctypes.byref(h)), "svt_ctx_create")
        self.handle = h
        self.tuning_import(tuning)
        for flag, value in getattr(self, "_debug", {}).items():
            _check(lib().svt_ctx_debug(self.handle, DEBUG[flag], int(value)), "svt_ctx_debug")

    def tuning_export(self) -> str:
        """The context's autotune results as JSON text (svt_tuning_export)."""
        n = ctypes.c_size_t(0)
        st = lib().svt_tuning_export(self.handle, None, 0, ctypes.byref(n))
        if st not in (OK, ERR_OOM):
            _check(st, "svt_tuning_export")
        buf = ctypes.create_string_buffer(n.value + 1)
        _check(lib().svt_tuning_export(self.handle, buf, n.value + 1, ctypes.byref(n)),
               "svt_tuning_export")
        return buf.value.decode()

    def tuning_import(self, text: str):
        """Merge autotune results written by tuning_export (svt_tuning_import); raises
        SVTError (ERR_INVALID) for text from another GPU or malformed text."""
        _check(lib().svt_tuning_import(self.handle, text.encode()), "svt_tuning_import")

    def save_tuning(self, path: str):
        with open(path, "w") as f:
            f.write(self.tuning_export())

    def load_tuning(self, path: str):
        with open(path) as f:
            self.tuning_import(f.read())

    def debug(self, flag: str, value: int):
        """Host-side fault injection and debug settings (svt_ctx_debug): "fail_plan" (the
        Nth plan build from now fails with ERR_OOM), "admit_delay_us" (serving admission
        delay), "wait_limit_ns" (device dependency-wait limit; 0 = default)."""
        _check(lib().svt_ctx_debug(self.handle, DEBUG[flag], int(value)), "svt_ctx_debug")
        self.__dict__.setdefault("_debug", {})[flag] = int(value)

    def cancel(self, ticket: int) -> int:
        """svt_serve_cancel: OK when the request is (or will be) cancelled, ERR_BUSY when
        its remaining work is already on the device, ERR_INVALID for unknown/completed."""
        return int(lib().svt_serve_cancel(self.handle, ctypes.c_uint64(ticket)))

    def serve_metrics(self, path):
        """Append one JSON line per retired serving request to `path` (None: stop)."""
        _check(lib().svt_serve_metrics(self.handle, None if path is None else str(path).encode()),
               "svt_serve_metrics")

    def polar(self, A, tau: float, out=None, status=None, stream=None, **opts):
        """Y = A_tau through svt_polar_ex (asynchronous on the current stream)."""
        import torch
        a_ptr, m, n, lda = _f32_matrix(A, "A")
        if out is None:
            out = torch.empty((m, n), dtype=torch.float32, device=A.device)
        y_ptr, ym, yn, ldy = _f32_matrix(out, "out")
        if (ym, yn) != (m, n):
            raise ValueError("out has the wrong shape")
        o = make_options(**opts)
        self.ensure_workspace(workspace_bytes(m, n, **opts))
        st_ptr = status.data_ptr() if status is not None else None
        _check(lib().svt_polar_ex(self.handle, ctypes.c_void_p(a_ptr), m, n, lda,
                                  ctypes.c_float(tau), ctypes.byref(o), ctypes.c_void_p(y_ptr),
                                  ldy, ctypes.c_void_p(st_ptr), ctypes.c_void_p(_stream_ptr(stream))),
               "svt_polar_ex")
        return out

    def polar_f64(self, A, tau: float, out=None, status=None, stream=None, **opts):
        """Y = A_tau in FP64 from the FP64 tier through svt_polar_f64 (asynchronous on
        the current stream). A: CUDA float32; out: CUDA float64 (allocated if None)."""
        import torch
        a_ptr, m, n, lda = _f32_matrix(A, "A")
        if out is None:
            out = torch.empty((m, n), dtype=torch.float64, device=A.device)
        if (not isinstance(out, torch.Tensor) or out.dtype != torch.float64 or not out.is_cuda
                or out.dim() != 2 or tuple(out.shape) != (m, n) or out.stride(1) != 1):
            raise ValueError("out must be a row-major CUDA float64 tensor of A's shape")
        opts = dict(opts, prec="fp64")
        o = make_options(**opts)
        self.ensure_workspace(workspace_bytes(m, n, **opts))
        st_ptr = status.data_ptr() if status is not None else None
        _check(lib().svt_polar_f64(self.handle, ctypes.c_void_p(a_ptr), m, n, lda,
                                   ctypes.c_float(tau), ctypes.byref(o),
                                   ctypes.c_void_p(out.data_ptr()), out.stride(0),
                                   ctypes.c_void_p(st_ptr), ctypes.c_void_p(_stream_ptr(stream))),
               "svt_polar_f64")
        return out

    def polar_fp8(self, A, tau: float, p_steps=(), s_steps=(), s_y2_only=False, out=None,
                  status=None, stream=None, **opts):
        """svt_polar_fp8: the BF16 tier with the listed steps on e4m3 operands (p_steps:
        the P chain's Y^2 products; s_steps: S-chain steps, all products or Y^2 only)."""
        import torch
        a_ptr, m, n, lda = _f32_matrix(A, "A")
        if out is None:
            out = torch.empty((m, n), dtype=torch.float32, device=A.device)
        y_ptr, ym, yn, ldy = _f32_matrix(out, "out")
        if (ym, yn) != (m, n):
            raise ValueError("out has the wrong shape")
        pol = fp8_policy(p_steps, s_steps, s_y2_only)
        o = make_options(**dict({"prec": "bf16"}, **opts))
        self.ensure_workspace(workspace_bytes_fp8(m, n, p_steps, s_steps, s_y2_only, **opts))
        st_ptr = status.data_ptr() if status is not None else None
        _check(lib().svt_polar_fp8(self.handle, ctypes.c_void_p(a_ptr), m, n, lda,
                                   ctypes.c_float(tau), ctypes.byref(o), ctypes.byref(pol),
                                   ctypes.c_void_p(y_ptr), ldy, ctypes.c_void_p(st_ptr),
                                   ctypes.c_void_p(_stream_ptr(stream))), "svt_polar_fp8")
        return out

    def debug_gemm_e4m3(self, L, R, D, K=None, tile=0, stream=None):
        """D = L R^T over the first K columns (default: all) of the e4m3 byte tensors
        L (M rows) and R (N rows) (svt_debug_gemm_e4m3)."""
        M, N = L.shape[0], R.shape[0]
        K = L.shape[1] if K is None else int(K)
        _check(lib().svt_debug_gemm_e4m3(self.handle, ctypes.c_void_p(L.data_ptr()),
                                         ctypes.c_void_p(R.data_ptr()), M, N, K, L.stride(0),
                                         R.stride(0), ctypes.c_void_p(D.data_ptr()), D.stride(0),
                                         int(tile), ctypes.c_void_p(_stream_ptr(stream))),
               "svt_debug_gemm_e4m3")
        return D

    def prox_grad_step(self, X, M, mask, lam: float, Z=None, step: float = 1.0, status=None,
                       stream=None, **opts):
        """One proximal-gradient step of nuclear-norm matrix completion through
        svt_prox_grad_step: Z = X + step P_Omega(M - X); X <- A_{step lam}(Z), in place.
        mask: CUDA uint8 tensor (nonzero = observed). Returns (X, Z)."""
        import torch
        x_ptr, m, n, ldx = _f32_matrix(X, "X")
        m_ptr, mm, mn, ldm = _f32_matrix(M, "M")
        if (mm, mn) != (m, n):
            raise ValueError("M has the wrong shape")
        if (not isinstance(mask, torch.Tensor) or mask.dtype != torch.uint8 or not mask.is_cuda
                or tuple(mask.shape) != (m, n) or mask.stride(1) != 1):
            raise ValueError("mask must be a row-major CUDA uint8 tensor of X's shape")
        if Z is None:
            Z = torch.empty((m, n), dtype=torch.float32, device=X.device)
        z_ptr, zm, zn, ldz = _f32_matrix(Z, "Z")
        if (zm, zn) != (m, n):
            raise ValueError("Z has the wrong shape")
        o = make_options(**opts)
        self.ensure_workspace(workspace_bytes(m, n, **opts))
        st_ptr = status.data_ptr() if status is not None else None
        _check(lib().svt_prox_grad_step(self.handle, ctypes.c_void_p(x_ptr), ldx,
                                        ctypes.c_void_p(m_ptr), ldm,
                                        ctypes.c_void_p(mask.data_ptr()), mask.stride(0),
                                        ctypes.c_void_p(z_ptr), ldz, m, n, ctypes.c_float(step),
                                        ctypes.c_float(lam), ctypes.byref(o),
                                        ctypes.c_void_p(st_ptr),
                                        ctypes.c_void_p(_stream_ptr(stream))),
               "svt_prox_grad_step")
        return X, Z

    def complete(self, M, mask, lam: float, steps: int, X=None, step: float = 1.0, status=None,
                 stream=None, **opts):
        """`steps` proximal-gradient steps from X (zeros if None); returns X."""
        import torch
        if X is None:
            X = torch.zeros_like(M)
        Z = torch.empty_like(M)
        for _ in range(int(steps)):
            self.prox_grad_step(X, M, mask, lam, Z=Z, step=step, status=status, stream=stream,
                                **opts)
        return X

    def complete_on_device(self, M, mask, lam: float, max_steps: int, lam0: float | None = None,
                           eta: float = 0.5, tol: float = 0.0, stage_steps: int = 0,
                           step: float = 1.0, X=None, Z=None, Xprev=None, stats=None,
                           stream=None, **opts):
        """Proximal-gradient completion as one device-resident loop (svt_complete):
        lambda continuation from lam0 (None: lam, one stage) by factor eta down to lam,
        stages ending when ||X_new - X_old||_F / ||P_Omega(M)||_F <= tol (the change
        measured against the data's scale, which stays meaningful when the iterate is
        zero) or after stage_steps steps, at most max_steps steps in all. X is the starting point (zeros if None)
        and receives the result. Returns (X, stats): stats is a CUDA byte tensor holding
        svt_completion_stats (read_completion_stats parses it)."""
        import torch
        m_ptr, m, n, ldm = _f32_matrix(M, "M")
        if (not isinstance(mask, torch.Tensor) or mask.dtype != torch.uint8 or not mask.is_cuda
                or tuple(mask.shape) != (m, n) or mask.stride(1) != 1):
            raise ValueError("mask must be a row-major CUDA uint8 tensor of M's shape")
        if X is None:
            X = torch.zeros((m, n), dtype=torch.float32, device=M.device)
        if Z is None:
            Z = torch.empty((m, n), dtype=torch.float32, device=M.device)
        if Xprev is None:
            Xprev = torch.empty((m, n), dtype=torch.float32, device=M.device)
        if stats is None:
            stats = torch.zeros(COMPLETION_STATS_BYTES, dtype=torch.uint8, device=M.device)
        if stats.numel() < COMPLETION_STATS_BYTES or stats.data_ptr() % 8:
            raise ValueError("stats must hold svt_completion_stats, 8-byte aligned")
        ptrs = []
        for t, name in ((X, "X"), (Z, "Z"), (Xprev, "Xprev")):
            p, tm, tn, ld = _f32_matrix(t, name)
            if (tm, tn) != (m, n):
                raise ValueError(f"{name} has the wrong shape")
            ptrs.append((p, ld))
        prm = CompletionParams(float(lam), float(lam if lam0 is None else lam0), float(eta),
                               float(step), float(tol), int(max_steps), int(stage_steps))
        o = make_options(**opts)
        self.ensure_workspace(workspace_bytes(m, n, **opts))
        _check(lib().svt_complete(self.handle, ctypes.c_void_p(ptrs[0][0]), ptrs[0][1],
                                  ctypes.c_void_p(m_ptr), ldm, ctypes.c_void_p(mask.data_ptr()),
                                  mask.stride(0), ctypes.c_void_p(ptrs[1][0]), ptrs[1][1],
                                  ctypes.c_void_p(ptrs[2][0]), ptrs[2][1], m, n,
                                  ctypes.byref(prm), ctypes.byref(o),
                                  ctypes.c_void_p(stats.data_ptr()),
                                  ctypes.c_void_p(_stream_ptr(stream))), "svt_complete")
        return X, stats

    def autotune_schedule(self, A, tau: float, target: float, max_iters: int = 32, stream=None,
                          **opts):
        """The fewest polynomial steps (and ell0) whose solve of A stays within `target` of
        an FP32-tier 32-step reference (svt_autotune_schedule). Returns
        {"iters", "ell0", "deviation"}."""
        import torch
        a_ptr, m, n, lda = _f32_matrix(A, "A")
        Y = torch.empty((m, n), dtype=torch.float32, device=A.device)
        R = torch.empty((m, n), dtype=torch.float32, device=A.device)
        o = make_options(**opts)
        ref, cand = dict(opts), dict(opts)
        ref.update(prec="fp32", iters=32)
        cand.update(iters=int(max_iters))
        self.ensure_workspace(max(workspace_bytes(m, n, **ref), workspace_bytes(m, n, **cand)))
        k, l0, dev = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        _check(lib().svt_autotune_schedule(self.handle, ctypes.c_void_p(a_ptr), m, n, lda,
                                           ctypes.c_float(tau), ctypes.byref(o), float(target),
                                           int(max_iters), ctypes.c_void_p(Y.data_ptr()), n,
                                           ctypes.c_void_p(R.data_ptr()), n, ctypes.byref(k),
                                           ctypes.byref(l0), ctypes.byref(dev),
                                           ctypes.c_void_p(_stream_ptr(stream))),
               "svt_autotune_schedule")
        return {"iters": k.value, "ell0": l0.value, "deviation": dev.value}

    def autotune(self, A, tau: float, out=None, reps: int = 2, stream=None, **opts):
        """Pick the product kernel's tile width per launch for this shape and options
        (svt_autotune); later polar() calls with them use the tuned plan."""
        import torch
        a_ptr, m, n, lda = _f32_matrix(A, "A")
        if out is None:
            out = torch.empty((m, n), dtype=torch.float32, device=A.device)
        y_ptr, _, _, ldy = _f32_matrix(out, "out")
        o = make_options(**opts)
        self.ensure_workspace(workspace_bytes(m, n, **opts))
        _check(lib().svt_autotune(self.handle, ctypes.c_void_p(a_ptr), m, n, lda,
                                  ctypes.c_float(tau), ctypes.byref(o), ctypes.c_void_p(y_ptr),
                                  ldy, int(reps), ctypes.c_void_p(_stream_ptr(stream))),
               "svt_autotune")
        return out

    def polar_host(self, A_host, tau: float, out_host=None, stream=None, **opts):
        """A_tau of a host (ideally pinned) FP32 matrix: copy in, solve, copy out.

        The device buffers are cached per shape; the copies and the solve are
        ordered on one stream, and the call returns after the result is on the host."""
        import torch
        if A_host.is_cuda or A_host.dim() != 2 or A_host.dtype != torch.float32:
            raise ValueError("A_host must be a 2-D float32 host tensor")
        key = tuple(A_host.shape)
        cache = self.__dict__.setdefault("_host_bufs", {})
        if key not in cache:
            dev = torch.device(f"cuda:{self.device}")
            cache[key] = (torch.empty(key, dtype=torch.float32, device=dev),
                          torch.empty(key, dtype=torch.float32, device=dev))
        a_dev, y_dev = cache[key]
        if out_host is None:
            out_host = torch.empty(key, dtype=torch.float32, pin_memory=True)
        a_dev.copy_(A_host, non_blocking=True)
        self.polar(a_dev, tau, out=y_dev, stream=stream, **opts)
        out_host.copy_(y_dev, non_blocking=True)
        return out_host

    def polar_basic(self, A, tau: float, iters: int, prec="bf16", out=None, status=None,
                    stream=None):
        """The svt_polar entry point (default options apart from iters and precision)."""
        import torch
        a_ptr, m, n, lda = _f32_matrix(A, "A")
        if out is None:
            out = torch.empty((m, n), dtype=torch.float32, device=A.device)
        y_ptr, _, _, ldy = _f32_matrix(out, "out")
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        self.ensure_workspace(workspace_bytes(m, n, prec=p))
        st_ptr = status.data_ptr() if status is not None else None
        _check(lib().svt_polar(self.handle, ctypes.c_void_p(a_ptr), m, n, lda, ctypes.c_float(tau),
                               int(iters), p, ctypes.c_void_p(y_ptr), ldy, ctypes.c_void_p(st_ptr),
                               ctypes.c_void_p(_stream_ptr(stream))), "svt_polar")
        return out

    def debug_gemm_bf16(self, nseg, L_hi, L_lo, R_hi, R_lo, D, sym=False, stream=None, tile=0):
        """D = sum of segment products (see svt_debug_gemm_bf16_ex)."""
        M, K = L_hi.shape
        N = R_hi.shape[0]
        ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else None)
        _check(lib().svt_debug_gemm_bf16_ex(self.handle, int(nseg), ptr(L_hi), ptr(L_lo),
                                            ptr(R_hi), ptr(R_lo), M, N, K, L_hi.stride(0),
                                            R_hi.stride(0), ptr(D), D.stride(0), 1 if sym else 0,
                                            int(tile), ctypes.c_void_p(_stream_ptr(stream))),
               "svt_debug_gemm_bf16_ex")
        return D

    def _matrix(self, A, tau, out, status, opts):
        import torch
        a_ptr, m, n, lda = _f32_matrix(A, "A")
        y_ptr, ym, yn, ldy = _f32_matrix(out, "out")
        if (ym, yn) != (m, n):
            raise ValueError("out has the wrong shape")
        mat = Matrix()
        mat.A, mat.m, mat.n, mat.lda = a_ptr, m, n, lda
        mat.tau = float(tau)
        mat.Y, mat.ldy = y_ptr, ldy
        mat.opt = make_options(**opts)
        mat.d_status = status.data_ptr() if status is not None else None
        return mat

    def batch(self, As, taus, outs=None, statuses=None, stream=None, opts=None):
        """A_tau for each matrix of the list through svt_batch (asynchronous)."""
        import torch
        count = len(As)
        if outs is None:
            outs = [torch.empty_like(a) for a in As]
        opts = opts or [{}] * count
        if isinstance(opts, dict):
            opts = [opts] * count
        arr = (Matrix * count)()
        for i in range(count):
            arr[i] = self._matrix(As[i], taus[i], outs[i],
                                  statuses[i] if statuses is not None else None, opts[i])
        need = ctypes.c_size_t(0)
        _check(lib().svt_batch_workspace_bytes(arr, count, ctypes.byref(need)),
               "svt_batch_workspace_bytes")
        self.ensure_workspace(int(need.value))
        _check(lib().svt_batch(self.handle, arr, count, ctypes.c_void_p(_stream_ptr(stream))),
               "svt_batch")
        return outs

    def autotune_batch(self, As, taus, outs=None, reps: int = 3, stream=None, opts=None):
        """svt_autotune_batch: the faster product tile width (128 or 256) of this grouped
        batch, from timed runs. Returns (tile, ms per batch); pass opts tile=<tile> to
        later batch() calls."""
        import torch
        count = len(As)
        if outs is None:
            outs = [torch.empty_like(a) for a in As]
        opts = opts or [{}] * count
        if isinstance(opts, dict):
            opts = [opts] * count
        arr = (Matrix * count)()
        for i in range(count):
            arr[i] = self._matrix(As[i], taus[i], outs[i], None, opts[i])
        need = ctypes.c_size_t(0)
        _check(lib().svt_batch_workspace_bytes(arr, count, ctypes.byref(need)),
               "svt_batch_workspace_bytes")
        self.ensure_workspace(int(need.value))
        tile, ms = ctypes.c_int(0), ctypes.c_double(0.0)
        _check(lib().svt_autotune_batch(self.handle, arr, count, int(reps),
                                        ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(tile),
                                        ctypes.byref(ms)), "svt_autotune_batch")
        return tile.value, ms.value

    def submit(self, A, tau, out, status=None, **opts) -> int:
        """Queue one serving request (svt_serve_submit); returns its ticket."""
        mat = self._matrix(A, tau, out, status, opts)
        t = ctypes.c_uint64(0)
        _check(lib().svt_serve_submit(self.handle, ctypes.byref(mat), ctypes.byref(t)),
               "svt_serve_submit")
        return int(t.value)

    def poll(self, ticket: int):
        """(status, latency_ms); status ERR_NOT_READY while pending."""
        lat = ctypes.c_double(0.0)
        st = lib().svt_serve_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(lat))
        return int(st), lat.value

    def release(self, ticket: int):
        return int(lib().svt_serve_release(self.handle, ctypes.c_uint64(ticket)))

    def sync(self, stream=None):
        _check(lib().svt_ctx_sync(self.handle, ctypes.c_void_p(_stream_ptr(stream))), "svt_ctx_sync")

    def launch_count(self) -> int:
        return int(lib().svt_ctx_launch_count(self.handle))

    def debug_wait_timeout(self, status, stream=None):
        """svt_debug_wait_timeout: a product-kernel launch whose bounded wait runs out;
        `status` (CUDA int32 tensor, zero) receives SVT_ERR_TIMEOUT."""
        _check(lib().svt_debug_wait_timeout(self.handle, ctypes.c_void_p(status.data_ptr()),
                                            ctypes.c_void_p(_stream_ptr(stream))),
               "svt_debug_wait_timeout")

    def profile(self, enable: bool = True):
        _check(lib().svt_ctx_profile(self.handle, 1 if enable else 0), "svt_ctx_profile")

    def profile_read(self):
        """(device ms, algorithmic flops, launches) of the tensor-core launches since the last reset."""
        ms, fl, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
        _check(lib().svt_ctx_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(fl),
                                          ctypes.byref(n)), "svt_ctx_profile_read")
        return ms.value, fl.value, int(n.value)

    def profile_read_ex(self):
        """(device ms, algorithmic flops, executed tensor flops, launches) of the
        tensor-core launches since the last reset (svt_ctx_profile_read_ex)."""
        ms, fl, tfl, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
        _check(lib().svt_ctx_profile_read_ex(self.handle, ctypes.byref(ms), ctypes.byref(fl),
                                             ctypes.byref(tfl), ctypes.byref(n)),
               "svt_ctx_profile_read_ex")
        return ms.value, fl.value, tfl.value, int(n.value)
