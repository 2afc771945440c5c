"""Thin Python binding of libfgk (``include/fgk.h``), same names as the C ABI.

Argument marshalling only: torch tensors are checked for device, dtype and
layout and passed to the library as raw pointers together with the current
torch CUDA stream.  Every step of the product and the solve runs inside
libfgk's CUDA kernels; there is no fallback path.  If the shared library is
missing, ``load()`` raises.
"""

from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfgk.so")

FGK_OK = 0
FGK_NOT_CONVERGED = 1
FGK_L1, FGK_PRODUCT = 0, 1
FGK_F64, FGK_F32, FGK_MIXED = 0, 1, 2

_STATUS = {
    0: "FGK_OK", 1: "FGK_NOT_CONVERGED", -1: "FGK_ERR_INVALID", -2: "FGK_ERR_NONFINITE", -3: "FGK_ERR_OOM",
    -4: "FGK_ERR_CUDA", -5: "FGK_ERR_BREAKDOWN", -6: "FGK_ERR_TIMEOUT", -7: "FGK_ERR_INTERNAL",
}


class FgkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = _STATUS.get(code, str(code))


class fgk_cg_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("refinements", ctypes.c_int32), ("mvm_f32", ctypes.c_int32),
                ("mvm_f64", ctypes.c_int32), ("max_true_resid", ctypes.c_double),
                ("true_resid", ctypes.POINTER(ctypes.c_double)), ("restarts", ctypes.c_int32),
                ("fp64_switch", ctypes.c_int32)]


class fgk_precond_report(ctypes.Structure):
    _fields_ = [("rank_requested", ctypes.c_int32), ("rank", ctypes.c_int32), ("sigma2", ctypes.c_double),
                ("trace_resid", ctypes.c_double), ("logdet", ctypes.c_double), ("device_bytes", ctypes.c_size_t)]


class fgk_slq_report(ctypes.Structure):
    _fields_ = [("logdet", ctypes.c_double), ("logdet_precond", ctypes.c_double), ("steps_max", ctypes.c_int32),
                ("solve_status", ctypes.c_int32), ("max_true_resid", ctypes.c_double)]


class fgk_grad_report(ctypes.Structure):
    _fields_ = [("yAy", ctypes.c_double), ("alpha_sq", ctypes.c_double), ("max_true_resid", ctypes.c_double),
                ("iterations", ctypes.c_int32), ("solve_status", ctypes.c_int32), ("n_grad", ctypes.c_int32)]


class fgk_plan_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("d", ctypes.c_int32), ("two_nu", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("L", ctypes.c_int32), ("n_levels", ctypes.c_int32), ("outscale2", ctypes.c_double),
                ("ell", ctypes.c_double * 3), ("device_bytes", ctypes.c_size_t)]


EXPORTS = ["fgk_set_allocator", "fgk_build", "fgk_matvec", "fgk_matvec_dlogell", "fgk_matvec_q", "fgk_matvec_q_noalloc", "fgk_cg_solve", "fgk_bytes_estimate",
           "fgk_destroy", "fgk_last_error", "fgk_kernel_launches", "fgk_scan_timing", "fgk_get_info",
           "fgk_get_permutation", "fgk_get_level", "fgk_batch_create", "fgk_batch_layout", "fgk_batch_matvec_q",
           "fgk_batch_cg_solve", "fgk_batch_destroy", "fgk_precond_build", "fgk_precond_info",
           "fgk_precond_factor", "fgk_precond_apply", "fgk_precond_destroy", "fgk_cg_solve_pc",
           "fgk_minres_solve", "fgk_shard_moments", "fgk_shard_fixup", "fgk_fma_rate",
           "fgk_kernel_timing", "fgk_predict", "fgk_batch_cg_solve_pc", "fgk_precond_sample", "fgk_slq_logdet",
           "fgk_lanczos_logquad", "fgk_loglik_grad"]

_lock = threading.Lock()
_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libfgk.so (built by ``paper_2508_01864_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise FileNotFoundError(f"libfgk.so not found at {p}; run paper_2508_01864_gb300.build.build() first")
        lib = ctypes.CDLL(p)
        vp, i64, i32, dbl, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        lib.fgk_set_allocator.argtypes = [vp, vp, vp]
        lib.fgk_set_allocator.restype = i32
        lib.fgk_build.argtypes = [vp, i64, i32, i32, ctypes.POINTER(dbl), dbl, i32, vp, ctypes.POINTER(vp)]
        lib.fgk_build.restype = i32
        lib.fgk_matvec.argtypes = [vp, vp, i32, vp, i32, vp]
        lib.fgk_matvec.restype = i32
        lib.fgk_matvec_dlogell.argtypes = [vp, vp, i32, vp, i32, i32, vp]
        lib.fgk_matvec_dlogell.restype = i32
        lib.fgk_matvec_q.argtypes = [vp, vp, i32, vp, i32, vp]
        lib.fgk_matvec_q.restype = i32
        lib.fgk_matvec_q_noalloc.argtypes = [vp, vp, i32, vp, i32, vp]
        lib.fgk_matvec_q_noalloc.restype = i32
        lib.fgk_kernel_launches.argtypes = []
        lib.fgk_kernel_launches.restype = ctypes.c_uint64
        lib.fgk_scan_timing.argtypes = [i32, ctypes.POINTER(dbl), ctypes.POINTER(i64)]
        lib.fgk_scan_timing.restype = i32
        lib.fgk_kernel_timing.argtypes = [i32, i32, ctypes.POINTER(dbl), ctypes.POINTER(i64)]
        lib.fgk_kernel_timing.restype = i32
        lib.fgk_cg_solve.argtypes = [vp, vp, i32, dbl, vp, i32, dbl, i32, i32, vp, vp, ctypes.POINTER(fgk_cg_info),
                                     vp]
        lib.fgk_cg_solve.restype = i32
        lib.fgk_bytes_estimate.argtypes = [i64, i32, i32, i32, i32]
        lib.fgk_bytes_estimate.restype = sz
        lib.fgk_destroy.argtypes = [vp]
        lib.fgk_destroy.restype = i32
        lib.fgk_last_error.argtypes = []
        lib.fgk_last_error.restype = ctypes.c_char_p
        lib.fgk_get_info.argtypes = [vp, ctypes.POINTER(fgk_plan_info)]
        lib.fgk_get_info.restype = i32
        lib.fgk_get_permutation.argtypes = [vp, i32, vp]
        lib.fgk_get_permutation.restype = i32
        lib.fgk_get_level.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(i64)]
        lib.fgk_get_level.restype = i32
        lib.fgk_batch_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, vp, ctypes.POINTER(vp)]
        lib.fgk_batch_create.restype = i32
        lib.fgk_batch_layout.argtypes = [vp, ctypes.POINTER(i64)]
        lib.fgk_batch_layout.restype = i32
        lib.fgk_batch_matvec_q.argtypes = [vp, vp, vp, vp]
        lib.fgk_batch_matvec_q.restype = i32
        lib.fgk_batch_cg_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(dbl), dbl, i32, ctypes.POINTER(vp),
                                           ctypes.POINTER(fgk_cg_info), vp]
        lib.fgk_batch_cg_solve.restype = i32
        lib.fgk_batch_cg_solve_pc.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(dbl), dbl,
                                              i32, ctypes.POINTER(vp), ctypes.POINTER(fgk_cg_info), vp]
        lib.fgk_batch_cg_solve_pc.restype = i32
        lib.fgk_batch_destroy.argtypes = [vp]
        lib.fgk_batch_destroy.restype = i32
        lib.fgk_precond_build.argtypes = [vp, i32, dbl, vp, ctypes.POINTER(vp)]
        lib.fgk_precond_build.restype = i32
        lib.fgk_precond_info.argtypes = [vp, ctypes.POINTER(fgk_precond_report), ctypes.POINTER(i64)]
        lib.fgk_precond_info.restype = i32
        lib.fgk_precond_factor.argtypes = [vp, vp, vp]
        lib.fgk_precond_factor.restype = i32
        lib.fgk_precond_apply.argtypes = [vp, vp, i32, vp, vp]
        lib.fgk_precond_apply.restype = i32
        lib.fgk_precond_sample.argtypes = [vp, vp, vp, i32, vp, vp]
        lib.fgk_precond_sample.restype = i32
        lib.fgk_slq_logdet.argtypes = [vp, vp, dbl, vp, i32, i32, dbl, vp, ctypes.POINTER(dbl), ctypes.POINTER(i32),
                                       ctypes.POINTER(fgk_slq_report), vp]
        lib.fgk_slq_logdet.restype = i32
        lib.fgk_lanczos_logquad.argtypes = [ctypes.POINTER(dbl), ctypes.POINTER(dbl), i32, ctypes.POINTER(dbl)]
        lib.fgk_lanczos_logquad.restype = i32
        lib.fgk_loglik_grad.argtypes = [vp, vp, dbl, vp, vp, i32, dbl, i32, i32, ctypes.POINTER(dbl),
                                        ctypes.POINTER(fgk_grad_report), vp]
        lib.fgk_loglik_grad.restype = i32
        lib.fgk_precond_destroy.argtypes = [vp]
        lib.fgk_precond_destroy.restype = i32
        lib.fgk_cg_solve_pc.argtypes = [vp, vp, vp, i32, dbl, vp, i32, dbl, i32, i32, vp, vp,
                                        ctypes.POINTER(fgk_cg_info), vp]
        lib.fgk_cg_solve_pc.restype = i32
        lib.fgk_minres_solve.argtypes = [vp, vp, i32, dbl, dbl, i32, vp, vp, vp]
        lib.fgk_minres_solve.restype = i32
        lib.fgk_shard_moments.argtypes = [vp, vp, i32, vp, vp]
        lib.fgk_shard_moments.restype = i32
        lib.fgk_shard_fixup.argtypes = [vp, vp, i32, vp, vp]
        lib.fgk_shard_fixup.restype = i32
        lib.fgk_fma_rate.argtypes = [i32, i32, ctypes.POINTER(dbl), vp]
        lib.fgk_fma_rate.restype = i32
        lib.fgk_predict.argtypes = [vp, vp, i32, vp, i64, vp, i32, vp, i32, vp, vp]
        lib.fgk_predict.restype = i32
        _lib = lib
        return lib


def _check(rc: int, allow_soft: bool = False) -> int:
    if rc == FGK_OK or (allow_soft and rc == FGK_NOT_CONVERGED):
        return rc
    msg = load().fgk_last_error()
    raise FgkError(rc, msg.decode() if msg else "")


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _two_nu(nu) -> int:
    t = int(round(2 * float(nu)))
    if t not in (1, 3, 5, 7, 9):
        raise ValueError(f"nu must be 1/2, 3/2, 5/2, 7/2 or 9/2, got {nu}")
    return t


def _kind(kind) -> int:
    if isinstance(kind, str):
        return {"l1": FGK_L1, "product": FGK_PRODUCT}[kind.lower()]
    return int(kind)


def _dev_f64_2d(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    if t.dim() == 1:
        t = t.unsqueeze(1)
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous (row-major)")
    return t


# The library receives bare pointers and cannot see a buffer's size: every
# row count, column count and output buffer is checked here, before the call,
# so that a mis-shaped tensor raises instead of being read or written past
# its end on the device.
def _rows(t: torch.Tensor, n: int, name: str, what: str = "the plan's points") -> None:
    if t.shape[0] != n:
        raise ValueError(f"{name} has {t.shape[0]} rows, {what} are {n}")


def _out_for(out, like: torch.Tensor, name: str = "out") -> torch.Tensor:
    """The caller's output buffer for a result shaped like ``like`` (2-D):
    same device and dtype, contiguous, the same shape (or a vector when the
    result has one column); returned as a view of like's shape.  A new
    tensor when ``out`` is None."""
    if out is None:
        return torch.empty_like(like)
    if (not isinstance(out, torch.Tensor) or out.device != like.device or out.dtype != like.dtype
            or not out.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous {like.dtype} tensor on {like.device}")
    vec = out.dim() == 1 and like.shape[1] == 1 and out.shape[0] == like.shape[0]
    if tuple(out.shape) != tuple(like.shape) and not vec:
        raise ValueError(f"{name} has shape {tuple(out.shape)}, the result {tuple(like.shape)}")
    return out.view(like.shape)


@dataclass
class Handle:
    ptr: int
    N: int
    d: int
    two_nu: int
    kind: int

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        fgk_destroy(self)


def fgk_build(X: torch.Tensor, nu, ell, outscale2: float = 1.0, kind="l1", stream=None) -> Handle:
    """Build the cached sort and dominance structure (see include/fgk.h)."""
    lib = load()
    X = _dev_f64_2d(X, "X")
    N, d = X.shape
    ellv = [float(e) for e in torch.as_tensor(ell, dtype=torch.float64).reshape(-1).broadcast_to((d,)).tolist()]
    ell_arr = (ctypes.c_double * d)(*ellv)
    out = ctypes.c_void_p()
    _check(lib.fgk_build(X.data_ptr(), N, d, _two_nu(nu), ell_arr, float(outscale2), _kind(kind), _stream(stream),
                         ctypes.byref(out)))
    return Handle(out.value, N, d, _two_nu(nu), _kind(kind))


def fgk_matvec(h: Handle, V: torch.Tensor, precision="f64", out: torch.Tensor | None = None, stream=None):
    """Y = K V (asynchronous on the stream)."""
    lib = load()
    prec = {"f64": FGK_F64, "f32": FGK_F32}[precision] if isinstance(precision, str) else int(precision)
    dt = torch.float64 if prec == FGK_F64 else torch.float32
    if not V.is_cuda or V.dtype != dt or not V.is_contiguous():
        raise TypeError(f"V must be a contiguous CUDA {dt} tensor")
    squeeze = V.dim() == 1
    V2 = V.unsqueeze(1) if squeeze else V
    _rows(V2, h.N, "V")
    out = _out_for(out, V2)
    _check(lib.fgk_matvec(h.ptr, V2.data_ptr(), V2.shape[1], out.data_ptr(), prec, _stream(stream)))
    return out.squeeze(1) if squeeze else out


def fgk_matvec_dlogell(h: Handle, V: torch.Tensor, dim: int = -1, precision="f64", out: torch.Tensor | None = None,
                       stream=None):
    """Y = (dK / d log ell_dim) V (dim = -1: all lengthscales scaled
    together); see include/fgk.h.  Asynchronous on the stream."""
    lib = load()
    prec = {"f64": FGK_F64, "f32": FGK_F32}[precision] if isinstance(precision, str) else int(precision)
    dt = torch.float64 if prec == FGK_F64 else torch.float32
    if not V.is_cuda or V.dtype != dt or not V.is_contiguous():
        raise TypeError(f"V must be a contiguous CUDA {dt} tensor")
    squeeze = V.dim() == 1
    V2 = V.unsqueeze(1) if squeeze else V
    _rows(V2, h.N, "V")
    out = _out_for(out, V2)
    _check(lib.fgk_matvec_dlogell(h.ptr, V2.data_ptr(), V2.shape[1], out.data_ptr(), int(dim), prec,
                                  _stream(stream)))
    return out.squeeze(1) if squeeze else out


def fgk_matvec_q(h: Handle, Vq: torch.Tensor, precision="f32", out: torch.Tensor | None = None, stream=None):
    """Y = K V with rows in the plan's internal order (see include/fgk.h)."""
    lib = load()
    prec = {"f64": FGK_F64, "f32": FGK_F32}[precision] if isinstance(precision, str) else int(precision)
    dt = torch.float64 if prec == FGK_F64 else torch.float32
    if not Vq.is_cuda or Vq.dtype != dt or not Vq.is_contiguous():
        raise TypeError(f"Vq must be a contiguous CUDA {dt} tensor")
    V2 = Vq.unsqueeze(1) if Vq.dim() == 1 else Vq
    _rows(V2, h.N, "Vq")
    out = _out_for(out, V2)
    _check(lib.fgk_matvec_q(h.ptr, V2.data_ptr(), V2.shape[1], out.data_ptr(), prec, _stream(stream)))
    return out


def fgk_matvec_q_noalloc(h: Handle, Vq: torch.Tensor, out: torch.Tensor, precision="f32", stream=None):
    """fgk_matvec_q without any device allocation: scratch in the library's
    fixed array, output into the caller's ``out``."""
    lib = load()
    prec = {"f64": FGK_F64, "f32": FGK_F32}[precision] if isinstance(precision, str) else int(precision)
    dt = torch.float64 if prec == FGK_F64 else torch.float32
    if not Vq.is_cuda or Vq.dtype != dt or not Vq.is_contiguous():
        raise TypeError(f"Vq must be a contiguous CUDA {dt} tensor")
    if out is None:
        raise TypeError("out is required (this call allocates nothing)")
    V2 = Vq.unsqueeze(1) if Vq.dim() == 1 else Vq
    _rows(V2, h.N, "Vq")
    out2 = _out_for(out, V2)
    _check(lib.fgk_matvec_q_noalloc(h.ptr, V2.data_ptr(), V2.shape[1], out2.data_ptr(), prec, _stream(stream)))
    return out


def fgk_kernel_launches() -> int:
    return int(load().fgk_kernel_launches())


FGK_TIMED_SCAN_OUT, FGK_TIMED_PC_LTR, FGK_TIMED_PC_APPLY = 0, 1, 2


def fgk_kernel_timing(kernel: int, enable: int = -1):
    """(total ms, launches) of a timed kernel; enable 1 resets and starts, 0 stops."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().fgk_kernel_timing(int(kernel), int(enable), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def fgk_scan_timing(enable: int = -1):
    """Start (1), stop (0) or read (-1) event timing of the main scan kernel;
    returns (total_ms, launches)."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().fgk_scan_timing(int(enable), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def fgk_fma_rate(precision="f32", reps: int = 5, stream=None) -> float:
    """Measured FMA throughput of the current device in FLOP/s (2 per FMA)."""
    prec = {"f64": FGK_F64, "f32": FGK_F32}[precision] if isinstance(precision, str) else int(precision)
    out = ctypes.c_double()
    _check(load().fgk_fma_rate(prec, int(reps), ctypes.byref(out), _stream(stream)))
    return out.value


def fgk_shard_moments(h: Handle, V: torch.Tensor, stream=None):
    """(x'_first, x'_last, M) of this shard (d = 1 plan): M[r, dir, q] as
    fgk_shard_moments documents (numpy, FP64)."""
    lib = load()
    V2 = _dev_f64_2d(V, "V")
    _rows(V2, h.N, "V")
    nrhs = V2.shape[1]
    if nrhs > 64:
        raise ValueError(f"at most 64 columns, got {nrhs}")
    P = (h.two_nu + 1) // 2
    out = np.zeros(2 + 2 * nrhs * P)
    _check(lib.fgk_shard_moments(h.ptr, V2.data_ptr(), nrhs, out.ctypes.data, _stream(stream)))
    return float(out[0]), float(out[1]), out[2:].reshape(nrhs, 2, P)


def fgk_shard_fixup(h: Handle, carry, Y: torch.Tensor, stream=None):
    """Y += the other shards' contributions, from carry[r, dir, q] (dir 0:
    the points before this shard, anchored at its first point; dir 1: after,
    at its last)."""
    lib = load()
    Y2 = _dev_f64_2d(Y, "Y")
    _rows(Y2, h.N, "Y")
    nrhs = Y2.shape[1]
    P = (h.two_nu + 1) // 2
    c = np.ascontiguousarray(carry, dtype=np.float64)
    if c.shape != (nrhs, 2, P):
        raise ValueError(f"carry must have shape {(nrhs, 2, P)}, got {c.shape}")
    _check(lib.fgk_shard_fixup(h.ptr, c.ctypes.data, nrhs, Y2.data_ptr(), _stream(stream)))
    return Y


def fgk_minres_solve(h: Handle, y: torch.Tensor, sigma2: float, tol: float = 1e-8, maxit: int = 100000,
                     stream=None):
    """Solve (K + sigma2 I) alpha = y by MINRES (symmetric, possibly
    indefinite: the L1 kernel at nu >= 3/2, d >= 2).  Returns (alpha, info
    dict, status) with status FGK_OK or FGK_NOT_CONVERGED; errors raise."""
    lib = load()
    y2 = _dev_f64_2d(y, "y")
    _rows(y2, h.N, "y")
    nrhs = y2.shape[1]
    if nrhs > 64:
        raise ValueError(f"fgk_minres_solve takes at most 64 columns, got {nrhs}")
    alpha = torch.empty_like(y2)
    res = (ctypes.c_double * nrhs)()
    info = fgk_cg_info()
    info.true_resid = ctypes.cast(res, ctypes.POINTER(ctypes.c_double))
    rc = lib.fgk_minres_solve(h.ptr, y2.data_ptr(), nrhs, float(sigma2), float(tol), int(maxit), alpha.data_ptr(),
                              ctypes.byref(info), _stream(stream))
    d = {"iterations": info.iterations, "restarts": info.restarts, "mvm_f64": info.mvm_f64,
         "max_true_resid": info.max_true_resid, "true_resid": list(res)}
    try:
        _check(rc, allow_soft=True)
    except FgkError as e:
        e.info = d
        raise
    if y.dim() == 1:
        alpha = alpha.squeeze(1)
    return alpha, d, rc


def fgk_cg_solve(h: Handle, y: torch.Tensor, sigma2: float, H: torch.Tensor | None = None, L: int = 0,
                 tol: float = 1e-8, maxit: int = 100000, mode="f64", stream=None, want_beta: bool = True,
                 precond=None):
    """Solve (K + sigma2 I) alpha = y, optionally with GLS fixed effects and
    a preconditioner from ``fgk_precond_build`` (calls fgk_cg_solve_pc).

    Returns (alpha, beta or None, info dict, status) where status is FGK_OK or
    FGK_NOT_CONVERGED; errors raise FgkError."""
    lib = load()
    y2 = _dev_f64_2d(y, "y")
    _rows(y2, h.N, "y")
    nrhs = y2.shape[1]
    m = {"f64": FGK_F64, "mixed": FGK_MIXED}[mode] if isinstance(mode, str) else int(mode)
    Hp = 0
    if H is not None:
        H = _dev_f64_2d(H, "H")
        _rows(H, h.N, "H")
        L = H.shape[1]
        Hp = H.data_ptr()
    Leff = L if L >= 0 else 1 + h.d
    alpha = torch.empty_like(y2)
    beta = torch.empty((Leff, nrhs), dtype=torch.float64, device=y2.device) if (Leff > 0 and want_beta) else None
    ncols = nrhs + max(Leff, 0)
    res = (ctypes.c_double * ncols)()
    info = fgk_cg_info()
    info.true_resid = ctypes.cast(res, ctypes.POINTER(ctypes.c_double))
    if precond is None:
        rc = lib.fgk_cg_solve(h.ptr, y2.data_ptr(), nrhs, float(sigma2), Hp, int(L), float(tol), int(maxit), m,
                              alpha.data_ptr(), beta.data_ptr() if beta is not None else 0, ctypes.byref(info),
                              _stream(stream))
    else:
        rc = lib.fgk_cg_solve_pc(h.ptr, precond.ptr, y2.data_ptr(), nrhs, float(sigma2), Hp, int(L), float(tol),
                                 int(maxit), m, alpha.data_ptr(), beta.data_ptr() if beta is not None else 0,
                                 ctypes.byref(info), _stream(stream))
    d = {"iterations": info.iterations, "refinements": info.refinements, "mvm_f32": info.mvm_f32,
         "mvm_f64": info.mvm_f64, "max_true_resid": info.max_true_resid, "true_resid": list(res),
         "restarts": info.restarts, "fp64_switch": info.fp64_switch}
    try:
        _check(rc, allow_soft=True)
    except FgkError as e:
        e.info = d  # the solve's report, filled on every return
        raise
    if y.dim() == 1:
        alpha = alpha.squeeze(1)
    return alpha, beta, d, rc


@dataclass
class Precond:
    ptr: int
    handle: Handle
    sigma2: float
    rank: int = 0  # the realised rank k (the factor's columns)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        fgk_precond_destroy(self)


def fgk_precond_build(h: Handle, rank: int, sigma2: float, stream=None) -> Precond:
    """Rank-k pivoted-Cholesky preconditioner P = L L^T + sigma2 I of the plan's K."""
    out = ctypes.c_void_p()
    lib = load()
    _check(lib.fgk_precond_build(h.ptr, int(rank), float(sigma2), _stream(stream), ctypes.byref(out)))
    rep = fgk_precond_report()
    rc = lib.fgk_precond_info(out.value, ctypes.byref(rep), None)
    if rc != FGK_OK:
        lib.fgk_precond_destroy(out.value)
        _check(rc)
    return Precond(out.value, h, float(sigma2), int(rep.rank))


def fgk_precond_info(pc: Precond) -> dict:
    rep = fgk_precond_report()
    piv = (ctypes.c_int64 * max(1, min(int(pc.handle.N), 1024)))()
    _check(load().fgk_precond_info(pc.ptr, ctypes.byref(rep), piv))
    return {"rank_requested": rep.rank_requested, "rank": rep.rank, "sigma2": rep.sigma2,
            "trace_resid": rep.trace_resid, "logdet": rep.logdet, "device_bytes": rep.device_bytes,
            "pivots": list(piv)[:rep.rank]}


def fgk_precond_factor(pc: Precond, stream=None) -> torch.Tensor:
    """L (N x k FP64, the caller's point order)."""
    k = fgk_precond_info(pc)["rank"]
    L = torch.zeros((pc.handle.N, max(k, 0)), dtype=torch.float64, device="cuda")
    if k > 0:
        _check(load().fgk_precond_factor(pc.ptr, L.data_ptr(), _stream(stream)))
    return L


def fgk_precond_apply(pc: Precond, R: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Z = P^{-1} R (Woodbury), R: N x ncols FP64 CUDA tensor in the caller's order."""
    R2 = _dev_f64_2d(R, "R")
    _rows(R2, pc.handle.N, "R")
    Z = _out_for(out, R2)
    _check(load().fgk_precond_apply(pc.ptr, R2.data_ptr(), R2.shape[1], Z.data_ptr(), _stream(stream)))
    return Z.squeeze(1) if R.dim() == 1 else Z


def fgk_precond_sample(pc: Precond, E_r: torch.Tensor, E_n: torch.Tensor, stream=None) -> torch.Tensor:
    """Probes B = L_hi E_r + sigma E_n ~ N(0, P) from the caller's standard
    normal draws E_r (k x nprobe) and E_n (N x nprobe), FP64 CUDA tensors."""
    En = _dev_f64_2d(E_n, "E_n")
    _rows(En, pc.handle.N, "E_n")
    if pc.rank > 0:
        Er = _dev_f64_2d(E_r, "E_r")
        _rows(Er, pc.rank, "E_r", "the preconditioner's rank")
        if Er.shape[1] != En.shape[1]:
            raise ValueError(f"E_r has {Er.shape[1]} columns, E_n {En.shape[1]}")
    else:
        Er = E_r
    B = torch.empty_like(En)
    _check(load().fgk_precond_sample(pc.ptr, Er.data_ptr() if pc.rank > 0 else None, En.data_ptr(), En.shape[1],
                                     B.data_ptr(), _stream(stream)))
    return B


def fgk_slq_logdet(h: Handle, B: torch.Tensor, sigma2: float, m: int, tol: float = 1e-8, pc: Precond | None = None,
                   want_solves: bool = False, stream=None) -> dict:
    """log det(K + sigma2 I) by stochastic Lanczos quadrature with the probe
    columns of B (N x nprobe FP64 CUDA tensor, caller's order); see
    include/fgk.h.  Returns the estimate, log det P, per-probe quadrature
    values and Lanczos steps, and (want_solves) the solves (K + sigma2 I)^-1 B."""
    B2 = _dev_f64_2d(B, "B")
    _rows(B2, h.N, "B")
    nprobe = B2.shape[1]
    X = torch.empty_like(B2) if want_solves else None
    quad = (ctypes.c_double * nprobe)()
    steps = (ctypes.c_int32 * nprobe)()
    rep = fgk_slq_report()
    _check(load().fgk_slq_logdet(h.ptr, pc.ptr if pc is not None else None, float(sigma2), B2.data_ptr(), nprobe,
                                 int(m), float(tol), X.data_ptr() if X is not None else None, quad, steps,
                                 ctypes.byref(rep), _stream(stream)))
    return {"logdet": rep.logdet, "logdet_precond": rep.logdet_precond, "steps_max": rep.steps_max,
            "solve_status": rep.solve_status, "max_true_resid": rep.max_true_resid, "quad": list(quad),
            "steps": list(steps), "X": X}


def fgk_loglik_grad(h: Handle, y: torch.Tensor, B: torch.Tensor, sigma2: float, tol: float = 1e-8,
                    maxit: int = 20000, mode: str = "mixed", pc: Precond | None = None, stream=None) -> dict:
    """The log-likelihood gradient in (log ell..., log varsigma^2, log sigma^2)
    with Hutchinson probes B; see include/fgk.h."""
    y1 = _dev_f64_2d(y, "y")
    _rows(y1, h.N, "y")
    if y1.shape[1] != 1:
        raise ValueError("y must be one column")
    B2 = _dev_f64_2d(B, "B") if B is not None else None
    if B2 is not None:
        _rows(B2, h.N, "B")
    g = (ctypes.c_double * 8)()
    rep = fgk_grad_report()
    m = FGK_MIXED if mode == "mixed" else FGK_F64
    _check(load().fgk_loglik_grad(h.ptr, pc.ptr if pc is not None else None, float(sigma2), y1.data_ptr(),
                                  B2.data_ptr() if B2 is not None else None, B2.shape[1] if B2 is not None else 0,
                                  float(tol), int(maxit), m, g, ctypes.byref(rep), _stream(stream)))
    return {"grad": list(g)[: rep.n_grad], "yAy": rep.yAy, "alpha_sq": rep.alpha_sq,
            "max_true_resid": rep.max_true_resid, "iterations": rep.iterations, "solve_status": rep.solve_status}


def fgk_lanczos_logquad(alpha, beta) -> float:
    """e_1^T log(T) e_1 of the Lanczos matrix built from CG coefficients
    (host computation, no GPU)."""
    a = (ctypes.c_double * len(alpha))(*[float(x) for x in alpha])
    b = (ctypes.c_double * max(1, len(beta)))(*([float(x) for x in beta] or [0.0]))
    out = ctypes.c_double()
    _check(load().fgk_lanczos_logquad(a, b, len(alpha), ctypes.byref(out)))
    return out.value


def fgk_precond_destroy(pc: Precond) -> None:
    if pc is not None and pc.ptr:
        _check(load().fgk_precond_destroy(pc.ptr))
        pc.ptr = 0


def fgk_predict(h: Handle, alpha: torch.Tensor, Z: torch.Tensor, beta: torch.Tensor | None = None,
                HZ: torch.Tensor | None = None, L: int = 0, precision="f64", stream=None) -> torch.Tensor:
    """Posterior mean at the rows of Z (eq. gp_mean): K(Z, X) alpha (+ h(Z) beta)."""
    a2 = _dev_f64_2d(alpha, "alpha")
    _rows(a2, h.N, "alpha")
    Z2 = _dev_f64_2d(Z, "Z")
    if Z2.shape[1] != h.d:
        raise ValueError("Z must have d columns")
    prec = {"f64": FGK_F64, "f32": FGK_F32}[precision] if isinstance(precision, str) else int(precision)
    Hp, bp = 0, 0
    if HZ is not None:
        HZ = _dev_f64_2d(HZ, "HZ")
        _rows(HZ, Z2.shape[0], "HZ", "the rows of Z")
        L = HZ.shape[1]
        Hp = HZ.data_ptr()
    if L != 0:
        if beta is None:
            raise ValueError("fixed effects need beta")
        beta = _dev_f64_2d(beta, "beta")
        Leff = L if L > 0 else 1 + h.d
        if tuple(beta.shape) != (Leff, a2.shape[1]):
            raise ValueError(f"beta has shape {tuple(beta.shape)}, expected {(Leff, a2.shape[1])}")
        bp = beta.data_ptr()
    out = torch.empty((Z2.shape[0], a2.shape[1]), dtype=torch.float64, device=a2.device)
    _check(load().fgk_predict(h.ptr, a2.data_ptr(), a2.shape[1], Z2.data_ptr(), Z2.shape[0], Hp, int(L), bp, prec,
                              out.data_ptr(), _stream(stream)))
    return out.squeeze(1) if alpha.dim() == 1 else out


def fgk_bytes_estimate(N: int, d: int, nu, kind="l1", nrhs: int = 1) -> int:
    return int(load().fgk_bytes_estimate(int(N), int(d), _two_nu(nu), _kind(kind), int(nrhs)))


def fgk_destroy(h: Handle) -> None:
    if h is not None and h.ptr:
        _check(load().fgk_destroy(h.ptr))
        h.ptr = 0


def fgk_last_error() -> str:
    m = load().fgk_last_error()
    return m.decode() if m else ""


def fgk_get_info(h: Handle) -> dict:
    info = fgk_plan_info()
    _check(load().fgk_get_info(h.ptr, ctypes.byref(info)))
    return {"N": info.N, "d": info.d, "two_nu": info.two_nu, "kind": info.kind, "L": info.L,
            "n_levels": info.n_levels, "outscale2": info.outscale2, "ell": list(info.ell)[:info.d],
            "device_bytes": info.device_bytes}


def fgk_get_permutation(h: Handle, dim: int):
    import numpy as np

    perm = np.empty(h.N, dtype=np.int32)
    _check(load().fgk_get_permutation(h.ptr, int(dim), perm.ctypes.data))
    return perm


def fgk_get_level(h: Handle, level: int) -> dict:
    import numpy as np

    N, nof = h.N, max(h.d - 1, 0)
    q = np.empty(N, dtype=np.uint32)
    roles = np.empty(N, dtype=np.uint8)
    dl64 = np.empty(N, dtype=np.float64)
    dl32 = np.empty(N, dtype=np.float32)
    off64 = np.empty((N, max(nof, 1)), dtype=np.float64)
    off32 = np.empty((N, max(nof, 1)), dtype=np.float32)
    S = ctypes.c_int64()
    _check(load().fgk_get_level(h.ptr, int(level), q.ctypes.data, roles.ctypes.data, dl64.ctypes.data,
                                dl32.ctypes.data, off64.ctypes.data if nof else 0, off32.ctypes.data if nof else 0,
                                ctypes.byref(S)))
    out = {"S": int(S.value), "q": q, "roles": roles, "dl64": dl64, "dl32": dl32}
    if nof:
        out["off64"] = off64[:, :nof]
        out["off32"] = off32[:, :nof]
    return out


# ------------------------------------------------------------ batches
@dataclass
class Batch:
    ptr: int
    handles: list
    nrhs: int
    rows: list  # packed row offsets, n + 1 values


def fgk_batch_create(handles: list, nrhs: int, rhs_per_cta: int = 0, stream=None) -> Batch:
    """Group built plans (d <= 2) for batched products and solves."""
    lib = load()
    arr = (ctypes.c_void_p * len(handles))(*[h.ptr for h in handles])
    out = ctypes.c_void_p()
    _check(lib.fgk_batch_create(arr, len(handles), int(nrhs), int(rhs_per_cta), _stream(stream), ctypes.byref(out)))
    offs = (ctypes.c_int64 * (len(handles) + 1))()
    _check(lib.fgk_batch_layout(out.value, offs))
    return Batch(out.value, list(handles), int(nrhs), list(offs))


def fgk_batch_matvec_q(b: Batch, Vq: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Packed FP32 products of every problem of the batch."""
    lib = load()
    if not Vq.is_cuda or Vq.dtype != torch.float32 or not Vq.is_contiguous() or Vq.shape != (b.rows[-1], b.nrhs):
        raise TypeError("Vq must be a contiguous CUDA float32 tensor of shape (total rows, nrhs)")
    out = _out_for(out, Vq)
    _check(lib.fgk_batch_matvec_q(b.ptr, Vq.data_ptr(), out.data_ptr(), _stream(stream)))
    return out


def fgk_batch_cg_solve(b: Batch, ys: list, sigma2s, tol: float = 1e-8, maxit: int = 100000, stream=None,
                       precs: list | None = None):
    """Mixed-precision CG for every problem and column (preconditioned by
    ``precs``, one per problem, when given); returns (alphas, infos, status)."""
    lib = load()
    n = len(b.handles)
    if len(ys) != n or len(sigma2s) != n or (precs is not None and len(precs) != n):
        raise ValueError(f"the batch has {n} problems: give one y, one sigma2 (and one preconditioner) each")
    ys = [_dev_f64_2d(y, "y") for y in ys]
    for y, hh in zip(ys, b.handles):
        _rows(y, hh.N, "y")
        if y.shape[1] != b.nrhs:
            raise ValueError(f"y has {y.shape[1]} columns, the batch {b.nrhs}")
    alphas = [torch.empty_like(y) for y in ys]
    yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
    ap = (ctypes.c_void_p * n)(*[a.data_ptr() for a in alphas])
    sg = (ctypes.c_double * n)(*[float(x) for x in sigma2s])
    infos = (fgk_cg_info * n)()
    res = [(ctypes.c_double * b.nrhs)() for _ in range(n)]
    for i in range(n):
        infos[i].true_resid = ctypes.cast(res[i], ctypes.POINTER(ctypes.c_double))
    if precs is None:
        rc = lib.fgk_batch_cg_solve(b.ptr, yp, sg, float(tol), int(maxit), ap, infos, _stream(stream))
    else:
        pp = (ctypes.c_void_p * n)(*[q.ptr for q in precs])
        rc = lib.fgk_batch_cg_solve_pc(b.ptr, pp, yp, sg, float(tol), int(maxit), ap, infos, _stream(stream))
    _check(rc, allow_soft=True)
    out = [{"iterations": infos[i].iterations, "refinements": infos[i].refinements, "mvm_f32": infos[i].mvm_f32,
            "mvm_f64": infos[i].mvm_f64, "max_true_resid": infos[i].max_true_resid, "true_resid": list(res[i]),
            "restarts": infos[i].restarts, "fp64_switch": infos[i].fp64_switch}
           for i in range(n)]
    return alphas, out, rc


def fgk_batch_destroy(b: Batch) -> None:
    if b is not None and b.ptr:
        _check(load().fgk_batch_destroy(b.ptr))
        b.ptr = 0


# ------------------------------------------------------------ torch allocator hook
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_hooks = []


def use_torch_allocator(enable: bool = True) -> None:
    """Route libfgk's device allocations through torch's caching allocator."""
    lib = load()
    if not enable:
        _check(lib.fgk_set_allocator(None, None, None))
        return

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream) if stream else 0)
        except Exception:  # allocation failure is reported to the library as NULL
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = _ALLOC_T(_alloc), _FREE_T(_free)
    _hooks[:] = [a, f]
    _check(lib.fgk_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None))
