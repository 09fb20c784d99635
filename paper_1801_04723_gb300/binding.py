"""Thin ctypes binding of the C ABI in ``include/spin.h``.

Argument marshalling only: tensors become device pointers and leading
dimensions, the current torch stream becomes the ``cudaStream_t``.  Every
step of the inversion runs in the CUDA library; if the library is missing
the calls raise instead of computing anything elsewhere.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB

SPIN_OK = 0
SPIN_ERR_INVALID_ARG = 1
SPIN_ERR_SINGULAR = 2
SPIN_ERR_NOT_CONVERGED = 3
SPIN_ERR_NOT_IMPLEMENTED = 8

SPIN_FP64 = 0
SPIN_MIXED_BF16X3 = 1
SPIN_MIXED_DIGITS = 3

PRECISIONS = {"fp64": SPIN_FP64, "bf16x3": SPIN_MIXED_BF16X3, "digits": SPIN_MIXED_DIGITS}


class Opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("leaf", ctypes.c_int32),
        ("tol", ctypes.c_double),
        ("max_refine", ctypes.c_int32),
        ("fp64_levels", ctypes.c_int32),
        ("blocking", ctypes.c_int32),
        ("residual_slices", ctypes.c_int32),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("pretransform", ctypes.c_int32),
        ("schedule", ctypes.c_int32),
        ("rbt_seed", ctypes.c_uint64),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("refine_iters", ctypes.c_int32),
        ("fail_leaf", ctypes.c_int64),
        ("fail_col", ctypes.c_int64),
        ("rel_residual", ctypes.c_double),
        ("pretransformed", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class ProfRecord(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("depth", ctypes.c_int32),
        ("m", ctypes.c_int64),
        ("n", ctypes.c_int64),
        ("k", ctypes.c_int64),
        ("flops", ctypes.c_double),
        ("bytes", ctypes.c_double),
        ("ms", ctypes.c_double),
    ]


KERNEL_KINDS = {0: "leaf_gj", 1: "gemm_f64", 2: "gemm_tc", 3: "split", 4: "residual", 5: "update", 6: "other"}


class ServeCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int32), ("priority_order", ctypes.c_int32),
                ("max_queued_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int32),
                ("batch_max_order", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("refine_iters", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("batch", ctypes.c_int32),
        ("rel_residual", ctypes.c_double),
        ("queue_ms", ctypes.c_double),
        ("run_ms", ctypes.c_double),
        ("latency_ms", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class ServeStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64),
        ("completed", ctypes.c_uint64),
        ("rejected", ctypes.c_uint64),
        ("queued", ctypes.c_uint64),
        ("running", ctypes.c_int32),
        ("peak_running", ctypes.c_int32),
        ("bytes_in_use", ctypes.c_size_t),
        ("shed", ctypes.c_uint64),
        ("deferred", ctypes.c_uint64),
        ("groups", ctypes.c_uint64),
        ("grouped", ctypes.c_uint64),
        ("max_group", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class SpinError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = status_string(code)
        if what:
            msg = f"{what}: {msg}"
        if code == 5:
            msg += f" ({last_error()})"
        super().__init__(msg)


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB):
            raise RuntimeError(f"CUDA library not built ({LIB}); run paper_1801_04723_gb300.build()")
        L = ctypes.CDLL(LIB)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        L.spin_opts_default.restype = Opts
        L.spin_invert.argtypes = [vp, vp, i64, i64, ctypes.c_int, vp]
        L.spin_invert.restype = ctypes.c_int
        L.spin_invert_ex.argtypes = [vp, i64, vp, i64, i64, ctypes.POINTER(Opts), ctypes.POINTER(Info), vp]
        L.spin_invert_ex.restype = ctypes.c_int
        L.spin_sync.argtypes = [vp, ctypes.POINTER(Info)]
        L.spin_sync.restype = ctypes.c_int
        L.spin_workspace_bytes.argtypes = [i64, ctypes.POINTER(Opts)]
        L.spin_rbt_diagonals.argtypes = [ctypes.c_uint64, i64, ctypes.c_int, vp, vp]
        L.spin_rbt_diagonals.restype = ctypes.c_int
        L.spin_model_seconds.argtypes = [i64, ctypes.c_int, ctypes.c_int]
        L.spin_model_seconds.restype = ctypes.c_double
        L.spin_workspace_bytes.restype = ctypes.c_size_t
        L.spin_default_leaf.argtypes = [i64, ctypes.c_int]
        L.spin_default_leaf.restype = ctypes.c_int
        L.spin_invert_host.argtypes = [vp, i64, vp, i64, i64, ctypes.POINTER(Opts), ctypes.POINTER(Info), vp]
        L.spin_invert_host.restype = ctypes.c_int
        L.spin_status_string.argtypes = [ctypes.c_int]
        L.spin_status_string.restype = ctypes.c_char_p
        L.spin_version.restype = ctypes.c_int
        L.spin_last_error.restype = ctypes.c_char_p
        L.spin_leaf_inverse.argtypes = [vp, i64, vp, i64, i64, vp, vp]
        L.spin_leaf_inverse.restype = ctypes.c_int
        L.spin_gemm_f64.argtypes = [i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, vp, i64, vp]
        L.spin_gemm_f64.restype = ctypes.c_int
        L.spin_profile_start.argtypes = [vp, ctypes.c_int]
        L.spin_profile_start.restype = ctypes.c_int
        L.spin_profile_stop.argtypes = [vp, ctypes.POINTER(ProfRecord), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.spin_profile_stop.restype = ctypes.c_int
        L.spin_probe_fp64_peak.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
        L.spin_probe_fp64_peak.restype = ctypes.c_int
        L.spin_probe_fp64_mma_peak.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
        L.spin_probe_fp64_mma_peak.restype = ctypes.c_int
        L.spin_gemm_bf16x3.argtypes = [i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, vp, i64, vp]
        L.spin_gemm_bf16x3.restype = ctypes.c_int
        L.spin_gemm_ozaki.argtypes = [i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, vp, i64, ctypes.c_int,
                                      ctypes.c_int, vp, vp]
        L.spin_gemm_ozaki.restype = ctypes.c_int
        L.spin_invert_batched.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.POINTER(Opts), vp, vp]
        L.spin_invert_batched.restype = ctypes.c_int
        L.spin_serve_create.argtypes = [ctypes.POINTER(ServeCfg), ctypes.POINTER(vp)]
        L.spin_serve_create.restype = ctypes.c_int
        L.spin_serve_submit.argtypes = [vp, vp, i64, i64, ctypes.c_int, dbl, ctypes.POINTER(ctypes.c_uint64)]
        L.spin_serve_submit.restype = ctypes.c_int
        L.spin_serve_poll.argtypes = [vp, ctypes.c_uint64, vp, i64, ctypes.POINTER(Result)]
        L.spin_serve_poll.restype = ctypes.c_int
        L.spin_serve_stats.argtypes = [vp, ctypes.POINTER(ServeStats)]
        L.spin_serve_stats.restype = ctypes.c_int
        L.spin_serve_destroy.argtypes = [vp]
        L.spin_serve_destroy.restype = ctypes.c_int
        L.spin_batched_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.spin_batched_stats.restype = ctypes.c_int
        L.spin_batched_refine_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
        L.spin_batched_refine_info.restype = ctypes.c_int
        L.spin_autotune_leaf.argtypes = [i64, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), vp, vp]
        L.spin_autotune_leaf.restype = ctypes.c_int
        L.spin_autotune_batched_leaf.argtypes = [ctypes.POINTER(i64), ctypes.c_int, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(dbl), vp]
        L.spin_autotune_batched_leaf.restype = ctypes.c_int
        L.spin_schedule_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.spin_schedule_stats.restype = ctypes.c_int
        L.spin_take_device_error.argtypes = [vp]
        L.spin_take_device_error.restype = ctypes.c_int
        L.spin_test_leaf_timeout.argtypes = [i64, ctypes.c_int, ctypes.c_double]
        L.spin_test_leaf_timeout.restype = ctypes.c_int
        L.spin_test_persistent_timeout.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                                   ctypes.POINTER(ctypes.c_int)]
        L.spin_test_persistent_timeout.restype = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int)
        L.spin_autotune_batched_persistent.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ip, ctypes.c_int,
                                                       ip, ctypes.c_int, ip, ip, ctypes.POINTER(ctypes.c_double), vp]
        L.spin_autotune_batched_persistent.restype = ctypes.c_int
        L.spin_invert_noalloc.argtypes = [vp, vp, i64, i64, ctypes.c_int, vp]
        L.spin_invert_noalloc.restype = ctypes.c_int
        _lib = L
        return L


def status_string(code: int) -> str:
    try:
        return lib().spin_status_string(int(code)).decode()
    except RuntimeError:
        return f"status {code}"


def last_error() -> str:
    return lib().spin_last_error().decode()


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _check_matrix(t, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or t.dim() != 2:
        raise TypeError(f"{name} must be a 2-D float64 CUDA tensor")
    if t.stride(1) != 1:
        raise ValueError(f"{name} must be row-major (unit column stride)")


SCHEDULES = {"default": 0, "lockstep": 1, "persistent": 2}


def make_opts(precision="fp64", leaf=0, tol=1e-10, max_refine=6, fp64_levels=2, blocking=True,
              workspace=None, residual_slices=0, pretransform=0, rbt_seed=0, schedule="default") -> Opts:
    o = lib().spin_opts_default()
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.leaf = int(leaf)
    o.tol = float(tol)
    o.max_refine = int(max_refine)
    o.fp64_levels = int(fp64_levels)
    o.blocking = 1 if blocking else 0
    o.residual_slices = int(residual_slices)
    o.pretransform = int(pretransform)
    o.rbt_seed = int(rbt_seed) & 0xFFFFFFFFFFFFFFFF
    o.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    if workspace is not None:
        o.workspace = ctypes.c_void_p(workspace.data_ptr())
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o


def invert(A, *, leaf: int = 0, precision="fp64", out=None, tol: float = 1e-10, max_refine: int = 6,
           fp64_levels: int = 2, stream=None, check: bool = True, workspace=None, blocking: bool = True,
           residual_slices: int = 0, pretransform: int = 0, rbt_seed: int = 0, schedule="default"):
    """X = A^-1 on the device (spin_invert_ex).  Returns (X, info dict).

    With ``blocking=False`` the call only enqueues the work on the stream and
    returns (X, None); :func:`sync` reads the status afterwards.  Raises
    :class:`SpinError` on an argument/CUDA error, and on a numerical failure
    when ``check``."""
    import torch

    _check_matrix(A, "A")
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("A must be square")
    X = out if out is not None else torch.empty((n, n), dtype=torch.float64, device=A.device)
    _check_matrix(X, "X")
    o = make_opts(precision, leaf, tol, max_refine, fp64_levels, blocking, workspace, residual_slices,
                  pretransform, rbt_seed, schedule)
    if not blocking:
        rc = lib().spin_invert_ex(ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(X.data_ptr()),
                                  X.stride(0), n, ctypes.byref(o), None, _stream(stream))
        if rc != SPIN_OK:
            raise SpinError(rc, "spin_invert_ex")
        return X, None
    info = Info()
    rc = lib().spin_invert_ex(ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(X.data_ptr()),
                              X.stride(0), n, ctypes.byref(o), ctypes.byref(info), _stream(stream))
    if rc not in (SPIN_OK, SPIN_ERR_SINGULAR, SPIN_ERR_NOT_CONVERGED) or (check and rc != SPIN_OK):
        raise SpinError(rc, "spin_invert_ex")
    return X, info.as_dict()


def sync(stream=None, check: bool = True) -> dict:
    """Wait for the stream and return the info of its latest non-blocking
    inversion (spin_sync)."""
    info = Info()
    rc = lib().spin_sync(_stream(stream), ctypes.byref(info))
    if rc not in (SPIN_OK, SPIN_ERR_SINGULAR, SPIN_ERR_NOT_CONVERGED) or (check and rc != SPIN_OK):
        raise SpinError(rc, "spin_sync")
    return info.as_dict()


def invert_host(A, *, leaf: int = 0, precision="fp64", out=None, tol: float = 1e-10, stream=None,
                pretransform: int = 0, rbt_seed: int = 0, schedule="default"):
    """X = A^-1 with host (numpy or CPU torch, float64, C-contiguous) buffers."""
    import numpy as np

    A = np.ascontiguousarray(A, dtype=np.float64) if not hasattr(A, "data_ptr") else A
    n = A.shape[0]
    if out is None:
        out = np.empty((n, n), dtype=np.float64)
    pa = A.ctypes.data if isinstance(A, np.ndarray) else A.data_ptr()
    px = out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()
    o = make_opts(precision, leaf, tol, pretransform=pretransform, rbt_seed=rbt_seed, schedule=schedule)
    info = Info()
    rc = lib().spin_invert_host(ctypes.c_void_p(pa), n, ctypes.c_void_p(px), n, n, ctypes.byref(o),
                                ctypes.byref(info), _stream(stream))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_invert_host")
    return out, info.as_dict()


def workspace_bytes(n: int, *, leaf: int = 0, precision="fp64", fp64_levels: int = 2,
                    residual_slices: int = 0, pretransform: int = 0, schedule="default") -> int:
    o = make_opts(precision, leaf, fp64_levels=fp64_levels, residual_slices=residual_slices,
                  pretransform=pretransform, schedule=schedule)
    return int(lib().spin_workspace_bytes(int(n), ctypes.byref(o)))


def rbt_diagonals(seed: int, n: int, depth: int = 2, stream=None):
    """The butterfly transform's random diagonals for order n
    (spin_rbt_diagonals): a float64 CUDA tensor of 2 * depth * np entries."""
    import torch

    q = 2 ** depth
    np_ = -(-int(n) // q) * q
    out = torch.empty(2 * depth * np_, dtype=torch.float64, device="cuda")
    rc = lib().spin_rbt_diagonals(ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), int(n), int(depth),
                                  ctypes.c_void_p(out.data_ptr()), _stream(stream))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_rbt_diagonals")
    return out


def model_seconds(n: int, leaf: int, precision="fp64") -> float:
    """Cost-model time of one inversion (spin_model_seconds; FP64 only)."""
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return float(lib().spin_model_seconds(int(n), int(leaf), p))


def default_leaf(n: int, precision="fp64") -> int:
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return int(lib().spin_default_leaf(int(n), p))


def leaf_inverse(A, out=None, info_dev=None, stream=None):
    """Gauss-Jordan leaf inversion of one block (spin_leaf_inverse); async."""
    import torch

    _check_matrix(A, "A")
    n = A.shape[0]
    X = out if out is not None else torch.empty((n, n), dtype=torch.float64, device=A.device)
    pinfo = ctypes.c_void_p(info_dev.data_ptr()) if info_dev is not None else None
    rc = lib().spin_leaf_inverse(ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(X.data_ptr()),
                                 X.stride(0), n, pinfo, _stream(stream))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_leaf_inverse")
    return X


def gemm_f64(A, B, *, alpha=1.0, beta=0.0, C=None, out=None, stream=None):
    """D = beta*C + alpha*(A @ B) in FP64 (spin_gemm_f64); async."""
    import torch

    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    D = out if out is not None else torch.empty((m, n), dtype=torch.float64, device=A.device)
    pc = ctypes.c_void_p(C.data_ptr()) if C is not None else None
    ldc = C.stride(0) if C is not None else 0
    rc = lib().spin_gemm_f64(m, n, k, float(alpha), ctypes.c_void_p(A.data_ptr()), A.stride(0),
                             ctypes.c_void_p(B.data_ptr()), B.stride(0), float(beta), pc, ldc,
                             ctypes.c_void_p(D.data_ptr()), D.stride(0), _stream(stream))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_gemm_f64")
    return D


def profile_start(max_records: int = 1 << 20, stream=None) -> None:
    rc = lib().spin_profile_start(_stream(stream), int(max_records))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_profile_start")


def profile_collect(stream=None, max_records: int = 1 << 20) -> list[dict]:
    """Stop recording and return the records (see :func:`profile_stop`)."""
    buf = (ProfRecord * max_records)()
    cnt = ctypes.c_int(0)
    rc = lib().spin_profile_stop(_stream(stream), buf, max_records, ctypes.byref(cnt))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_profile_stop")
    out = []
    for i in range(min(cnt.value, max_records)):
        r = buf[i]
        out.append({"kind": KERNEL_KINDS.get(r.kind, str(r.kind)), "depth": r.depth, "m": r.m, "n": r.n, "k": r.k,
                    "flops": r.flops, "bytes": r.bytes, "ms": r.ms})
    return out


def probe_fp64_peak(stream=None) -> float:
    """FP64 FMA throughput of this GPU in TFLOP/s (DFMA-bound probe kernel)."""
    v = ctypes.c_double(0.0)
    rc = lib().spin_probe_fp64_peak(ctypes.byref(v), _stream(stream))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_probe_fp64_peak")
    return v.value


def probe_fp64_mma_peak(stream=None) -> float:
    """FP64 throughput of this GPU through mma.sync f64 (DMMA) in TFLOP/s."""
    v = ctypes.c_double(0.0)
    rc = lib().spin_probe_fp64_mma_peak(ctypes.byref(v), _stream(stream))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_probe_fp64_mma_peak")
    return v.value


def _gemm_args(A, B, C, out):
    import torch

    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    D = out if out is not None else torch.empty((m, n), dtype=torch.float64, device=A.device)
    pc = ctypes.c_void_p(C.data_ptr()) if C is not None else None
    ldc = C.stride(0) if C is not None else 0
    return m, n, k, D, pc, ldc


def gemm_bf16x3(A, B, *, alpha=1.0, beta=0.0, C=None, out=None, stream=None):
    """D = beta*C + alpha*(A @ B) on the BF16 tensor cores, 3-term split (spin_gemm_bf16x3)."""
    m, n, k, D, pc, ldc = _gemm_args(A, B, C, out)
    rc = lib().spin_gemm_bf16x3(m, n, k, float(alpha), ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                ctypes.c_void_p(B.data_ptr()), B.stride(0), float(beta), pc, ldc,
                                ctypes.c_void_p(D.data_ptr()), D.stride(0), _stream(stream))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_gemm_bf16x3")
    return D


def gemm_ozaki(A, B, *, slices=7, alpha=1.0, beta=0.0, C=None, out=None, add_identity=False, sumsq=None,
               stream=None):
    """D = beta*C + alpha*(A @ B) (+ I) with FP64-class accuracy from fixed-point
    BF16 digit slices (spin_gemm_ozaki)."""
    m, n, k, D, pc, ldc = _gemm_args(A, B, C, out)
    ps = ctypes.c_void_p(sumsq.data_ptr()) if sumsq is not None else None
    rc = lib().spin_gemm_ozaki(m, n, k, float(alpha), ctypes.c_void_p(A.data_ptr()), A.stride(0),
                               ctypes.c_void_p(B.data_ptr()), B.stride(0), float(beta), pc, ldc,
                               ctypes.c_void_p(D.data_ptr()), D.stride(0), int(slices), 1 if add_identity else 0,
                               ps, _stream(stream))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_gemm_ozaki")
    return D


def take_device_error(stream=None) -> int:
    return int(lib().spin_take_device_error(_stream(stream)))


def leaf_exchange_timeout(order: int, mute_rank: int, limit_ms: float) -> int:
    """Status of a leaf whose CTA mute_rank sends nothing (spin_test_leaf_timeout)."""
    return int(lib().spin_test_leaf_timeout(int(order), int(mute_rank), float(limit_ms)))


def persistent_wait_timeout(limit_ms: float):
    """Statuses of the two matrices of a persistent batch whose first level
    product waits for a count nothing reaches (spin_test_persistent_timeout)."""
    s0, s1 = ctypes.c_int(-1), ctypes.c_int(-1)
    rc = lib().spin_test_persistent_timeout(float(limit_ms), ctypes.byref(s0), ctypes.byref(s1))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_test_persistent_timeout")
    return s0.value, s1.value


def invert_noalloc(A, *, leaf: int = 0, out=None, stream=None):
    """X = A^-1 through spin_invert_noalloc (no device allocation by the
    library; fixed 8 MB workspace per device).  Returns (X, status)."""
    import torch

    _check_matrix(A, "A")
    n = A.shape[0]
    X = out if out is not None else torch.empty((n, n), dtype=torch.float64, device=A.device)
    if X.stride(0) != n:
        raise ValueError("X must be contiguous (leading dimension n)")
    rc = lib().spin_invert_noalloc(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(X.data_ptr()), n, A.stride(0),
                                   int(leaf), _stream(stream))
    return X, int(rc)


def batched_stats(stream=None) -> dict:
    """Kernel launches per call and buckets of the latest batched graph on the stream."""
    k, b = ctypes.c_int(0), ctypes.c_int(0)
    rc = lib().spin_batched_stats(_stream(stream), ctypes.byref(k), ctypes.byref(b))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_batched_stats")
    return {"kernels": k.value, "buckets": b.value}


def invert_batched(As, *, leaf: int = 0, outs=None, stream=None, blocking: bool = True, precision="fp64",
                   tol: float = 1e-10, max_refine: int = 6, fp64_levels: int = 2, schedule="default"):
    """X_i = A_i^-1 for a list of square float64 CUDA tensors of any orders
    (spin_invert_batched).  Returns (list of X, int32 CUDA tensor of statuses).
    precision "bf16x3" runs the mixed form (its refinement is part of the
    captured graph).  schedule (plain form): "default" / "persistent" (one
    persistent launch over a device-side task list) or "lockstep" (launches
    per order bucket on a pool of streams).  With ``blocking=False`` the call
    returns once the work is enqueued on the stream."""
    import torch

    count = len(As)
    if outs is None:
        outs = [torch.empty((a.shape[0], a.shape[0]), dtype=torch.float64, device=a.device) for a in As]
    for a, x in zip(As, outs):
        _check_matrix(a, "A")
        _check_matrix(x, "X")
        if x.stride(0) != x.shape[0]:
            raise ValueError("each X must be contiguous")
    pa = (ctypes.c_void_p * count)(*[a.data_ptr() for a in As])
    px = (ctypes.c_void_p * count)(*[x.data_ptr() for x in outs])
    lda = (ctypes.c_int64 * count)(*[a.stride(0) for a in As])
    ns = (ctypes.c_int64 * count)(*[a.shape[0] for a in As])
    info = torch.zeros(count, dtype=torch.int32, device=As[0].device)
    o = make_opts(precision, leaf, blocking=blocking, tol=tol, max_refine=max_refine, fp64_levels=fp64_levels,
                  schedule=schedule)
    rc = lib().spin_invert_batched(pa, lda, px, ns, count, ctypes.byref(o), ctypes.c_void_p(info.data_ptr()),
                                   _stream(stream))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_invert_batched")
    return outs, info


def autotune_batched_leaf(orders, precision="fp64", candidates=(32, 64, 128), stream=None) -> dict:
    """Per order bucket of a batch, the fastest leaf among the candidates
    (spin_autotune_batched_leaf); recorded for later batched calls with leaf 0.
    Returns {order: (leaf, ms per bucket run)}.  Empty candidates forget the
    records of these orders (ms -1, leaf the default)."""
    orders = [int(v) for v in orders]
    cand = [int(c) for c in candidates]
    arr = (ctypes.c_int64 * len(orders))(*orders)
    carr = (ctypes.c_int * max(len(cand), 1))(*cand)
    out = (ctypes.c_int * len(orders))()
    ms = (ctypes.c_double * len(orders))()
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    rc = lib().spin_autotune_batched_leaf(arr, len(orders), p, carr, len(cand), out, ms, _stream(stream))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_autotune_batched_leaf")
    return {o: (out[i], ms[i]) for i, o in enumerate(orders)}


def autotune_batched_persistent(orders, leaves=(32, 64), tiles=(64, 32, 16), stream=None) -> dict:
    """Per order bucket of a plain batch, the fastest (leaf, largest product
    tile) pair of the persistent schedule (spin_autotune_batched_persistent);
    recorded for later plain batched calls with leaf 0.  Returns
    {order: (leaf, tile, ms per bucket run)}."""
    orders = [int(v) for v in orders]
    la = (ctypes.c_int * len(leaves))(*[int(v) for v in leaves])
    ta = (ctypes.c_int * len(tiles))(*[int(v) for v in tiles])
    arr = (ctypes.c_int64 * len(orders))(*orders)
    lo = (ctypes.c_int * len(orders))()
    to = (ctypes.c_int * len(orders))()
    ms = (ctypes.c_double * len(orders))()
    rc = lib().spin_autotune_batched_persistent(arr, len(orders), la, len(leaves), ta, len(tiles), lo, to, ms,
                                                _stream(stream))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_autotune_batched_persistent")
    return {o: (lo[i], to[i], ms[i]) for i, o in enumerate(orders)}


def schedule_stats(stream=None) -> dict:
    """Graph replays of single inversions on the stream, and the node count
    of the captured schedule (spin_schedule_stats)."""
    r, nd = ctypes.c_int64(), ctypes.c_int64()
    rc = lib().spin_schedule_stats(_stream(stream), ctypes.byref(r), ctypes.byref(nd))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_schedule_stats")
    return {"replays": r.value, "nodes": nd.value}


def batched_refine_info(stream=None) -> dict:
    """Refinement of the latest mixed batch on the stream: steps and worst residual."""
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    rc = lib().spin_batched_refine_info(_stream(stream), ctypes.byref(it), ctypes.byref(rel))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_batched_refine_info")
    return {"refine_iters": it.value, "worst_rel_residual": rel.value}


SPIN_ERR_BUSY = 7


class Server:
    """Request server (spin_serve_*): submit matrices (host numpy arrays or
    CUDA tensors, kept alive by the caller until polled), poll results.
    With ``max_queued_bytes`` a submit that would overfill the queue is shed:
    ``submit`` returns None.  With ``priority_order`` > 0, requests of order
    up to it run on high-priority streams.  A request whose device memory
    cannot be allocated while others run waits for one of them to finish
    (``stats()["deferred"]``).  Requests of order <= ``batch_max_order``
    (0: 1024) with the same padded order, precision and tolerance run
    together in batched launch groups of up to ``max_batch`` (0: 64; 1:
    off); each result carries the size of its group (``batch``)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 4, max_queued_bytes: int = 0,
                 priority_order: int = 0, max_batch: int = 0, batch_max_order: int = 0):
        cfg = ServeCfg(int(hbm_budget_bytes), int(max_slots), int(priority_order), int(max_queued_bytes),
                       int(max_batch), int(batch_max_order))
        h = ctypes.c_void_p()
        rc = lib().spin_serve_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != SPIN_OK:
            raise SpinError(rc, "spin_serve_create")
        self._h = h
        self._keep = {}

    def submit(self, A, precision="bf16x3", tol: float = 1e-10):
        import numpy as np

        if hasattr(A, "data_ptr"):
            ptr, lda, n = A.data_ptr(), A.stride(0), A.shape[0]
        else:
            A = np.ascontiguousarray(A, dtype=np.float64)
            ptr, lda, n = A.ctypes.data, A.shape[1], A.shape[0]
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        t = ctypes.c_uint64(0)
        rc = lib().spin_serve_submit(self._h, ctypes.c_void_p(ptr), lda, n, p, float(tol), ctypes.byref(t))
        if rc == SPIN_ERR_BUSY:
            return None  # shed: the queue is full
        if rc != SPIN_OK:
            raise SpinError(rc, "spin_serve_submit")
        self._keep[t.value] = A
        return t.value

    def poll(self, ticket: int, out=None, discard: bool = False):
        """None while busy; else (X, result dict).  X is a numpy array unless
        ``out`` (numpy array or CUDA tensor) is given; with ``discard`` the
        result is dropped on the device and X is None."""
        import numpy as np

        A = self._keep.get(ticket)
        n = A.shape[0] if A is not None else 0
        if discard:
            out, ptr, ld = None, None, n
        else:
            if out is None:
                out = np.empty((n, n), dtype=np.float64)
            ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
            ld = out.stride(0) if hasattr(out, "data_ptr") else out.shape[1]
        r = Result()
        rc = lib().spin_serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.c_void_p(ptr) if ptr else None, ld,
                                   ctypes.byref(r))
        if rc == SPIN_ERR_BUSY:
            return None
        if rc != SPIN_OK:
            raise SpinError(rc, "spin_serve_poll")
        self._keep.pop(ticket, None)
        return out, r.as_dict()

    def stats(self) -> dict:
        st = ServeStats()
        lib().spin_serve_stats(self._h, ctypes.byref(st))
        return st.as_dict()

    def close(self):
        if self._h:
            lib().spin_serve_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune_leaf(n: int, precision="fp64", candidates=(64, 128, 256, 512, 1024, 2048), stream=None):
    """Time the candidate leaf orders at order n (spin_autotune_leaf); returns
    (best leaf, {leaf: ms})."""
    cand = [int(c) for c in candidates]
    arr = (ctypes.c_int * len(cand))(*cand)
    ms = (ctypes.c_double * len(cand))()
    best = ctypes.c_int(0)
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    rc = lib().spin_autotune_leaf(int(n), p, arr, len(cand), ctypes.byref(best), ms, _stream(stream))
    if rc != SPIN_OK:
        raise SpinError(rc, "spin_autotune_leaf")
    return best.value, {c: ms[i] for i, c in enumerate(cand) if ms[i] >= 0}
