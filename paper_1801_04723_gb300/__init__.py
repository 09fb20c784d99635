"""GB300 (sm_103a) implementation of Strassen's block-recursive matrix
inversion, the method of SPIN (Misra et al., ICDCN'18, arXiv 1801.04723).

The computation lives in the CUDA library ``_build/libspin.so`` behind the C
ABI of ``include/spin.h``; :mod:`.binding` marshals torch tensors / numpy
arrays into that ABI and nothing else.  ``build()`` compiles the library.
There is no CPU fallback: every entry point raises if the library is absent.
"""
from .binding import (  # noqa: F401
    SPIN_FP64,
    SPIN_MIXED_BF16X3,
    SPIN_MIXED_DIGITS,
    SpinError,
    Server,
    Info,
    Opts,
    default_leaf,
    model_seconds,
    rbt_diagonals,
    autotune_leaf,
    autotune_batched_leaf,
    schedule_stats,
    gemm_f64,
    gemm_bf16x3,
    gemm_ozaki,
    take_device_error,
    leaf_exchange_timeout,
    persistent_wait_timeout,
    autotune_batched_persistent,
    invert,
    invert_host,
    invert_noalloc,
    invert_batched,
    batched_stats,
    batched_refine_info,
    leaf_inverse,
    lib,
    status_string,
    sync,
    profile_start,
    profile_collect,
    probe_fp64_peak,
    probe_fp64_mma_peak,
    workspace_bytes,
)
from .build import build  # noqa: F401
