"""ctypes binding of libbcur.so (the C ABI declared in include/bcur.h).

Argument marshalling only: every step of the Block CUR path runs in the
library's CUDA kernels.  PyTorch supplies device memory and the current CUDA
stream.  If the library is missing the calls raise; there is no other path.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int32, c_int64, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbcur.so")

BCUR_F64, BCUR_F32, BCUR_TF32, BCUR_BF16, BCUR_BF16X3, BCUR_FP8, BCUR_BF16X3A, BCUR_FP8B = range(8)
PREC = {"f64": BCUR_F64, "f32": BCUR_F32, "tf32": BCUR_TF32, "bf16": BCUR_BF16,
        "bf16x3": BCUR_BF16X3, "fp8": BCUR_FP8, "bf16x3a": BCUR_BF16X3A, "fp8b": BCUR_FP8B}
STATUS = {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ERANK", 5: "ENONFINITE",
          6: "ETIMEOUT", 7: "ENOTSUP", 8: "ESTATE"}

#: Every entry point include/bcur.h declares.
EXPORTS = [
    "bcur_plan", "bcur_set_workspace", "bcur_scores", "bcur_factors", "bcur_sample", "bcur_fit",
    "bcur_error", "bcur_rank", "bcur_sync_status", "bcur_destroy", "bcur_status_string",
    "bcur_block_scores", "bcur_sample_blocks", "bcur_residual_workspace", "bcur_residual",
    "bcur_gemm", "bcur_launch_count", "bcur_version", "bcur_residual_noalloc",
    "bcur_gemm_split", "bcur_block_stable_rank_workspace", "bcur_block_stable_rank",
    "bcur_alg1_workspace", "bcur_alg1", "bcur_truncate", "bcur_batch_plan",
    "bcur_batch_set_workspace", "bcur_batch_run", "bcur_batch_dims", "bcur_batch_sync_status",
    "bcur_batch_destroy", "bcur_batch_profile", "bcur_batch_profile_count",
    "bcur_batch_profile_entry", "bcur_batch_set_stream", "bcur_host_staging_bytes",
    "bcur_decompose_host", "bcur_set_wait_budget_ns", "bcur_autotune_measured",
    "bcur_rank_k_error", "bcur_boost_select", "bcur_cholesky_inverse", "bcur_svd_small",
    "bcur_gather_blocks", "bcur_incoherence", "bcur_fit_terms", "bcur_batch_set_fit",
    "bcur_batch_fit_terms", "bcur_gemm_fp8_blocks",
]


class BcurError(RuntimeError):
    def __init__(self, status: int, where: str, lib=None):
        msg = STATUS.get(status, str(status))
        if lib is not None:
            try:
                msg = lib.bcur_status_string(status).decode()
            except Exception:  # pragma: no cover
                pass
        super().__init__(f"{where}: {STATUS.get(status, status)} ({msg})")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [
        ("m", c_int64), ("n", c_int64), ("lda", c_int64),
        ("a_dtype", c_int32), ("k", c_int32), ("p", c_int32), ("q", c_int32),
        ("G_col", c_int32), ("col_off", POINTER(c_int64)),
        ("G_row", c_int32), ("row_off", POINTER(c_int64)),
        ("g_col", c_int32), ("g_row", c_int32), ("replacement", c_int32),
        ("sketch_prec", c_int32), ("fit_prec", c_int32),
    ]


class BatchItem(ctypes.Structure):
    _fields_ = [
        ("m", c_int64), ("n", c_int64), ("lda", c_int64),
        ("k", c_int32), ("p", c_int32), ("block", c_int32), ("g_col", c_int32),
        ("g_row", c_int32),
    ]


class BatchIO(ctypes.Structure):
    _fields_ = [(name, c_void_p) for name in (
        "A", "omega", "u_col", "u_row", "col_scores", "row_scores", "col_idx", "row_idx", "U",
        "err")]


_lib = None


def load():
    """Load libbcur.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the Block CUR path has no non-CUDA fallback)")
    L = ctypes.CDLL(LIB_PATH)
    st = c_int32
    L.bcur_plan.argtypes = [POINTER(Desc), c_void_p, POINTER(c_void_p), POINTER(c_size_t)]
    L.bcur_plan.restype = st
    L.bcur_set_workspace.argtypes = [c_void_p, c_void_p, c_size_t]
    L.bcur_set_workspace.restype = st
    L.bcur_scores.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
    L.bcur_scores.restype = st
    L.bcur_factors.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    L.bcur_factors.restype = st
    L.bcur_sample.argtypes = [c_void_p] + [c_void_p] * 8
    L.bcur_sample.restype = st
    L.bcur_fit.argtypes = [c_void_p] + [c_void_p] * 6
    L.bcur_fit.restype = st
    L.bcur_error.argtypes = [c_void_p, c_void_p, c_void_p]
    L.bcur_error.restype = st
    L.bcur_fit_terms.argtypes = [c_void_p, POINTER(c_int32), POINTER(c_double)]
    L.bcur_fit_terms.restype = st
    L.bcur_batch_set_fit.argtypes = [c_void_p, c_int32]
    L.bcur_batch_set_fit.restype = st
    L.bcur_batch_fit_terms.argtypes = [c_void_p, c_void_p]
    L.bcur_batch_fit_terms.restype = st
    L.bcur_gemm_fp8_blocks.argtypes = [c_int64, c_int64, c_int64, c_void_p, c_int64, c_void_p,
                                       c_int64, c_void_p, c_void_p, c_int64, c_int64, c_void_p,
                                       c_int64, c_void_p]
    L.bcur_gemm_fp8_blocks.restype = st
    L.bcur_rank.argtypes = [c_void_p] + [POINTER(c_int64)] * 4
    L.bcur_rank.restype = st
    L.bcur_sync_status.argtypes = [c_void_p]
    L.bcur_sync_status.restype = st
    L.bcur_destroy.argtypes = [c_void_p]
    L.bcur_destroy.restype = None
    L.bcur_status_string.argtypes = [c_int32]
    L.bcur_status_string.restype = ctypes.c_char_p
    L.bcur_block_scores.argtypes = [c_void_p, c_int32, c_int32, c_int64, c_int64, c_void_p,
                                    c_int32, c_void_p, c_void_p]
    L.bcur_block_scores.restype = st
    L.bcur_sample_blocks.argtypes = [c_void_p, c_int32, c_void_p, c_int32, c_int32, c_void_p,
                                     c_void_p, c_void_p]
    L.bcur_sample_blocks.restype = st
    L.bcur_residual_workspace.argtypes = [c_int64, c_int64, c_int32]
    L.bcur_residual_workspace.restype = c_size_t
    L.bcur_residual.argtypes = [c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_int64, c_int64,
                                c_int64, c_int64, c_int32, c_int32, c_void_p, c_void_p, c_size_t,
                                c_void_p]
    L.bcur_residual.restype = st
    L.bcur_residual_noalloc.argtypes = [c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_int64,
                                        c_int64, c_int64, c_int64, c_int32, c_int32, c_void_p,
                                        c_void_p]
    L.bcur_residual_noalloc.restype = st
    L.bcur_host_staging_bytes.argtypes = [c_void_p]
    L.bcur_host_staging_bytes.restype = c_size_t
    L.bcur_decompose_host.argtypes = [c_void_p] + [c_void_p] * 5 + [c_size_t] + [c_void_p] * 6
    L.bcur_decompose_host.restype = st
    L.bcur_set_wait_budget_ns.argtypes = [ctypes.c_uint64]
    L.bcur_set_wait_budget_ns.restype = st
    L.bcur_autotune_measured.argtypes = []
    L.bcur_autotune_measured.restype = c_int32
    L.bcur_rank_k_error.argtypes = [c_void_p, c_void_p, c_void_p]
    L.bcur_rank_k_error.restype = st
    L.bcur_boost_select.argtypes = [c_int32, c_void_p, c_int64, c_void_p, c_int64, c_void_p,
                                    c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p]
    L.bcur_boost_select.restype = st
    L.bcur_cholesky_inverse.argtypes = [c_void_p, c_int64, c_int32, c_void_p, c_void_p, c_void_p,
                                        c_double, c_void_p, c_size_t, c_void_p]
    L.bcur_cholesky_inverse.restype = st
    L.bcur_svd_small.argtypes = [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                 c_void_p, c_size_t, c_void_p, c_void_p]
    L.bcur_svd_small.restype = st
    L.bcur_gather_blocks.argtypes = [c_void_p, c_int64, c_int64, c_int64, c_int32, c_int32,
                                     c_void_p, c_int32, c_void_p, c_int32, c_int64, c_void_p,
                                     c_int64, c_void_p, c_void_p]
    L.bcur_gather_blocks.restype = st
    L.bcur_incoherence.argtypes = [c_void_p, c_int32, c_int32, c_int64, c_int64, c_void_p,
                                   c_void_p, c_void_p]
    L.bcur_incoherence.restype = st
    L.bcur_gemm.argtypes = [c_int64, c_int64, c_int64, c_void_p, c_int64, c_int32, c_void_p,
                            c_int64, c_int32, c_void_p, c_int64, c_int32, c_int32, c_void_p]
    L.bcur_gemm.restype = st
    L.bcur_gemm_split.argtypes = [c_int64, c_int64, c_int64, c_void_p, c_void_p, c_int64, c_int32,
                                  c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_int64,
                                  c_void_p]
    L.bcur_gemm_split.restype = st
    L.bcur_block_stable_rank_workspace.argtypes = [c_int32, c_int32]
    L.bcur_block_stable_rank_workspace.restype = c_size_t
    L.bcur_block_stable_rank.argtypes = [c_void_p, c_int32, c_int32, c_int64, c_int64, c_void_p,
                                         c_int32, c_void_p, c_void_p, c_size_t, c_void_p]
    L.bcur_block_stable_rank.restype = st
    L.bcur_alg1_workspace.argtypes = [c_int64, c_int64, c_void_p, c_int32, c_int32, c_int32, c_int32]
    L.bcur_alg1_workspace.restype = c_size_t
    L.bcur_alg1.argtypes = [c_void_p, c_int64, c_int64, c_int64, c_int32, c_void_p, c_int32, c_int32,
                            c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                            c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]
    L.bcur_alg1.restype = st
    L.bcur_truncate.argtypes = [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p]
    L.bcur_truncate.restype = st
    L.bcur_batch_plan.argtypes = [POINTER(BatchItem), c_int32, c_int32, c_void_p,
                                  POINTER(c_void_p), POINTER(c_size_t)]
    L.bcur_batch_plan.restype = st
    L.bcur_batch_set_workspace.argtypes = [c_void_p, c_void_p, c_size_t]
    L.bcur_batch_set_workspace.restype = st
    L.bcur_batch_run.argtypes = [c_void_p, POINTER(BatchIO), c_int32]
    L.bcur_batch_run.restype = st
    L.bcur_batch_dims.argtypes = [c_void_p, c_int32, POINTER(c_int64), POINTER(c_int64),
                                  POINTER(c_int64)]
    L.bcur_batch_dims.restype = st
    L.bcur_batch_sync_status.argtypes = [c_void_p]
    L.bcur_batch_sync_status.restype = st
    L.bcur_batch_profile.argtypes = [c_void_p, c_int32]
    L.bcur_batch_profile.restype = st
    L.bcur_batch_profile_count.argtypes = [c_void_p]
    L.bcur_batch_profile_count.restype = c_int32
    L.bcur_batch_profile_entry.argtypes = [c_void_p, c_int32, POINTER(ctypes.c_char_p),
                                           POINTER(c_double)]
    L.bcur_batch_profile_entry.restype = st
    L.bcur_batch_set_stream.argtypes = [c_void_p, c_void_p]
    L.bcur_batch_set_stream.restype = st
    L.bcur_batch_destroy.argtypes = [c_void_p]
    L.bcur_batch_destroy.restype = None
    L.bcur_launch_count.argtypes = []
    L.bcur_launch_count.restype = ctypes.c_uint64
    L.bcur_version.argtypes = []
    L.bcur_version.restype = ctypes.c_char_p
    _lib = L
    return L


def check(status: int, where: str):
    if status != 0:
        raise BcurError(status, where, _lib)
