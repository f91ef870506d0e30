"""ctypes declarations of the C ABI in include/svlcov.h (argument marshalling
only; every step of an update runs in the CUDA library)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

SVLCOV_OK = 0
SVLCOV_ERR_INVALID_ARG = 1
SVLCOV_ERR_CAPACITY = 2
SVLCOV_ERR_CUDA = 3
SVLCOV_ERR_STATE = 4
SVLCOV_DEV_BAD_CSR = 0x10
SVLCOV_DEV_NONFINITE = 0x20
SVLCOV_DEV_NOT_PD = 0x40
SVLCOV_DEV_GAP_WARN = 0x80
SVLCOV_DEV_TIMEOUT = 0x100
SVLCOV_FP64, SVLCOV_FP32, SVLCOV_BF16 = 0, 1, 2
SVLCOV_SMALL_FP64, SVLCOV_SMALL_FP32, SVLCOV_SMALL_MIXED = 0, 1, 2
SVLCOV_MAX_K = 128
SVLCOV_MAX_S = 1024
SVLCOV_SMALL_SVD_STATIC_MAX_N = 256
SVLCOV_APPROX_GKL, SVLCOV_APPROX_RPI = 1, 2


class svlcov_csr(C.Structure):
    _fields_ = [("rows", C.c_int32), ("cols", C.c_int32), ("nnz", C.c_int64),
                ("indptr", C.c_void_p), ("indices", C.c_void_p), ("values", C.c_void_p),
                ("values_dtype", C.c_int32)]


class svlcov_init_desc(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("k", C.c_int32),
                ("max_m", C.c_int64), ("max_n", C.c_int64), ("max_s", C.c_int32), ("max_nnz", C.c_int64),
                ("storage", C.c_int32), ("small", C.c_int32),
                ("U0", C.c_void_p), ("sigma0", C.c_void_p), ("V0", C.c_void_p), ("init_dtype", C.c_int32),
                ("ubuf", C.c_void_p), ("vbuf", C.c_void_p),
                ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t),
                ("tau", C.c_double), ("reset_threshold", C.c_double), ("jacobi_block", C.c_int32),
                ("reorth", C.c_int32), ("gemm_split", C.c_int32), ("tensor_gemm", C.c_int32),
                ("s1_secular", C.c_int32), ("literal_steps", C.c_int32)]


class svlcov_op(C.Structure):
    _fields_ = [("kind", C.c_int32), ("a", svlcov_csr), ("b", svlcov_csr)]


class svlcov_approx(C.Structure):
    _fields_ = [("method", C.c_int32), ("l", C.c_int32), ("t", C.c_int32), ("start", C.c_void_p),
                ("work", C.c_void_p)]


# name -> (restype, argtypes)
SIGNATURES = {
    "svlcov_workspace_bytes": (C.c_size_t, [C.POINTER(svlcov_init_desc)]),
    "svlcov_init": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(svlcov_init_desc), C.c_void_p]),
    "svlcov_add_cols": (C.c_int, [C.c_void_p, C.POINTER(svlcov_csr), C.c_void_p]),
    "svlcov_add_rows": (C.c_int, [C.c_void_p, C.POINTER(svlcov_csr), C.c_void_p]),
    "svlcov_update_weights": (C.c_int, [C.c_void_p, C.POINTER(svlcov_csr), C.POINTER(svlcov_csr), C.c_void_p]),
    "svlcov_get_factors": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "svlcov_query_rows": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32,
                                    C.c_void_p]),
    "svlcov_get_shape": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int32)]),
    "svlcov_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_void_p]),
    "svlcov_get_small_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.POINTER(C.c_int64), C.c_void_p]),
    "svlcov_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p]),
    "svlcov_set_state": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "svlcov_get_intermediate": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t,
                                          C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_void_p]),
    "svlcov_approx_work_bytes": (C.c_size_t, [C.c_void_p, C.c_int32]),
    "svlcov_add_cols_approx": (C.c_int, [C.c_void_p, C.POINTER(svlcov_csr), C.POINTER(svlcov_approx), C.c_void_p]),
    "svlcov_add_rows_approx": (C.c_int, [C.c_void_p, C.POINTER(svlcov_csr), C.POINTER(svlcov_approx), C.c_void_p]),
    "svlcov_update_weights_approx": (C.c_int, [C.c_void_p, C.POINTER(svlcov_csr), C.POINTER(svlcov_csr),
                                               C.POINTER(svlcov_approx), C.c_void_p]),
    "svlcov_add_cols_backward_work_bytes": (C.c_size_t, [C.c_void_p]),
    "svlcov_add_cols_backward": (C.c_int, [C.c_void_p, C.POINTER(svlcov_csr), C.c_void_p, C.c_int32, C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                           C.c_void_p]),
    "svlcov_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "svlcov_profile_read": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                      C.POINTER(C.c_int64)]),
    "svlcov_kernel_launches": (C.c_uint64, []),
    "svlcov_batch_run": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(svlcov_op), C.c_int32, C.c_int32, C.c_void_p]),
    "svlcov_destroy": (None, [C.c_void_p]),
    "svlcov_strerror": (C.c_char_p, [C.c_int32]),
    "svlcov_small_svd_work_bytes": (C.c_size_t, [C.c_int32]),
    "svlcov_small_svd": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_int32, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p]),
    "svlcov_project": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(svlcov_csr), C.c_void_p, C.c_void_p, C.c_void_p]),
    "svlcov_score_pairs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                                     C.c_void_p]),
    "svlcov_small_svd_arrow_work_bytes": (C.c_size_t, []),
    "svlcov_small_svd_arrow": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p]),
    "svlcov_dgemm": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_void_p,
                                C.c_int32, C.c_void_p, C.c_int32, C.c_double, C.c_void_p, C.c_int32, C.c_int32,
                                C.c_void_p]),
    "svlcov_small_svd_static": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_int32, C.POINTER(C.c_int32), C.c_void_p]),
}

_LIB = None


def lib() -> C.CDLL:
    """Load libsvlcov.so (building it first if it is missing or stale).
    Raises if the CUDA toolkit is unavailable: there is no CPU fallback."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not _build.up_to_date():
            path = _build.build()
        L = C.CDLL(path, mode=os.RTLD_LAZY | getattr(os, "RTLD_GLOBAL", 0))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


class SvlcovError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().svlcov_strerror(code)
        super().__init__(f"{where}: error {code} ({msg.decode() if msg else '?'})")
        self.code = code


def check(code: int, where: str) -> None:
    if code != SVLCOV_OK:
        raise SvlcovError(code, where)
