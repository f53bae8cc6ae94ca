"""ctypes declarations of the bkrylov C ABI (``include/bkrylov.h``).

Every C entry point is exposed under its own name with its C signature;
nothing here computes anything.  Loading fails loudly if the compiled
library is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libbkrylov.so")

BK_FP64, BK_FP32, BK_FP32_IR = 0, 1, 2
BK_OK, BK_ERR_ARG, BK_ERR_CUDA, BK_ERR_ALLOC = 0, 1, 2, 3
BK_NOT_CONVERGED, BK_BREAKDOWN, BK_NONFINITE, BK_TIMEOUT, BK_ERR_UNSUPPORTED = 4, 5, 6, 7, 8
BK_STENCIL_CONST7, BK_STENCIL_VAR7, BK_STENCIL_EDGE5, BK_STENCIL_EDGE5_LOG = 0, 1, 2, 3
MAX_S = 32


class bkrylov_opts(C.Structure):
    _fields_ = [
        ("eta", C.c_double), ("restart", C.c_int),
        ("ortho", C.c_int), ("prec", C.c_int), ("ir_inner_tol", C.c_double),
        ("ir_max_outer", C.c_int), ("forced_reortho", C.POINTER(C.c_uint8)), ("n_forced", C.c_int),
        ("sync_every", C.c_int), ("profile", C.c_int), ("subalgebra_p", C.c_int),
        ("precond", C.c_void_p), ("norm_mode", C.c_int), ("one_reduction", C.c_int),
        ("replace_every", C.c_int), ("qr_mode", C.c_int),
    ]


class bkrylov_info(C.Structure):
    _fields_ = [
        ("iters", C.c_int), ("reorths", C.c_int), ("converged", C.c_int), ("status", C.c_int),
        ("outer", C.c_int), ("relres_max", C.c_double), ("relres", C.POINTER(C.c_double)),
        ("history", C.POINTER(C.c_double)), ("decisions", C.POINTER(C.c_uint8)),
        ("history_len", C.c_int), ("elapsed_ms", C.c_double), ("reorths_cholqr", C.c_int),
        ("replacements", C.c_int),
    ]


# (name, restype, argtypes) of every exported symbol, in header order.
SIGNATURES = [
    ("bkrylov_create", C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    ("bkrylov_destroy", C.c_int, [C.c_void_p]),
    ("bkrylov_set_stream", C.c_int, [C.c_void_p, C.c_void_p]),
    ("bkrylov_status_string", C.c_char_p, [C.c_int]),
    ("bkrylov_version", C.c_int, []),
    ("bkrylov_opts_default", None, [C.POINTER(bkrylov_opts)]),
    ("bkrylov_op_csr", C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_int, C.POINTER(C.c_void_p)]),
    ("bkrylov_op_stencil", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                     C.POINTER(C.c_void_p)]),
    ("bkrylov_op_diag", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("bkrylov_op_jacobi", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("bkrylov_op_transpose", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("bkrylov_op_destroy", C.c_int, [C.c_void_p]),
    ("bkrylov_op_size", C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    ("bkrylov_spmm", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    ("bkrylov_spmm_gram", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_int, C.c_int]),
    ("bkrylov_residual", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_int]),
    ("bkrylov_bdot", C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_int, C.c_int]),
    ("bkrylov_bdot_noalloc", C.c_int, [C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_int, C.c_int, C.c_void_p]),
    ("bkrylov_tsqr", C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_int]),
    ("bkrylov_solve_bcg", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                    C.POINTER(bkrylov_opts), C.POINTER(bkrylov_info)]),
    ("bkrylov_solve_bbicgstab", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                          C.POINTER(bkrylov_opts), C.POINTER(bkrylov_info)]),
    ("bkrylov_solve_bgmres", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                       C.POINTER(bkrylov_opts), C.POINTER(bkrylov_info)]),
    ("bkrylov_profile_count", C.c_int, []),
    ("bkrylov_profile_get", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_double),
                                      C.POINTER(C.c_longlong)]),
    ("bkrylov_profile_reset", C.c_int, [C.c_void_p]),
    ("bkrylov_kappa_d", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("bkrylov_reortho_decision", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_double, C.c_double,
                                           C.c_void_p]),
    ("bkrylov_bcg_launches_per_iteration", C.c_int, [C.c_int64, C.c_int, C.c_void_p]),
    ("bkrylov_adjoint_scatter", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_void_p]),
    ("bkrylov_edge_theta_grad", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_void_p]),
]

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"bkrylov CUDA library not built: {path} is missing "
                          "(run __graft_entry__.build() or paper_2104_02494_gb300/build.py)")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def default_opts() -> bkrylov_opts:
    o = bkrylov_opts()
    load().bkrylov_opts_default(C.byref(o))
    return o


def status_string(st: int) -> str:
    return load().bkrylov_status_string(st).decode()


INF = math.inf
