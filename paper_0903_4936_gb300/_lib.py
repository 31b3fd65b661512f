"""ctypes declarations of the C ABI in ``include/bkrylov.h``.

Loading fails loudly when ``libbkrylov.so`` has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbkrylov.so")

BK_OK = 0
STATUS_NAMES = {
    0: "BK_OK", 1: "BK_ERR_INVALID_ARG", 2: "BK_ERR_OUT_OF_MEMORY", 3: "BK_ERR_CUDA",
    4: "BK_ERR_NOT_CONVERGED", 5: "BK_ERR_BREAKDOWN", 6: "BK_ERR_NONFINITE", 7: "BK_ERR_NO_GAUGE",
}
PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "df64": 3}
METHOD = {"bicgstab": 0, "bicggr": 1}

# Every symbol include/bkrylov.h declares.
EXPORTED = [
    "bk_status_string", "bk_last_error", "bk_create", "bk_destroy", "bk_upload_gauge",
    "bk_build_clover", "bk_field_bytes", "bk_pack", "bk_unpack", "bk_dslash_dev", "bk_dslash", "bk_schur_dslash",
    "bk_gamma5", "bk_block_gram", "bk_block_xmy", "bk_small_solve", "bk_block_solve",
    "bk_block_solve_batched", "bk_dot", "bk_gauge_force", "bk_block_gram_noalloc", "bk_dslash_multi",
    "bk_set_clover", "bk_probe_peak", "bk_kappa_grad",
]
LAYOUT = {"canonical": 0, "device": 1}


class SolveParams(C.Structure):
    _fields_ = [
        ("method", C.c_int), ("prec", C.c_int), ("tol", C.c_double), ("maxiter", C.c_int),
        ("reliable_delta", C.c_double), ("x0_given", C.c_int), ("buffers_on_host", C.c_int),
        ("rtilde_mode", C.c_int), ("seed", C.c_uint64), ("rtilde", C.c_void_p), ("restart_on_update", C.c_int),
        ("orth_mode", C.c_int), ("record_history", C.c_int),
        ("timing", C.c_int), ("update_prec", C.c_int), ("deflate", C.c_int), ("eo", C.c_int),
        ("fp64_anchor", C.c_double),
    ]


class SolveInfo(C.Structure):
    _fields_ = [
        ("iterations", C.c_int), ("matvecs", C.c_int), ("matvecs_fp64", C.c_int),
        ("reliable_updates", C.c_int), ("restarts", C.c_int), ("converged", C.c_int), ("breakdown", C.c_int),
        ("true_res_max", C.c_double), ("rec_res_max", C.c_double),
        ("true_res", C.POINTER(C.c_double)), ("history", C.POINTER(C.c_double)),
        ("history_len", C.c_int), ("time_total_ms", C.c_double), ("time_dslash_ms", C.c_double),
        ("n_dslash", C.c_int), ("n_dslash_inner", C.c_int), ("time_dslash_inner_ms", C.c_double),
        ("n_launches", C.c_longlong),
        ("cols_dslash_inner", C.c_longlong), ("deflated", C.c_int),
    ]


class BKError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {detail}")


_lib = None


def lib():
    """The loaded library (raises if it is missing: nothing runs without it)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -m paper_0903_4936_gb300.build` "
            "(the library has no CPU fallback)")
    L = C.CDLL(LIB_PATH)
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    sig = {
        "bk_status_string": (C.c_char_p, [C.c_int]),
        "bk_last_error": (C.c_char_p, []),
        "bk_create": (C.c_int, [C.POINTER(C.c_int), C.c_int, C.POINTER(vp)]),
        "bk_destroy": (C.c_int, [vp]),
        "bk_upload_gauge": (C.c_int, [vp, vp, C.c_int, vp]),
        "bk_build_clover": (C.c_int, [vp, C.c_double, vp]),
        "bk_field_bytes": (C.c_size_t, [vp, C.c_int, C.c_int]),
        "bk_pack": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, vp]),
        "bk_unpack": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, vp]),
        "bk_dslash_dev": (C.c_int, [vp, dp, vp, vp, C.c_int, C.c_int, vp]),
        "bk_dslash": (C.c_int, [vp, dp, vp, vp, C.c_int, C.c_int, vp]),
        "bk_schur_dslash": (C.c_int, [vp, dp, vp, vp, C.c_int, C.c_int, vp]),
        "bk_gamma5": (C.c_int, [vp, vp, vp, C.c_int, vp]),
        "bk_block_gram": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, vp, vp]),
        "bk_block_xmy": (C.c_int, [vp, vp, vp, dp, vp, vp, C.c_int, C.c_int, vp]),
        "bk_small_solve": (C.c_int, [C.c_int, vp, vp, dp, vp, vp, vp]),
        "bk_block_solve": (C.c_int, [vp, C.POINTER(SolveParams), C.c_double, vp, vp, C.c_int,
                                     C.POINTER(SolveInfo), vp]),
        "bk_block_solve_batched": (C.c_int, [vp, C.POINTER(SolveParams), C.c_int, dp, ip, vp, vp,
                                             C.POINTER(SolveInfo), vp]),
        "bk_dot": (C.c_int, [vp, vp, vp, C.c_int, dp, vp]),
        "bk_block_gram_noalloc": (C.c_int, [C.c_int, vp, vp, C.c_int, C.c_int, vp, vp]),
        "bk_gauge_force": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, C.c_double, vp, vp]),
        "bk_dslash_multi": (C.c_int, [vp, C.c_double, vp, vp, C.c_int, C.c_int, C.c_int, vp]),
        "bk_set_clover": (C.c_int, [vp, C.c_double]),
        "bk_probe_peak": (C.c_int, [C.c_int, C.c_int, dp]),
        "bk_kappa_grad": (C.c_int, [vp, C.c_double, vp, vp, vp, C.c_int, dp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(status: int, where: str):
    if status != BK_OK:
        detail = lib().bk_last_error().decode(errors="replace")
        raise BKError(status, where, detail)
