"""ctypes binding of libtpmg.so (include/tpmg.h): argument marshalling only.

Every step of the solver runs in the CUDA library; this module converts
torch tensors to device pointers and the current torch stream to a
cudaStream_t.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libtpmg.so")

MG_OK, MG_ERR_ARG, MG_ERR_COEFF, MG_ERR_NONFINITE, MG_ERR_NOT_CONVERGED = 0, 1, 2, 3, 4
MG_ERR_DIVERGED, MG_ERR_TIMEOUT, MG_ERR_CUDA, MG_ERR_WORKSPACE = 5, 6, 7, 8
MG_METHOD_CG, MG_METHOD_STATIONARY, MG_METHOD_BICGSTAB, MG_METHOD_BICGSTAB_LINE = 0, 1, 2, 3
MG_PREC_FP64, MG_PREC_FP32 = 0, 1
MG_COARSE_JACOBI, MG_COARSE_PCG, MG_COARSE_CHEBYSHEV = 0, 1, 2
# kernel classes of mg_profile_read
K_SMOOTH, K_SMOOTH0, K_RESID, K_APPLY, K_RESTRICT, K_PROLONG, K_VEC = range(7)

STATUS_NAMES = {0: "MG_OK", 1: "MG_ERR_ARG", 2: "MG_ERR_COEFF", 3: "MG_ERR_NONFINITE",
                4: "MG_ERR_NOT_CONVERGED", 5: "MG_ERR_DIVERGED", 6: "MG_ERR_TIMEOUT",
                7: "MG_ERR_CUDA", 8: "MG_ERR_WORKSPACE"}


class MGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class mg_grid(ctypes.Structure):
    _fields_ = [("nlon", ctypes.c_int), ("nlat", ctypes.c_int), ("nz", ctypes.c_int)]


class mg_coeffs(ctypes.Structure):
    _fields_ = [("tx", ctypes.c_void_p), ("ty", ctypes.c_void_p), ("tz", ctypes.c_void_p),
                ("h", ctypes.c_void_p)]


class mg_ns_coeffs(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("h", "tx", "ty", "tz", "txr", "tyr", "tzr")]


class mg_params(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("coarse_iters", ctypes.c_int), ("method", ctypes.c_int), ("mixed", ctypes.c_int),
                ("maxit", ctypes.c_int), ("inner_maxit", ctypes.c_int),
                ("omega", ctypes.c_double), ("alpha_c", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("coarse_method", ctypes.c_int),
                ("line_sweeps", ctypes.c_int), ("iso_ratio", ctypes.c_double)]


class mg_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("inner_iterations", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("history", ctypes.POINTER(ctypes.c_double)),
                ("history_cap", ctypes.c_int), ("history_len", ctypes.c_int)]


_LIB = None


def load() -> ctypes.CDLL:
    """Load libtpmg.so; raises if it is missing (no fallback exists)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libtpmg.so not built ({LIB_PATH}); run __graft_entry__.build() "
                           "or python -m paper_2307_04528_gb300.build")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    H = ctypes.c_void_p
    sig = {
        "mg_default_params": (None, [ctypes.POINTER(mg_params)]),
        "mg_workspace_bytes": (I, [ctypes.POINTER(mg_grid), ctypes.POINTER(mg_params),
                                   ctypes.POINTER(S)]),
        "mg_setup": (I, [ctypes.POINTER(mg_grid), ctypes.POINTER(mg_coeffs),
                         ctypes.POINTER(mg_params), P, S, P, ctypes.POINTER(H)]),
        "mg_destroy": (None, [H]),
        "mg_apply": (I, [H, P, P, P]),
        "mg_vcycle": (I, [H, P, P, P]),
        "mg_vcycle_prec": (I, [H, I, P, P, P]),
        "mg_solve": (I, [H, P, P, D, ctypes.POINTER(mg_stats), P]),
        "mg_solve_mixed": (I, [H, P, P, D, ctypes.POINTER(mg_stats), P]),
        "mg_solve_single": (I, [H, P, P, D, ctypes.POINTER(mg_stats), P]),
        "mg_coeff_grad": (I, [H, P, P, P, P, P, P, P]),
        "mg_num_levels": (I, [H]),
        "mg_level_shape": (I, [H, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "mg_level_coeffs": (I, [H, I, P, P, P, P, P]),
        "mg_level_apply": (I, [H, I, I, P, P, P]),
        "mg_level_residual": (I, [H, I, I, P, P, P, P]),
        "mg_level_smooth": (I, [H, I, I, P, P, P, P]),
        "mg_level_smooth_dot": (I, [H, I, I, P, P, P, ctypes.POINTER(D), P]),
        "mg_level_dir_apply": (I, [H, I, I, P, P, D, P, P, ctypes.POINTER(D), P]),
        "mg_level_relax": (I, [H, I, I, I, P, P, P]),
        "mg_coarse_solve": (I, [H, I, P, P, P]),
        "mg_level_residual_restrict": (I, [H, I, I, P, P, P, P]),
        "mg_level_presmooth_restrict": (I, [H, I, I, P, P, P, P]),
        "mg_level_restrict": (I, [H, I, I, P, P, P]),
        "mg_level_prolong_add": (I, [H, I, I, P, P, P]),
        "mg_fp32_scale": (D, [H]),
        "mg_cast_fp32": (I, [P, P, D, S, P]),
        "mg_update_fp64": (I, [P, P, D, S, P]),
        "mg_profile_enable": (I, [H, I]),
        "mg_profile_read": (I, [H, I, I, I, ctypes.POINTER(I), ctypes.POINTER(D)]),
        "mg_launch_count": (ctypes.c_ulonglong, []),
        "mg_residual_norm_noalloc": (I, [ctypes.POINTER(mg_grid), ctypes.POINTER(mg_coeffs), P, P,
                                         P, ctypes.POINTER(D), P]),
        "mg_last_error": (ctypes.c_char_p, []),
        "mg_batch_workspace_bytes": (I, [I, ctypes.POINTER(mg_grid), ctypes.POINTER(mg_params),
                                         ctypes.POINTER(S)]),
        "mg_batch_setup": (I, [I, ctypes.POINTER(mg_grid), ctypes.POINTER(mg_coeffs),
                               ctypes.POINTER(mg_params), P, S, P, ctypes.POINTER(H)]),
        "mg_batch_destroy": (None, [H]),
        "mg_batch_handle": (I, [H, I, ctypes.POINTER(H)]),
        "mg_batch_tuning": (I, [H, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                ctypes.POINTER(I)]),
        "mg_batch_solve": (I, [H, ctypes.POINTER(P), ctypes.POINTER(P), D, I,
                               ctypes.POINTER(mg_stats), ctypes.POINTER(I), P]),
        "mg_ns_workspace_bytes": (I, [ctypes.POINTER(mg_grid), ctypes.POINTER(mg_params),
                                      ctypes.POINTER(S)]),
        "mg_ns_setup": (I, [ctypes.POINTER(mg_grid), ctypes.POINTER(mg_ns_coeffs),
                            ctypes.POINTER(mg_params), P, S, P, ctypes.POINTER(H)]),
        "mg_ns_destroy": (None, [H]),
        "mg_ns_apply": (I, [H, I, P, P, P]),
        "mg_ns_vcycle": (I, [H, I, P, P, P]),
        "mg_ns_solve": (I, [H, I, P, P, D, ctypes.POINTER(mg_stats), P]),
        "mg_ns_solve_mixed": (I, [H, I, P, P, D, ctypes.POINTER(mg_stats), P]),
        "mg_ns_vcycle_prec": (I, [H, I, I, P, P, P]),
        "mg_ns_fp32_scale": (D, [H]),
        "mg_ns_coeff_grad": (I, [H, P, P, P, P, P, P, P, P, P, P]),
        "mg_ns_num_levels": (I, [H]),
        "mg_ns_level_shape": (I, [H, I, ctypes.POINTER(I), ctypes.POINTER(I),
                                  ctypes.POINTER(I)]),
        "mg_ns_level_coeffs": (I, [H, I, I, P, P, P, P, P, P, P, P]),
        "mg_ns_level_smooth": (I, [H, I, I, I, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(status: int, allow=()) -> int:
    if status != MG_OK and status not in allow:
        msg = load().mg_last_error().decode(errors="replace")
        raise MGError(status, msg)
    return status


def default_params(**kw) -> mg_params:
    p = mg_params()
    load().mg_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p
