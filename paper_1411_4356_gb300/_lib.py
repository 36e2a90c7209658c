"""ctypes declarations for libomss.so (include/omss.h).

Loading fails loudly if the library has not been built; there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_i32, c_i64, c_dbl, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class om_params(ctypes.Structure):
    _fields_ = [("Nc", c_i32), ("Nm", c_i32), ("omega_m", c_dbl), ("Delta", c_dbl), ("kappa", c_dbl),
                ("g0", c_dbl), ("E", c_dbl), ("Q_m", c_dbl), ("n_th", c_dbl), ("g2", c_dbl), ("lam", c_dbl)]


class om_build_opts(ctypes.Structure):
    _fields_ = [("trace_mode", c_i32), ("nth_floor", c_dbl)]


class om_solve_opts(ctypes.Structure):
    _fields_ = [("restart", c_i32), ("max_iters", c_i32), ("precision", c_i32), ("precond_fp64", c_i32),
                ("tol", c_dbl), ("wait_timeout_ns", c_i64)]


class om_solve_info(ctypes.Structure):
    _fields_ = [("iterations", c_i32), ("cycles", c_i32), ("eta", c_dbl), ("trace_before", c_dbl),
                ("seconds", c_dbl), ("residual_history", c_dbl * 64)]


STATUS = {0: "OM_OK", -1: "OM_EINVAL", -2: "OM_ENOMEM", -3: "OM_ECUDA", -4: "OM_EZEROPIVOT",
          -5: "OM_ENOCONV", -6: "OM_EBREAKDOWN", -7: "OM_ENUMERIC", -8: "OM_ETIMEOUT"}

ALLOC_FN = ctypes.CFUNCTYPE(c_vp, ctypes.c_size_t, c_vp, c_vp)
FREE_FN = ctypes.CFUNCTYPE(None, c_vp, c_vp, c_vp)

# name -> (restype, argtypes); every entry point declared in include/omss.h
SIGNATURES = {
    "om_set_allocator": (c_i32, [ALLOC_FN, FREE_FN, c_vp]),
    "om_allocator_hook_calls": (c_i64, []),
    "om_build_liouvillian": (c_i32, [ctypes.POINTER(om_params), ctypes.POINTER(om_build_opts), c_vp, ctypes.POINTER(c_vp)]),
    "om_matrix_info": (c_i32, [c_vp, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64), ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl)]),
    "om_matrix_export": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "om_permute": (c_i32, [c_vp, c_vp, c_vp, ctypes.POINTER(c_vp)]),
    "om_permute_ex": (c_i32, [c_vp, c_i32, c_vp, c_vp, ctypes.POINTER(c_vp)]),
    "om_ilu_factor": (c_i32, [c_vp, c_dbl, c_dbl, c_i32, c_vp, ctypes.POINTER(c_vp)]),
    "om_steady_state_sweep_nojump": (c_i32, [c_i32, c_vp, ctypes.POINTER(om_build_opts), c_i32,
                                             ctypes.POINTER(om_solve_opts), c_vp, c_vp, c_vp, c_i32, c_vp]),
    "om_liouvillian_row_host": (c_i32, [ctypes.POINTER(om_params), ctypes.POINTER(om_build_opts), c_i64, c_vp, c_vp,
                                        ctypes.POINTER(c_i32)]),
    "om_rcm_order_host": (c_i32, [c_i64, c_vp, c_vp, c_vp]),
    "om_ilu_factor_host": (c_i32, [c_i64, c_vp, c_vp, c_vp, c_dbl, c_dbl, c_dbl, c_i32, ctypes.POINTER(c_vp)]),
    "om_host_ilu_sizes": (c_i32, [c_vp] + [ctypes.POINTER(c_i64)] * 4),
    "om_host_ilu_export": (c_i32, [c_vp] + [c_vp] * 10),
    "om_host_ilu_free": (None, [c_vp]),
    "om_ilutp_factor": (c_i32, [c_vp, c_dbl, c_dbl, c_dbl, c_i32, c_vp, ctypes.POINTER(c_vp)]),
    "om_ilu_pivots": (c_i32, [c_vp, ctypes.POINTER(c_i32), ctypes.POINTER(c_i64), c_vp, c_vp]),
    "om_ilu_info": (c_i32, [c_vp] + [ctypes.POINTER(c_i64)] * 5),
    "om_ilu_timings": (c_i32, [c_vp, ctypes.POINTER(c_dbl)]),
    "om_steady_state_solve": (c_i32, [c_vp, c_vp, c_vp, ctypes.POINTER(om_solve_opts), c_vp, c_vp,
                                      ctypes.POINTER(om_solve_info), c_vp]),
    "om_steady_state_adjoint": (c_i32, [c_vp, c_vp, c_vp, ctypes.POINTER(om_solve_opts), ctypes.POINTER(om_params),
                                        c_vp, c_vp, ctypes.POINTER(c_dbl * 4), ctypes.POINTER(om_solve_info), c_vp]),
    "om_steady_state_solve_batched": (c_i32, [c_i32, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp), ctypes.POINTER(c_vp),
                                              ctypes.POINTER(om_solve_opts), ctypes.POINTER(c_vp),
                                              ctypes.POINTER(om_solve_info), ctypes.POINTER(c_i32), c_i32, c_vp]),
    "om_nojump_factor": (c_i32, [ctypes.POINTER(om_params), ctypes.POINTER(om_build_opts), c_i32, c_vp,
                                 ctypes.POINTER(c_vp)]),
    "om_nojump_info": (c_i32, [c_vp, ctypes.POINTER(c_i32), ctypes.POINTER(c_i32), ctypes.POINTER(c_dbl),
                               ctypes.POINTER(c_dbl * 3)]),
    "om_nojump_apply": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp]),
    "om_steady_state_solve_nojump": (c_i32, [c_vp, c_vp, ctypes.POINTER(om_solve_opts), c_vp, c_vp,
                                             ctypes.POINTER(om_solve_info), c_vp]),
    "om_steady_state_adjoint_nojump": (c_i32, [c_vp, c_vp, ctypes.POINTER(om_solve_opts), ctypes.POINTER(om_params),
                                               c_vp, c_vp, ctypes.POINTER(c_dbl * 4), ctypes.POINTER(om_solve_info),
                                               c_vp]),
    "om_nojump_free": (None, [c_vp]),
    "om_spmv": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "om_liouvillian_apply": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "om_ilu_apply": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp]),
    "om_ilu_apply_noalloc": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_vp]),
    "om_ilu_condest": (c_i32, [c_vp, c_i32, ctypes.POINTER(c_dbl), c_vp]),
    "om_observables": (c_i32, [c_i32, c_i32, c_vp, ctypes.POINTER(c_dbl * 2), c_vp]),
    "om_phonon_distribution": (c_i32, [c_i32, c_i32, c_vp, c_vp, ctypes.POINTER(c_dbl * 3), c_vp]),
    "om_kernel_launches": (c_i64, []),
    "om_profile": (c_i32, [c_i32]),
    "om_profile_read": (c_i32, [c_i32, ctypes.POINTER(c_dbl), ctypes.POINTER(c_i64)]),
    "om_matrix_free": (None, [c_vp]),
    "om_ilu_free": (None, [c_vp]),
    "om_status_str": (ctypes.c_char_p, [c_i32]),
    "om_last_error": (ctypes.c_char_p, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libomss.so; builds it first when missing or stale (nvcc required)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libomss.so not found at {path}: run paper_1411_4356_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class OMError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != 0:
        raise OMError(status, where, (load().om_last_error() or b"").decode())
