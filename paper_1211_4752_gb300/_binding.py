"""ctypes declarations of the C ABI in include/hh.h (argument marshalling only).

The shared library is built in-tree by ``paper_1211_4752_gb300.build``.  If it
is missing, ``lib()`` raises: there is no fallback implementation.
"""

from __future__ import annotations

import ctypes as ct
from pathlib import Path

_LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libhh_gb300.so"

HH_OK = 0
HH_ERR_ARG = 1
HH_ERR_CUDA = 2
HH_ERR_OOM = 3
HH_ERR_NOT_CONVERGED = 4
HH_ERR_DIVERGED = 5
HH_ERR_TIMEOUT = 6
HH_ERR_UNSUPPORTED = 7
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM",
                4: "ERR_NOT_CONVERGED", 5: "ERR_DIVERGED", 6: "ERR_TIMEOUT",
                7: "ERR_UNSUPPORTED"}

HH_FORM_CSL = 0
HH_FORM_CSG = 1
HH_FP64 = 0
HH_MIXED = 1
HH_USE_GUESS = 1
HH_SMOOTH_JACOBI = 0
HH_SMOOTH_GMRES = 1


class HHGrid(ct.Structure):
    _fields_ = [("dim", ct.c_int), ("n", ct.c_int), ("layer_lo", ct.c_int),
                ("layer_hi", ct.c_int), ("ecs_angle", ct.c_double), ("sommerfeld", ct.c_int)]


class HHShift(ct.Structure):
    _fields_ = [("form", ct.c_int), ("theta_max", ct.c_double), ("p", ct.c_int),
                ("theta", ct.POINTER(ct.c_double)),
                ("c", ct.POINTER(ct.c_double))]


class HHOptions(ct.Structure):
    _fields_ = [("omega_re", ct.c_double), ("omega_im", ct.c_double),
                ("nu1", ct.c_int), ("nu2", ct.c_int), ("precision", ct.c_int),
                ("coarsest", ct.c_int), ("max_cycles", ct.c_int),
                ("div_limit", ct.c_double), ("inner_tol", ct.c_double),
                ("max_inner", ct.c_int), ("smoother", ct.c_int), ("gmres_m", ct.c_int),
                ("tuner_cache", ct.c_char_p),
                ("dev_alloc", ct.c_void_p), ("dev_free", ct.c_void_p),
                ("alloc_ctx", ct.c_void_p)]


# allocator callbacks of hh_options (void *(size_t, void *), void (void *, void *))
DEV_ALLOC = ct.CFUNCTYPE(ct.c_void_p, ct.c_size_t, ct.c_void_p)
DEV_FREE = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_void_p)


class HHSolveInfo(ct.Structure):
    _fields_ = [("cycles", ct.c_int), ("refinements", ct.c_int),
                ("rel_residual", ct.c_double), ("status", ct.c_int)]


class HHGroupItem(ct.Structure):
    _fields_ = [("h", ct.c_void_p), ("rhs_dev", ct.c_void_p), ("u_dev", ct.c_void_p),
                ("batch", ct.c_int), ("flags", ct.c_int),
                ("info", ct.POINTER(HHSolveInfo))]


# name -> (restype, argtypes); every symbol include/hh.h declares.
_P = ct.c_void_p
_I = ct.c_int
_D = ct.c_double
SIGNATURES = {
    "hh_default_shift": (None, [ct.POINTER(HHShift)]),
    "hh_default_options": (None, [ct.POINTER(HHOptions)]),
    "hh_setup": (_I, [ct.POINTER(HHGrid), _P, _D, ct.POINTER(HHShift),
                      ct.POINTER(HHOptions), _I, _P, ct.POINTER(_P)]),
    "hh_solve": (_I, [_P, _P, _P, _I, _D, _I, ct.POINTER(HHSolveInfo), _P]),
    "hh_solve_host": (_I, [_P, _P, _P, _I, _D, _I, ct.POINTER(HHSolveInfo), _P]),
    "hh_adjoint": (_I, [_P, _P, _P, _I, _D, _I, ct.POINTER(HHSolveInfo), _P]),
    "hh_fgmres": (_I, [_P, _P, _P, _I, _D, _I, _I, _I, ct.POINTER(HHSolveInfo), _P]),
    "hh_solve_group": (_I, [ct.POINTER(HHGroupItem), _I, _D, _P]),
    "hh_group_create": (_I, [ct.POINTER(_P), ct.POINTER(_I), _I, ct.POINTER(_P)]),
    "hh_group_solve": (_I, [_P, ct.POINTER(HHGroupItem), _D, _P]),
    "hh_group_kernels": (ct.c_longlong, [_P]),
    "hh_group_destroy": (_I, [_P]),
    "hh_grad_k2": (_I, [_P, _P, _P, _I, _P, _P]),
    "hh_apply": (_I, [_P, _I, _I, _P, _P, _I, _P]),
    "hh_cycles": (_I, [_P, _P, _P, _I, _I, _P]),
    "hh_smooth": (_I, [_P, _I, _P, _P, _P, _I, _P]),
    "hh_residual_restrict": (_I, [_P, _I, _P, _P, _P, _I, _P]),
    "hh_correct_smooth": (_I, [_P, _I, _P, _P, _P, _P, _I, _P]),
    "hh_coarse_solve": (_I, [_P, _P, _P, _I, _P]),
    "hh_time_kernel": (_I, [_P, _I, _I, _I, _I, ct.POINTER(_D), _P]),
    "hh_num_levels": (_I, [_P]),
    "hh_level_points": (_I, [_P, _I]),
    "hh_cycle_kernels": (_I, [_P]),
    "hh_solve_kernels": (ct.c_longlong, [_P]),
    "hh_rel_residual_static": (_I, [_P, _P, _P, _I, _P, _P]),
    "hh_tile_shape": (_I, [_P, _I, ct.POINTER(_I), ct.POINTER(_I)]),
    "hh_tuner_key": (_I, [_P, ct.c_char_p, _I]),
    "hh_coarse_schedule": (_I, [_P, ct.POINTER(_I), _I]),
    "hh_test_barrier_timeout": (_I, [_P, _I]),
    "hh_destroy": (_I, [_P]),
    "hh_last_error": (ct.c_char_p, []),
}

_lib = None


def lib_path() -> Path:
    return _LIB_PATH


def lib() -> ct.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise RuntimeError(
                f"{_LIB_PATH} is missing: build the CUDA library first "
                "(python -m paper_1211_4752_gb300.build); there is no CPU "
                "fallback")
        L = ct.CDLL(str(_LIB_PATH))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class HHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status):
    if status != HH_OK:
        msg = lib().hh_last_error()
        raise HHError(status, msg.decode() if msg else "")
    return status
