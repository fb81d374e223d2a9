"""ctypes declarations of the C ABI in ``include/rkab.h``.

Loads the in-tree ``librkab.so``; there is no fallback: if the library is
missing or fails to load, importing the binding raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librkab.so")

RK_OK = 0
RK_EINVAL = -1
RK_EALIGN = -2
RK_ENOTCORESIDENT = -3
RK_ETIMEOUT = -4
RK_EDIVERGED = -5
RK_ECUDA = -6
RK_EWORKSPACE = -7
RK_ESETUP = -8
RK_ETOOLARGE = -9

RK_F32, RK_BF16, RK_FP8E4M3 = 0, 1, 2


class RkOpts(ctypes.Structure):
    """Mirror of ``rk_opts``."""
    _fields_ = [
        ("omega", ctypes.c_float),
        ("check_every", ctypes.c_int64),
        ("tol", ctypes.c_double),
        ("criterion", ctypes.c_int),
        ("x_ref", ctypes.c_void_p),
        ("round0", ctypes.c_int64),
        ("stream_id", ctypes.c_uint32),
        ("same_stream", ctypes.c_int),
        ("cluster_size", ctypes.c_int),
        ("timeout_s", ctypes.c_double),
        ("lookahead", ctypes.c_int),
        ("sampling", ctypes.c_int),
        ("row_weight", ctypes.c_void_p),
        ("worker_weight", ctypes.c_void_p),
    ]


# name -> (restype, argtypes); every function declared in include/rkab.h
_V = ctypes.c_void_p
_SIG = {
    "rk_opts_default": (None, [ctypes.POINTER(RkOpts)]),
    "rk_setup_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64]),
    "rk_setup": (ctypes.c_int, [_V, ctypes.c_int, _V, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_int64, _V, ctypes.c_size_t, _V, ctypes.POINTER(_V)]),
    "rk_plan_status": (ctypes.c_int, [_V, _V, ctypes.POINTER(ctypes.c_uint64),
                                      ctypes.POINTER(ctypes.c_int32)]),
    "rk_plan_tables": (ctypes.c_int, [_V, ctypes.POINTER(_V), ctypes.POINTER(_V),
                                      ctypes.POINTER(_V), ctypes.POINTER(_V),
                                      ctypes.POINTER(_V)]),
    "rk_plan_destroy": (None, [_V]),
    "rk_plan_frobenius2": (ctypes.c_int, [_V, _V, ctypes.POINTER(ctypes.c_double)]),
    "rk_sample_indices": (ctypes.c_int, [_V, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_uint64, ctypes.c_int64, _V, _V]),
    "rk_sample_indices_ex": (ctypes.c_int, [_V, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_int, ctypes.c_uint64,
                                            ctypes.c_int64, _V, _V]),
    "rk_solve_workspace_bytes": (ctypes.c_size_t, [_V, ctypes.c_int]),
    "rkab_solve": (ctypes.c_int, [_V, _V, _V, _V, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_uint64, ctypes.POINTER(RkOpts), _V, ctypes.c_size_t,
                                  _V]),
    "rkab_solve_noalloc": (ctypes.c_int, [_V, _V, _V, _V, ctypes.c_int, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(RkOpts),
                                          _V, _V]),
    "rka_solve": (ctypes.c_int, [_V, _V, _V, _V, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                 ctypes.POINTER(RkOpts), _V, ctypes.c_size_t, _V]),
    "rk_solve_status": (ctypes.c_int, [_V, _V, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_double)]),
    "rk_quantize": (ctypes.c_int, [_V, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_int, _V, ctypes.c_int64, _V, _V]),
    "rk_refine_workspace_bytes": (ctypes.c_size_t, [_V, ctypes.c_int]),
    "rkab_refine": (ctypes.c_int, [_V, _V, ctypes.c_int64, _V, _V, _V, ctypes.c_int,
                                   ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                   ctypes.POINTER(RkOpts), _V, ctypes.c_size_t, _V,
                                   ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_double)]),
    "rk_transpose": (ctypes.c_int, [_V, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _V,
                                    ctypes.c_int64, _V]),
    "rk_rank2": (ctypes.c_int, [_V, _V, _V, _V, ctypes.c_int64, ctypes.c_int64, _V, ctypes.c_int64,
                                _V]),
    "rk_adjoint_workspace_bytes": (ctypes.c_size_t, [_V, _V, ctypes.c_int, ctypes.c_int]),
    "rkab_adjoint": (ctypes.c_int, [_V, _V, _V, _V, _V, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                    ctypes.c_int64,
                                    ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                    ctypes.POINTER(RkOpts), ctypes.POINTER(RkOpts), _V, _V, _V,
                                    ctypes.c_int64, _V, ctypes.c_size_t, _V]),
    "rk_residual_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64]),
    "rk_residual": (ctypes.c_int, [_V, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _V, _V,
                                   _V, _V, ctypes.c_int, _V, ctypes.c_size_t, _V]),
    "rk_solve_residual_workspace_bytes": (ctypes.c_size_t, [_V, ctypes.c_int]),
    "rkab_solve_residual": (ctypes.c_int, [_V, _V, ctypes.c_int64, _V, _V, _V, ctypes.c_int,
                                           ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_uint64, ctypes.POINTER(RkOpts), ctypes.c_int,
                                           ctypes.c_double, _V, ctypes.c_size_t, _V,
                                           ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_double)]),
    "rk_alpha_star": (ctypes.c_double, [ctypes.c_int, ctypes.c_double, ctypes.c_double]),
    "rk_spectrum_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int]),
    "rk_spectrum": (ctypes.c_int, [_V, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_uint64, _V, ctypes.c_size_t, _V,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "rk_spectrum_ex": (ctypes.c_int, [_V, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_uint64, ctypes.c_double, _V, ctypes.c_size_t, _V,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "rk_spectrum_ratios": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]),
    "rk_optimal_weight": (ctypes.c_int, [_V, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_uint64, ctypes.c_double, _V, ctypes.c_size_t,
                                         _V, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int)]),
    "rk_partial_alpha_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                                           ctypes.c_int]),
    "rk_partial_alpha_star": (ctypes.c_int, [_V, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_uint64, _V, ctypes.c_size_t, _V,
                                             ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)]),
    "rk_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "rk_launch_count": (ctypes.c_uint64, []),
}

_lib = None


def load():
    """Load librkab.so and declare every exported function (raises if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIG.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_functions():
    return list(_SIG)


class RkError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = load().rk_strerror(code).decode()
        super().__init__(f"{what}: {msg} (code {code})" if what else f"{msg} (code {code})")


def check(code: int, what: str = ""):
    if code != RK_OK:
        raise RkError(code, what)
