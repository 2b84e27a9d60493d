"""ctypes loader of libgenp.so (the C ABI declared in include/genp.h).

The library is built in-tree by ``paper_1212_4560_gb300.build``.  There is
no fallback: if it is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgenp.so")

GENP_OK = 0
STATUS_NAMES = {0: "GENP_OK", -1: "GENP_ERR_ARG", -2: "GENP_ERR_BREAKDOWN", -3: "GENP_ERR_NOCONV",
                -4: "GENP_ERR_CUDA", -5: "GENP_ERR_TIMEOUT", -6: "GENP_ERR_NOMEM", -7: "GENP_ERR_UNSUPPORTED"}

GAUSSIAN, CIRCULANT, SPARSE_PM1, CIRCULANT_PM1, IDENTITY, TOEPLITZ, HOUSEHOLDER_PM1 = 0, 1, 2, 3, 4, 5, 6
RIGHT, LEFT = 0, 1
PROF_TENSOR, PROF_TRSV, PROF_GEMV, PROF_FACTOR_AUX, PROF_OUTER, PROF_PRECOND = 0, 1, 2, 3, 4, 5
FP64, FP32, BF16, FP8_E4M3, BF16X3, BF16_SLICED = 0, 1, 2, 3, 4, 5
MAX_REFINE = 32

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_int = ctypes.c_int
_dbl = ctypes.c_double


class GenpInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("refine_iters", ctypes.c_int32), ("breakdown_step", ctypes.c_int64),
                ("min_abs_pivot", _dbl), ("max_abs_pivot", _dbl), ("growth", _dbl),
                ("bwd_err", _dbl * (MAX_REFINE + 1)), ("krylov_steps", ctypes.c_int32), ("reserved", ctypes.c_int32)]


# name -> (restype, argtypes); every entry point of include/genp.h
SIGNATURES = {
    "genp_version": (ctypes.c_char_p, []),
    "genp_status_string": (ctypes.c_char_p, [_int]),
    "genp_make_multiplier": (_int, [_int, _i64, _u64, _u64, _dbl, _int, _int, _vp, ctypes.POINTER(_vp)]),
    "genp_redraw_multiplier": (_int, [_vp, _u64, _u64, _vp]),
    "genp_multiplier_side": (_int, [_vp, _int]),
    "genp_launch_count": (_u64, []),
    "genp_make_sparse_noalloc": (_int, [_i64, _int, _u64, _u64, _vp, _vp, _vp, _vp, _vp]),
    "genp_gemm_bf16": (_int, [_i64, _i64, _i64, ctypes.c_float, _vp, _i64, _vp, _i64, ctypes.c_float, _vp, _i64,
                              _vp, _i64, _vp]),
    "genp_quantize_e4m3": (_int, [_vp, _i64, _int, _i64, _i64, _int, _vp, _i64, _vp, _vp]),
    "genp_gemm_e4m3": (_int, [_i64, _i64, _i64, ctypes.c_float, _vp, _i64, _vp, _vp, _i64, _vp, ctypes.c_float, _vp,
                              _i64, _vp, _i64, _vp]),
    "genp_gemm_sliced": (_int, [_i64, _i64, _i64, _dbl, _vp, _i64, _vp, _i64, _dbl, _vp, _i64, _int, _vp]),
    "genp_numerical_rank": (_int, [_i64, _i64, _vp, _i64, _i64, _i64, _dbl, _u64, _u64, _vp, _vp, _i64, _vp]),
    "genp_lowrank": (_int, [_i64, _i64, _vp, _i64, _i64, _int, _u64, _u64, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64,
                            _vp, _vp]),
    "genp_sliced_digits": (_int, [_int]),
    "genp_sliced_precondition_digits": (_int, [_int]),
    "genp_sliced_multiplier_digits": (_int, [_int]),
    "genp_profile_enable": (_int, [_int]),
    "genp_profile_read": (_int, [_vp, _vp, _vp]),
    "genp_profile_launches": (_int, [_vp, _vp, _int, _vp]),
    "genp_profile_class": (_int, [_int, _vp, _vp, _vp]),
    "genp_refine_graphs": (_int, [_int]),
    "genp_device_check": (_int, [_int]),
    "genp_batched_plan_create": (_int, [_i64, _vp, _i64, _int, _int, _int, _dbl, _int, _vp, ctypes.POINTER(_vp)]),
    "genp_batched_layout": (_int, [_vp, _vp, _vp]),
    "genp_batched_block_size": (_int, [_vp, _i64]),
    "genp_batched_run": (_int, [_vp, _u64, _vp, _vp, _vp, _vp]),
    "genp_batched_adjoint": (_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "genp_batched_status": (_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "genp_batched_profile": (_int, [_vp, _int]),
    "genp_batched_profile_read": (_int, [_vp, _vp, _vp]),
    "genp_batched_multipliers": (_int, [_vp, _vp, _vp, _vp]),
    "genp_batched_plan_destroy": (None, [_vp]),
    "genp_multiplier_export": (_int, [_vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    "genp_multiplier_query": (_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "genp_multiplier_destroy": (None, [_vp]),
    "genp_precondition": (_int, [_vp, _vp, _i64, _int, _vp, _i64, _int, _vp]),
    "genp_factor": (_int, [_vp, _i64, _i64, _int, _i64, _vp, ctypes.POINTER(_vp)]),
    "genp_refactor": (_int, [_vp, _vp, _i64, _vp]),
    "genp_block_factor": (_int, [_vp, _i64, _i64, _i64, _vp, ctypes.POINTER(_vp)]),
    "genp_factors_destroy": (None, [_vp]),
    "genp_solve": (_int, [_vp, _vp, _vp, _i64, _i64, _vp, _i64, _vp]),
    "genp_refine": (_int, [_vp, _i64, _vp, _vp, _vp, _i64, _i64, _vp, _i64, _dbl, _int, _int, _vp]),
    "genp_adjoint": (_int, [_vp, _vp, _vp, _i64, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp]),
    "genp_info_fetch": (_int, [_vp, ctypes.POINTER(GenpInfo), _vp]),
}

_lib = None


class GenpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


def load():
    """Returns the loaded library, raising if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgenp.so is not built ({LIB_PATH}); run paper_1212_4560_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != GENP_OK:
        raise GenpError(status, where)
