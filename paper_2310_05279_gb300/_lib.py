"""ctypes declarations of the C ABI in include/d3gb.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libd3gb.so")

D3_OK, D3_ERR_ARG, D3_ERR_CUDA, D3_ERR_CAPACITY, D3_ERR_NONFINITE, D3_ERR_TIMEOUT, D3_ERR_TYPE, D3_ERR_STATE = range(8)
D3_FP64, D3_MIXED = 0, 1
STATUS_NAMES = {0: "D3_OK", 1: "D3_ERR_ARG", 2: "D3_ERR_CUDA", 3: "D3_ERR_CAPACITY", 4: "D3_ERR_NONFINITE",
                5: "D3_ERR_TIMEOUT", 6: "D3_ERR_TYPE", 7: "D3_ERR_STATE"}

# Every symbol include/d3gb.h declares, with (restype, argtypes).
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)
_vp = C.c_void_p


class D3Params(C.Structure):
    _fields_ = [("s6", C.c_double), ("s8", C.c_double), ("a1", C.c_double), ("a2_bohr", C.c_double),
                ("k1", C.c_double), ("k2", C.c_double), ("k3", C.c_double), ("rc_disp_A", C.c_double),
                ("rc_cn_A", C.c_double), ("skin_A", C.c_double), ("precision", C.c_int32)]


class D3Tables(C.Structure):
    _fields_ = [("ntypes", C.c_int32), ("max_ref", C.c_int32), ("nref", _ip), ("cn_ref", _dp),
                ("c6_ref", _dp), ("rcov_bohr", _dp), ("sqrtq", _dp)]


SIGNATURES = {
    "d3_create": (C.c_int, [C.POINTER(D3Params), C.POINTER(D3Tables), C.POINTER(_vp)]),
    "d3_destroy": (None, [_vp]),
    "d3_set_damping": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, C.c_double]),
    "d3_build_neighbors": (C.c_int, [_vp, C.c_int32, _lp, _vp, _vp, _dp, _ip, _vp]),
    "d3_compute": (C.c_int, [_vp, _vp, _vp, C.c_int64, _dp, _ip, _vp, _vp, _vp, _vp]),
    "d3_compute_batch": (C.c_int, [_vp, C.c_int32, _lp, _vp, _vp, _dp, _ip, _vp, _vp, _vp, _vp]),
    "d3_compute_batch_ex": (C.c_int, [_vp, C.c_int32, _lp, _vp, _vp, _dp, _ip, _vp, _vp, _vp, _vp, _vp, _vp]),
    "d3_compute_batch_host": (C.c_int, [_vp, C.c_int32, _lp, _vp, _vp, _dp, _ip, _vp, _vp, _vp, _vp]),
    "d3_compute_batch_atoms": (C.c_int, [_vp, C.c_int32, _lp, _vp, _vp, _dp, _ip, _vp, _vp, _vp, _vp, _vp, _vp,
                                         _vp]),
    "d3_heat_current": (C.c_int, [C.c_int64, _vp, _vp, _vp, _vp]),
    "d3_backward": (C.c_int, [_vp, C.c_int32, _lp, _vp, _vp, _dp, _ip, _vp, _vp, _vp, _vp, _vp]),
    "d3_sync_status": (C.c_int, [_vp]),
    "d3_last_error": (C.c_char_p, [_vp]),
    "d3_build_count": (C.c_int, [_vp, _lp]),
    "d3_set_accumulate": (C.c_int, [_vp, C.c_int32]),
    "d3_set_three_body": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double]),
    "d3_set_graphs": (C.c_int, [_vp, C.c_int32]),
    "d3_set_autotune": (C.c_int, [_vp, C.c_int32]),
    "d3_launch_shapes": (C.c_int, [_vp, _ip, _lp]),
    "d3_set_launch_shapes": (C.c_int, [_vp, _ip]),
    "d3_version": (C.c_char_p, []),
    "d3_profile_enable": (C.c_int, [_vp, C.c_int32]),
    "d3_profile_read": (C.c_int, [_vp, _dp, _lp, _lp]),
    "d3_profile_reset": (C.c_int, [_vp]),
    "d3_structure_energies_noalloc": (C.c_int, [C.c_int32, _lp, _vp, _vp, _vp]),
    "d3_profile_stage": (C.c_int, [_vp, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "d3_list_stats": (C.c_int, [_vp, C.POINTER(C.c_int64)]),
    "d3_tune_times": (C.c_int, [_vp, C.POINTER(C.c_float)]),
    "d3_peak_rates": (C.c_int, [C.POINTER(C.c_double), _vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libd3gb.so.  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2310_05279_gb300.build` "
                           "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib
