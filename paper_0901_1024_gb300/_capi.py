"""ctypes declarations of the C ABI in include/dg.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdg.so")

DG_OK = 0
ERRORS = {-1: "DG_ERR_ARG", -2: "DG_ERR_MESH", -3: "DG_ERR_ORDER", -4: "DG_ERR_CUDA",
          -5: "DG_ERR_OOM", -6: "DG_ERR_UNSTABLE", -7: "DG_ERR_STATE"}

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_intp = C.POINTER(C.c_int)
_vp = C.c_void_p

# name -> (restype, argtypes); the complete exported surface of include/dg.h
SIGNATURES = {
    "dg_mesh_create": (C.c_int, [_dp, C.c_int64, _ip, C.c_int64, C.POINTER(_vp)]),
    "dg_set_order": (C.c_int, [_vp, C.c_int]),
    "dg_mesh_pack": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(_vp)]),
    "dg_info": (C.c_int, [_vp, _i64p, _intp, _intp, _dp]),
    "dg_nodes": (C.c_int, [_vp, _dp]),
    "dg_get_connectivity": (C.c_int, [_vp, _ip, _ip]),
    "dg_partition_order": (C.c_int, [_vp, C.c_int64, _i64p]),
    "dg_get_operators": (C.c_int, [_vp, _dp, _dp, _dp, _dp, _dp]),
    "dg_get_geometry": (C.c_int, [_vp, _dp, _dp, _dp, _dp]),
    "dg_set_flux": (C.c_int, [_vp, C.c_double]),
    "dg_set_materials": (C.c_int, [_vp, _dp, _dp]),
    "dg_set_boundary": (C.c_int, [_vp, _vp]),
    "dg_set_stage_impl": (C.c_int, [_vp, C.c_int]),
    "dg_set_energy_check": (C.c_int, [_vp, C.c_double]),
    "dg_set_stage_shape": (C.c_int, [_vp, C.c_int]),
    "dg_rhs": (C.c_int, [_vp, _vp, _vp, _vp]),
    "dg_step": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_int, _vp]),
    "dg_rk_stage": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, C.c_double, _vp]),
    "dg_rk_stage_elem": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, _vp, _vp]),
    "dg_rk_stage_range": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, C.c_double, C.c_int64, C.c_int64,
                                    _vp]),
    "dg_stage_tile": (C.c_int, [_vp, _vp, _vp, _vp, _intp]),
    "dg_check_wait_timeout": (C.c_int, [_vp, C.c_uint32, _dp]),
    "dg_rk_stage_multi": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(_vp), C.POINTER(_vp),
                                    C.POINTER(_vp), C.POINTER(_vp), C.c_int, C.c_double,
                                    C.POINTER(C.c_double), _vp]),
    "dg_energy": (C.c_int, [_vp, _vp, _dp, _vp]),
    "dg_energy_range": (C.c_int, [_vp, _vp, C.c_int64, C.c_int64, _dp, _vp]),
    "dg_energy_noalloc": (C.c_int, [_vp, _vp, _vp, _vp]),
    "dg_step_host": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_int, _dp, _vp]),
    "dg_last_launch_count": (C.c_int64, [_vp]),
    "dg_trace_enable": (C.c_int, [_vp, C.c_int]),
    "dg_trace_read": (C.c_int, [_vp, _dp, _ip, C.c_int64, _i64p]),
    "dg_mesh_destroy": (None, [_vp]),
    "dg_last_error": (C.c_char_p, []),
}

_lib = None


def library_path() -> str:
    return _LIB_PATH


def load() -> C.CDLL:
    """Load libdg.so from the package directory; raise if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(
                f"{_LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        lib = C.CDLL(_LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class DGError(RuntimeError):
    def __init__(self, code: int, fn: str, msg: str):
        super().__init__(f"{fn} failed with {ERRORS.get(code, code)}: {msg}")
        self.code = code


def check(code: int, fn: str):
    if code != DG_OK:
        raise DGError(code, fn, load().dg_last_error().decode())
