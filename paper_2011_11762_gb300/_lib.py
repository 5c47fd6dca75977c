"""ctypes declarations of libcht's C ABI (include/cht.h)."""

from __future__ import annotations

import ctypes
import os

from . import build as _build

_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_PVP = ctypes.POINTER(_VP)
_PI64 = ctypes.POINTER(_I64)
_PI32 = ctypes.POINTER(_I32)
_PD = ctypes.POINTER(ctypes.c_double)

# name: (restype, argtypes)
SIGNATURES = {
    "cht_set_allocator": (ctypes.c_int, [_VP, _VP, _VP]),
    "cht_mat_from_blocks": (ctypes.c_int, [_I64, _I32, _I64, _VP, _VP, _VP, _VP, _PVP]),
    "cht_mat_info": (ctypes.c_int, [_VP, _PI64, _PI32, _PI64]),
    "cht_mat_leaves": (ctypes.c_int, [_VP, _PVP, _PVP, _PVP]),
    "cht_to_dense": (ctypes.c_int, [_VP, _VP, _I64, _VP]),
    "cht_mat_like": (ctypes.c_int, [_VP, _VP, _PVP]),
    "cht_mat_free": (ctypes.c_int, [_VP]),
    "cht_symbolic_multiply": (ctypes.c_int, [_VP, _VP, _VP, _PVP, _PI64, _PI64]),
    "cht_symbolic_multiply_spamm": (ctypes.c_int, [_VP, _VP, ctypes.c_double, _VP, _PVP,
                                                   _PI64, _PI64]),
    "cht_symbolic_multiply_symsquare": (ctypes.c_int, [_VP, _VP, _PVP, _PI64, _PI64]),
    "cht_symbolic_multiply_upper": (ctypes.c_int, [_VP, _VP, _VP, _PVP, _PI64, _PI64]),
    "cht_mat_mirror_upper": (ctypes.c_int, [_VP, _VP, _PVP]),
    "cht_add": (ctypes.c_int, [ctypes.c_double, _VP, ctypes.c_double, _VP, _VP, _PVP]),
    "cht_add_identity": (ctypes.c_int, [ctypes.c_double, _VP, ctypes.c_double, _VP, _PVP]),
    "cht_truncate": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int, _VP, _PVP,
                                    ctypes.POINTER(ctypes.c_double)]),
    "cht_multiply_to_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int32]),
    "cht_plan_info": (ctypes.c_int, [_VP, _PI64, _PI64]),
    "cht_plan_arrays": (ctypes.c_int, [_VP, _PVP, _PVP, _PVP, _PVP, _PVP, _PVP]),
    "cht_plan_free": (ctypes.c_int, [_VP]),
    "cht_multiply": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _I32, _VP, _PVP, _PD]),
    "cht_multiply_backward": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, _VP, _PVP,
                                             _PVP]),
    "cht_multiply_f64_noalloc": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "cht_batch_create": (ctypes.c_int, [_I32, _PVP, _PVP, _PVP, ctypes.c_int, _I32, _VP,
                                        _PVP]),
    "cht_batch_run": (ctypes.c_int, [_VP, _VP]),
    "cht_batch_output": (ctypes.c_int, [_VP, _I32, _PVP]),
    "cht_batch_free": (ctypes.c_int, [_VP]),
    "cht_set_option": (ctypes.c_int, [ctypes.c_int, _I64]),
    "cht_get_option": (ctypes.c_int, [ctypes.c_int, _PI64]),
    "cht_sync_status": (ctypes.c_int, [_VP]),
    "cht_launch_count": (_I64, []),
    "cht_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "cht_last_error": (ctypes.c_char_p, []),
    "cht_measure_fp64_peak": (ctypes.c_int, [ctypes.c_int, _VP, _PD]),
    "cht_measure_fp64_peak_cfg": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, _VP, _PD]),
}

_lib = None


def checked() -> bool:
    """CHT_BOUNDS_CHECK=1 selects the bounds-checked debug build."""
    return os.environ.get("CHT_BOUNDS_CHECK", "0") == "1"


def lib_path() -> str:
    return _build.LIB_CHECKED if checked() else _build.LIB


def load(build_if_needed: bool = True):
    """The loaded library.  Builds it from source when it is missing or
    older than its sources; raises if that is impossible (there is no
    fallback implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if build_if_needed and _build.stale(checked()):
        _build.build(checked=checked())
    if not os.path.exists(path):
        raise ImportError(f"libcht is not built ({path}); run build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
