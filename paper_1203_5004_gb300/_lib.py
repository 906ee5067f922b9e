"""ctypes declarations of libwagener.so (include/wg.h). Argument marshalling only.

The library is loaded from this package directory. If it is missing the
import fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwagener.so")

WG_OK = 0
STATUS_NAMES = {
    0: "WG_OK", 1: "WG_ERR_INVALID_VALUE", 2: "WG_ERR_WORKSPACE", 3: "WG_ERR_UNSORTED",
    4: "WG_ERR_OFF_GRID", 5: "WG_ERR_TIMEOUT", 6: "WG_ERR_CUDA", 7: "WG_ERR_UNSUPPORTED",
}
WG_PRED_FILTERED = 0
WG_PRED_FP64 = 1
NUM_TILE_CONFIGS = 4

# Every function the header declares, with (restype, argtypes).
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_sz = ctypes.c_size_t


class Options(ctypes.Structure):
    _fields_ = [
        ("pred_mode", _i32),
        ("count_predicates", _i32),
        ("validate", _i32),
        ("tile_config", _i32),
        ("segments_per_cta", _i32),
        ("schedule", _i32),
        ("batch_seg_tiles", _i32),
        ("reserved", _i32 * 1),
    ]


_OPT_P = ctypes.POINTER(Options)

SIGNATURES = {
    "wg_options_default": (None, [_OPT_P]),
    "wg_upper_hood_workspace_size": (_sz, [_i64]),
    "wg_upper_hood": (_i32, [_vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "wg_upper_hood_ex": (_i32, [_vp, _i64, _vp, _vp, _vp, _sz, _OPT_P, _vp]),
    "wg_convex_hull_workspace_size": (_sz, [_i64]),
    "wg_convex_hull": (_i32, [_vp, _i64, _vp, _vp, _vp, _sz, _OPT_P, _vp]),
    "wg_sort_points_workspace_size": (_sz, [_i64]),
    "wg_sort_points": (_i32, [_vp, _i64, _vp, _vp, _vp, _sz, _vp]),
    "wg_upper_hood_unsorted_workspace_size": (_sz, [_i64]),
    "wg_upper_hood_unsorted": (_i32, [_vp, _i64, _vp, _vp, _vp, _sz, _OPT_P, _vp]),
    "wg_upper_hood_plain_workspace_size": (_sz, [_i64]),
    "wg_upper_hood_plain": (_i32, [_vp, _i64, _vp, _vp, _vp, _sz, _OPT_P, _vp]),
    "wg_upper_hood_batched_workspace_size": (_sz, [_vp, _i32]),
    "wg_upper_hood_batched": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, _sz, _OPT_P, _vp]),
    "wg_upper_hood_from_host": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _OPT_P, _vp]),
    "wg_get_device_status": (_i32, [_vp, _vp]),
    "wg_read_counters": (_i32, [_vp, _vp, _vp, _vp]),
    "wg_status_string": (ctypes.c_char_p, [_i32]),
    "wg_autotune": (_i32, [_vp, _i64, _vp, _vp, _vp, _sz, _OPT_P, _vp]),
    "wg_autotune_batched": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, _sz, _OPT_P, _vp]),
    "wg_debug_orient": (_i32, [_vp, _i64, _vp, _vp, _i32, _vp]),
    "wg_debug_bridge": (_i32, [_vp, _i32, _vp, _i32, _vp, _i32, _vp]),
    "wg_debug_warp_hood": (_i32, [_vp, _i32, _vp, _vp, _i32, _vp]),
    "wg_debug_bridge_cta": (_i32, [_vp, _i32, _vp, _i32, _vp, _i32, _vp]),
    "wg_debug_set_stall": (_i32, [_vp, _i32, _vp]),
    "wg_upper_hood_noalloc": (_i32, [_vp, _i64, _vp, _vp, _vp]),
    "wg_version": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


class WagenerError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        name = STATUS_NAMES.get(code, str(code))
        super().__init__(f"{where}: {name}" if where else name)


def load():
    """Load libwagener.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(code: int, where: str = "") -> None:
    if code != WG_OK:
        raise WagenerError(code, where)


def default_options(**kw) -> Options:
    o = Options()
    load().wg_options_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o
