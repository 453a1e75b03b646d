"""ctypes binding of libsvr.so (include/svr.h): argument marshalling only.

The structs mirror the C declarations field for field.  Loading fails loudly
when the library has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# SVR_DEBUG=1 in the environment loads the index-checked build instead
DEBUG = os.environ.get("SVR_DEBUG", "") not in ("", "0")
LIB_PATH = os.path.join(HERE, "libsvr_debug.so" if DEBUG else "libsvr.so")

SVR_OK = 0
SVR_ERR_INVALID = 1
SVR_ERR_LIMIT = 2
SVR_ERR_CAPACITY = 3
SVR_ERR_CUDA = 4
SVR_ERR_TIMEOUT = 5
SVR_FLAG_INVALID_VOXEL = 1
SVR_FLAG_CAPACITY = 2
SVR_FLAG_NO_FORWARD = 4

_P = ctypes.c_void_p


class SvrCamera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("w2c", ctypes.c_float * 12),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class SvrParams(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("t_stop", ctypes.c_float), ("tile", ctypes.c_int32),
                ("bg", ctypes.c_float * 3)]


class SvrScene(ctypes.Structure):
    _fields_ = [("world_center", ctypes.c_float * 3), ("world_size", ctypes.c_float),
                ("n_vox", ctypes.c_int64), ("n_pts", ctypes.c_int64),
                ("max_level", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("centre", _P), ("level", _P), ("corner_idx", _P), ("grid", _P), ("sh", _P)]


SVR_MAX_VIEWS = 32


class SvrFrame(ctypes.Structure):
    _fields_ = [("scene", SvrScene), ("params", SvrParams), ("n_views", ctypes.c_int32),
                ("key_shift", ctypes.c_int32), ("total_tiles", ctypes.c_int64),
                ("cams", SvrCamera * SVR_MAX_VIEWS), ("tile_base", ctypes.c_int32 * (SVR_MAX_VIEWS + 1)),
                ("pixel_base", ctypes.c_int64 * (SVR_MAX_VIEWS + 1)),
                ("ray_origin", (ctypes.c_double * 3) * SVR_MAX_VIEWS),
                ("ws", _P), ("ws_bytes", ctypes.c_size_t), ("pair_capacity", ctypes.c_int64),
                ("n_pairs", ctypes.c_int64), ("stage", ctypes.c_int32),
                ("sorted_alt", ctypes.c_int32), ("offsets", ctypes.c_uint64 * 24)]


class SvrBuffers(ctypes.Structure):
    _fields_ = [("status", _P), ("tile_mask", _P), ("octpath", _P), ("rect", _P), ("count", _P),
                ("offset", _P), ("record", _P), ("keys", _P), ("values", _P), ("ranges", _P)]


class SvrRenderExtras(ctypes.Structure):
    _fields_ = [("normal", _P), ("max_weight", _P), ("d_normal", _P), ("priority", _P), ("distortion", _P),
                ("d_distortion", _P)]


class SvrError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: status {code}: {msg}")
        self.code = code


_LIB = None

# name -> (restype, argtypes)
SIGNATURES = {
    "svr_workspace_size": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64, _P, _P]),
    "svr_workspace_size_views": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64, _P, ctypes.c_int, _P]),
    "svr_preprocess": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_size_t, ctypes.c_int64, _P]),
    "svr_preprocess_views": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, ctypes.c_size_t,
                                            ctypes.c_int64, _P]),
    "svr_render_batched": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P, ctypes.c_size_t,
                                          ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "svr_bin_sort": (ctypes.c_int, [_P, _P, _P]),
    "svr_render_fwd": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "svr_render_bwd": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "svr_render_stats": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "svr_render_fwd_ex": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "svr_render_bwd_ex": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "svr_render_fwd_static": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "svr_l2_loss": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P]),
    "svr_downsample": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int,
                                      ctypes.c_int, _P]),
    "svr_downsample_bwd": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int,
                                          ctypes.c_int, _P]),
    "svr_t_concentration_loss": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_float, _P, _P, _P]),
    "svr_weighted_mean": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_float, _P, _P]),
    "svr_adam": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int64, _P]),
    "svr_frame_status": (ctypes.c_int, [_P, _P, _P, _P]),
    "svr_frame_buffers": (ctypes.c_int, [_P, _P]),
    "svr_last_error": (ctypes.c_char_p, []),
    "svr_version": (ctypes.c_int, []),
    "svr_debug_build": (ctypes.c_int, []),
    "svr_debug_report": (ctypes.c_int, [_P]),
}


def lib():
    """The loaded libsvr.so; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2412_04459_gb300.build.build("
                               f"{'debug=True' if DEBUG else ''}) (nvcc, sm_103a); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def debug_report():
    """(failed checks, site, index, bound) of the current device's index-check
    report (all zero unless the SVR_DEBUG build is loaded); clears it."""
    out = (ctypes.c_uint64 * 4)()
    check(lib().svr_debug_report(out), "svr_debug_report")
    return tuple(int(x) for x in out)


def check(code: int, where: str):
    if code != SVR_OK:
        msg = lib().svr_last_error().decode(errors="replace")
        raise SvrError(code, where, msg)


def ref(x):
    return ctypes.byref(x)
