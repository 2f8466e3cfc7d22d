"""ctypes loader of libges.so and mirrors of the C structs in include/ges.h.

The library is built in-tree on first use (nvcc, sm_103a). There is no
fallback: if it cannot be built or loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

MAX_VIEWS = 32
STATUS_NAMES = {0: "GES_OK", 1: "GES_ERR_INVALID_ARG", 2: "GES_ERR_CAPACITY", 3: "GES_ERR_CUDA",
                4: "GES_ERR_NUMERIC", 5: "GES_ERR_TOO_LARGE", 6: "GES_ERR_BOUNDS"}
GES_OK, GES_ERR_INVALID_ARG, GES_ERR_CAPACITY, GES_ERR_CUDA, GES_ERR_NUMERIC, GES_ERR_TOO_LARGE, GES_ERR_BOUNDS = \
    range(7)
GES_BUILD_DEBUG = 1
NOALLOC_MAX_ENTRIES = 524288


class GESError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)} ({status_string(status)})")


class Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("viewmat", ctypes.c_float * 12), ("znear", ctypes.c_float)]


class Config(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("sh_degree", ctypes.c_int32), ("phi_mode", ctypes.c_int32), ("rho", ctypes.c_float),
                ("lowpass", ctypes.c_float), ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("t_min", ctypes.c_float), ("jac_clamp", ctypes.c_float), ("bg", ctypes.c_float * 3),
                ("persistent", ctypes.c_int32), ("color_storage", ctypes.c_int32)]


class Layout(ctypes.Structure):
    _fields_ = [("proj_records", ctypes.c_uint64), ("proj_binrec", ctypes.c_uint64), ("proj_g2d", ctypes.c_uint64),
                ("proj_bytes", ctypes.c_uint64), ("bins_inst_tile", ctypes.c_uint64),
                ("bins_inst_entry", ctypes.c_uint64), ("bins_ranges", ctypes.c_uint64),
                ("bins_queue", ctypes.c_uint64), ("bins_bytes", ctypes.c_uint64), ("n_tiles", ctypes.c_uint32),
                ("tile_base", ctypes.c_uint32 * MAX_VIEWS)]


# exported function -> (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int32
_S = ctypes.c_size_t
_CAM = ctypes.POINTER(Camera)
_CFG = ctypes.POINTER(Config)
SIGNATURES = {
    "ges_abi_version": (ctypes.c_int32, []),
    "ges_build_flags": (ctypes.c_int32, []),
    "ges_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ges_proj_bytes": (_S, [_I, _I]),
    "ges_bins_bytes": (_S, [_I, _I, _CAM, _CFG, ctypes.c_uint64]),
    "ges_get_layout": (ctypes.c_int, [_I, _I, _CAM, _CFG, ctypes.c_uint64, ctypes.POINTER(Layout)]),
    "ges_preprocess": (ctypes.c_int, [_I, _P, _P, _P, _P, _I, _CAM, _CFG, _P, _S, _P]),
    "ges_preprocess_range": (ctypes.c_int, [_I, _I, _I, _P, _P, _P, _P, _I, _CAM, _CFG, _P, _S, _P]),
    "ges_preprocess_bwd_range": (ctypes.c_int, [_I, _I, _I, _I, _CAM, _CFG, _P, _P, _P, _P, _P, _S, _P, _P, _P, _P,
                                                _P, _P]),
    "ges_instance_count": (ctypes.c_int, [_P, _S, ctypes.POINTER(ctypes.c_uint64), _P]),
    "ges_bin": (ctypes.c_int, [_I, _I, _CAM, _CFG, _P, _S, _P, _S, _P]),
    "ges_render_fwd": (ctypes.c_int, [_I, _I, _CAM, _CFG, _P, _S, _P, _S, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ges_render_bwd_screen": (ctypes.c_int, [_I, _I, _CAM, _CFG, _P, _S, _P, _S, _P, _P, _P, _P, _P, _P, _P, _P,
                                             _P, _P, _P]),
    "ges_preprocess_bwd": (ctypes.c_int, [_I, _I, _CAM, _CFG, _P, _P, _P, _P, _P, _S, _P, _P, _P, _P, _P, _P]),
    "ges_render_bwd": (ctypes.c_int, [_I, _I, _CAM, _CFG, _P, _P, _P, _P, _P, _S, _P, _S, _P, _P, _P, _P, _P,
                                      _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ges_sync_status": (ctypes.c_int, [_P, _S, _P]),
    "ges_render_bwd_noalloc": (ctypes.c_int, [_I, _I, _CAM, _CFG, _P, _P, _P, _P, _P, _S, _P, _S, _P, _P, _P, _P,
                                              _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ges_loss_workspace_bytes": (_S, [_I, _CAM]),
    "ges_loss_rgb": (ctypes.c_int, [_I, _CAM, _P, _P, ctypes.c_float, _P, _S, _P, _P, _P]),
    "ges_knn_workspace_bytes": (_S, [_I]),
    "ges_knn": (ctypes.c_int, [_I, _P, _P, _S, _P, _P]),
    "ges_gsr_workspace_bytes": (_S, [_I, _I]),
    "ges_knn_points_workspace_bytes": (_S, [_I, _I]),
    "ges_knn_points": (ctypes.c_int, [_I, _P, _I, _P, _P, _S, _P, _P]),
    "ges_levelset_workspace_bytes": (_S, [_I, _I]),
    "ges_levelset": (ctypes.c_int, [_I, _P, _P, _P, _CFG, _I, _CAM, _P, _P, _I, _P, _I, ctypes.c_float, _P, _S, _P,
                                    _P]),
    "ges_gsr": (ctypes.c_int, [_I, _P, _P, _P, _CFG, _P, _I, _P, _P, ctypes.c_float, ctypes.c_float, _P, _S, _P,
                               _P, _P, _P, _P, _P]),
    "ges_peak_run": (ctypes.c_int, [_I, _I, _I, _P, ctypes.c_uint64, _P, ctypes.POINTER(ctypes.c_uint64)]),
}

_lock = threading.Lock()
_lib = None


def debug_variant() -> bool:
    """GES_LIB_VARIANT=debug in the environment selects the debug build (device-side bounds
    checks, see ges_build_flags) for this process."""
    return os.environ.get("GES_LIB_VARIANT", "") == "debug"


def library_path() -> str:
    return _build.lib_path(debug_variant())


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """The loaded libges.so (built in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            dbg = debug_variant()
            path = _build.build(debug=dbg) if build_if_missing else _build.lib_path(dbg)
            if not os.path.exists(path):
                raise RuntimeError(f"libges.so not found at {path}; the GES rasterizer has no CPU fallback")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().ges_status_string(int(status)).decode()
    except Exception:
        return "?"


def check(status: int, what: str) -> None:
    if status != GES_OK:
        raise GESError(status, what)
