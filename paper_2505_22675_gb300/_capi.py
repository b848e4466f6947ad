"""ctypes declarations for libbathygrid.so (include/bathygrid.h).

Loading fails loudly when the library has not been built: there is no
fallback implementation of any step.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbathygrid.so")

BG_OK = 0
BG_PENDING = 1
STATUS = {
    0: "BG_OK", 1: "BG_PENDING", -1: "BG_ERR_INVALID_ARG", -2: "BG_ERR_OOM_BUDGET",
    -3: "BG_ERR_CUDA", -4: "BG_ERR_TIMEOUT", -5: "BG_ERR_CANCELLED", -6: "BG_ERR_INTERNAL",
    -7: "BG_ERR_NOT_FOUND",
}


class BGError(RuntimeError):
    """A libbathygrid call returned an error status."""

    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")


class Variogram(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("nugget_m2", ctypes.c_float),
                ("sill_m2", ctypes.c_float), ("range_m", ctypes.c_float)]


class SoundingsInfo(ctypes.Structure):
    _fields_ = [("n_total", ctypes.c_int64), ("n_valid", ctypes.c_int64),
                ("bbox_x0_cm", ctypes.c_int32), ("bbox_y0_cm", ctypes.c_int32),
                ("bbox_x1_cm", ctypes.c_int32), ("bbox_y1_cm", ctypes.c_int32),
                ("cell_cm", ctypes.c_int32), ("ncx", ctypes.c_int32), ("ncy", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("x_cm", ctypes.c_void_p), ("y_cm", ctypes.c_void_p), ("z_m", ctypes.c_void_p),
                ("n", ctypes.c_int64),
                ("x0_cm", ctypes.c_int32), ("y0_cm", ctypes.c_int32), ("cell_cm", ctypes.c_int32),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("method", ctypes.c_int32), ("k", ctypes.c_int32), ("power", ctypes.c_float),
                ("variogram", Variogram),
                ("depth_out", ctypes.c_void_p), ("var_out", ctypes.c_void_p)]


# bg_tile has bg_request's layout; its pointers are device addresses
Tile = Request


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("nodes", ctypes.c_int64),
                ("t_submit_us", ctypes.c_double), ("t_start_us", ctypes.c_double),
                ("t_done_us", ctypes.c_double)]


_lib = None

P = ctypes.c_void_p
PP = ctypes.POINTER(ctypes.c_void_p)

_SIGNATURES = {
    "bg_version": ([], ctypes.c_char_p),
    "bg_last_error": ([], ctypes.c_char_p),
    "bg_status_str": ([ctypes.c_int], ctypes.c_char_p),
    "bg_launch_count": ([ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "bg_alu_peak": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                     ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "bg_profile_enable": ([P, ctypes.c_int], ctypes.c_int),
    "bg_profile_read": ([P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                         ctypes.POINTER(ctypes.c_int64), ctypes.c_int], ctypes.c_int),
    "bg_ctx_create": ([ctypes.c_int, ctypes.c_size_t, PP], ctypes.c_int),
    "bg_ctx_destroy": ([P], ctypes.c_int),
    "bg_ctx_device_bytes": ([P, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "bg_grid_create": ([P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                        ctypes.c_int32, PP], ctypes.c_int),
    "bg_grid_destroy": ([P], ctypes.c_int),
    "bg_soundings_upload": ([P, P, P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_int32, P, PP],
                            ctypes.c_int),
    "bg_soundings_info_get": ([P, ctypes.POINTER(SoundingsInfo)], ctypes.c_int),
    "bg_soundings_destroy": ([P], ctypes.c_int),
    "bg_interp_idw": ([P, P, ctypes.c_int, ctypes.c_float, P, P, P], ctypes.c_int),
    "bg_interp_okrige": ([P, P, ctypes.c_int, ctypes.POINTER(Variogram), P, P, P, P],
                         ctypes.c_int),
    "bg_interp_idw_okrige": ([P, P, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                              ctypes.POINTER(Variogram), P, P, P, P], ctypes.c_int),
    "bg_interp_idw_okrige_host": ([P, P, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                   ctypes.POINTER(Variogram), P, P, P, P, P, P, P], ctypes.c_int),
    "bg_interp_idw_points": ([P, P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_float, P, P, P],
                             ctypes.c_int),
    "bg_interp_okrige_points": ([P, P, P, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(Variogram),
                                 P, P, P, P], ctypes.c_int),
    "bg_resample_points": ([P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                            ctypes.c_int32, ctypes.c_int, P, P, ctypes.c_int64, P, P, P],
                           ctypes.c_int),
    "bg_resample_grid": ([P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                          ctypes.c_int32, ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                          ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P], ctypes.c_int),
    "bg_submit": ([P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "bg_poll": ([P, ctypes.c_uint64, ctypes.POINTER(Result)], ctypes.c_int),
    "bg_wait": ([P, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(Result)], ctypes.c_int),
    "bg_cancel": ([P, ctypes.c_uint64], ctypes.c_int),
    "bg_serve_stats": ([P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                        ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "bg_serve_shutdown": ([P], ctypes.c_int),
    "bg_batch_create": ([P, ctypes.POINTER(Request), ctypes.c_int, PP], ctypes.c_int),
    "bg_batch_run": ([P, P], ctypes.c_int),
    "bg_batch_set_cell_target": ([P, ctypes.c_float], ctypes.c_int),
    "bg_batch_tune": ([P, P, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "bg_batch_set_shape": ([P, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "bg_batch_get_config": ([P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "bg_batch_status": ([P, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "bg_batch_destroy": ([P], ctypes.c_int),
    "bg_interp_idw_noalloc": ([P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                               ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int,
                               ctypes.c_float, P, P, P], ctypes.c_int),
}


def load():
    """Load libbathygrid.so (built by paper_2505_22675_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()'); "
            "there is no fallback path")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def optional(name, args, res):
    """Declare an entry point that newer builds export; returns None if absent."""
    lib = load()
    try:
        fn = getattr(lib, name)
    except AttributeError:
        return None
    fn.argtypes = args
    fn.restype = res
    return fn


def check(status: int, where: str) -> int:
    if status < 0:
        detail = load().bg_last_error().decode(errors="replace")
        raise BGError(status, where, detail)
    return status
