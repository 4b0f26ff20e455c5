"""ctypes declarations of the libdd C ABI (include/dd.h, include/dd_bench.h).

Argument marshalling only; the library is built in-tree by ``build.py`` and
loading fails loudly if it is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import builder as _build

_lock = threading.Lock()
_lib = None

DD_OK, DD_ERR_INVALID_ARG, DD_ERR_UNSUPPORTED, DD_ERR_SHAPE = 0, 1, 2, 3
DD_ERR_BUDGET, DD_ERR_CUDA, DD_ERR_TIMEOUT = 4, 5, 6
DD_U8, DD_U16, DD_F32, DD_U4 = 1, 2, 3, 4
DD_MAX_RANGES = 16
DD_KERNEL_GENERIC, DD_KERNEL_TILED = 1, 2
DD_TILE_PATTERN = 0x104
DD_TILE_PACKED = 0x106
DD_ADJOINT_GATHER, DD_ADJOINT_PATTERN = 1, 2


class DDError(RuntimeError):
    """A libdd call returned a non-OK status."""

    def __init__(self, status: int, detail: str):
        self.status = status
        self.detail = detail
        super().__init__(f"{status_name(status)}: {detail}")


class Range(ctypes.Structure):
    _fields_ = [("dm_lo", ctypes.c_double), ("dm_hi", ctypes.c_double),
                ("dm_step", ctypes.c_double), ("bin", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_chan", ctypes.c_int32), ("n_ranges", ctypes.c_int32),
                ("dtype", ctypes.c_int), ("n_samp", ctypes.c_int64),
                ("n_dm_total", ctypes.c_int64),
                ("n_dm", ctypes.c_int64 * DD_MAX_RANGES),
                ("s_max", ctypes.c_int64 * DD_MAX_RANGES),
                ("n_out", ctypes.c_int64 * DD_MAX_RANGES),
                ("out_offset", ctypes.c_int64 * DD_MAX_RANGES),
                ("out_elems", ctypes.c_int64), ("max_delay_raw", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_size_t),
                ("kernel", ctypes.c_int32 * DD_MAX_RANGES),
                ("tile_dms", ctypes.c_int32 * DD_MAX_RANGES),
                ("adjoint_kernel", ctypes.c_int32),
                ("tile_shape", ctypes.c_int32 * DD_MAX_RANGES),
                ("packed_copy", ctypes.c_int32 * DD_MAX_RANGES)]


class TileShape(ctypes.Structure):
    _fields_ = [("words_per_lane", ctypes.c_int32), ("dms_per_lane", ctypes.c_int32),
                ("warps", ctypes.c_int32), ("channels_per_stage", ctypes.c_int32),
                ("channel_pairs", ctypes.c_int32), ("float_pairs", ctypes.c_int32),
                ("automatic", ctypes.c_int32)]


# name -> (restype, argtypes) for every exported entry point.
_VP = ctypes.c_void_p
_I32, _I64, _SZ, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
SIGNATURES = {
    "dd_plan_create": (ctypes.c_int, [ctypes.POINTER(_D), _I32, _D, _D, ctypes.POINTER(Range),
                                      _I32, ctypes.c_int, ctypes.POINTER(_VP)]),
    "dd_plan_destroy": (ctypes.c_int, [_VP]),
    "dd_plan_query": (ctypes.c_int, [_VP, _I64, ctypes.POINTER(PlanInfo)]),
    "dd_plan_shifts": (ctypes.c_int, [_VP, _I32, _VP]),
    "dd_plan_upload": (ctypes.c_int, [_VP, _VP, _SZ, _VP]),
    "dd_plan_set_tile": (ctypes.c_int, [_VP, _I32, _I32]),
    "dd_run": (ctypes.c_int, [_VP, _VP, _I64, _I64, _VP, _VP]),
    "dd_run_adjoint": (ctypes.c_int, [_VP, _VP, _VP, _I64, _I64, _VP]),
    "dd_run_scratch": (ctypes.c_int, [_VP, _VP, _I64, _I64, _VP, _VP, _SZ, _VP]),
    "dd_run_host_scratch": (ctypes.c_int, [_VP, _VP, _I64, _I64, _VP, _VP, _VP, _VP, _SZ, _VP]),
    "dd_plan_input_scratch_bytes": (ctypes.c_int, [_VP, _I64, ctypes.POINTER(_SZ)]),
    "dd_plan_packed_scratch_bytes": (ctypes.c_int, [_VP, _I64, _I32, ctypes.POINTER(_SZ)]),
    "dd_run_adjoint_scratch": (ctypes.c_int, [_VP, _VP, _VP, _I64, _I64, _VP, _SZ, _VP]),
    "dd_adjoint_scratch_bytes": (ctypes.c_int, [_VP, _I64, ctypes.POINTER(_SZ)]),
    "dd_plan_device_status": (ctypes.c_int, [_VP, _VP]),
    "dd_run_u8_noalloc": (ctypes.c_int, [_VP, _VP, _I64, _I64, _VP, _VP]),
    "dd_run_u8_noalloc_status": (ctypes.c_int, [_VP]),
    "dd_run_window": (ctypes.c_int, [_VP, _VP, _I64, _I64, ctypes.POINTER(_I64), _VP, _VP, _SZ,
                                     _VP]),
    "dd_plan_set_wait_limit": (ctypes.c_int, [_VP, _I32, _I32]),
    "dd_tile_shapes": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_I32)]),
    "dd_plan_set_tile_shape": (ctypes.c_int, [_VP, _I32, _I32, _I32]),
    "dd_pack_input": (ctypes.c_int, [_VP, _VP, _I64, _I64, _VP, _SZ, _VP]),
    "dd_run_packed": (ctypes.c_int, [_VP, _VP, _I64, _I64, _VP, _VP, _SZ, _VP]),
    "dd_run_host": (ctypes.c_int, [_VP, _VP, _I64, _I64, _VP, _VP, _VP, _VP]),
    "dd_run_host_tmajor": (ctypes.c_int, [_VP, _VP, _I64, _I64, _VP, _VP, _VP, _I64, _VP, _VP]),
    "dd_transpose": (ctypes.c_int, [ctypes.c_int, _VP, _I64, _I32, _VP, _I64, _I64, _I64, _VP]),
    "dd_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(_I64), _I32,
                                       ctypes.POINTER(_VP)]),
    "dd_batch_destroy": (ctypes.c_int, [_VP]),
    "dd_batch_workspace_bytes": (ctypes.c_int, [_VP, ctypes.POINTER(_SZ)]),
    "dd_plan_dm_ranges": (ctypes.c_int, [_VP, _I32, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, _I32, _I32, _VP,
                                          ctypes.POINTER(_I32)]),
    "dd_batch_info": (ctypes.c_int, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I32)]),
    "dd_batch_launches": (ctypes.c_int, [_VP, ctypes.POINTER(_I32)]),
    "dd_batch_upload": (ctypes.c_int, [_VP, _VP, _SZ, _VP]),
    "dd_batch_bind": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_I64),
                                     ctypes.POINTER(_VP), _VP]),
    "dd_batch_run": (ctypes.c_int, [_VP, _VP]),
    "dd_batch_plan_scratch_bytes": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_SZ)]),
    "dd_batch_bind_scratch": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_I64),
                                             ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                             ctypes.POINTER(_SZ), _VP]),
    "dd_batch_status": (ctypes.c_int, [_VP, _VP]),
    "dd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "dd_last_error_detail": (ctypes.c_char_p, []),
    "dd_version": (ctypes.c_char_p, []),
    "dd_bench_launch": (ctypes.c_int, [_I32, _I32, _I32, _I64, _VP, _VP,
                                       ctypes.POINTER(_D)]),
    "dd_bench_device": (ctypes.c_int, [ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
}


def lib_path() -> str:
    return _build.LIB


def load(auto_build: bool = True):
    """Load libdd.so (building it first if asked and it is stale or missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if auto_build else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libdd.so is missing at {path}; run build() first")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_name(status: int) -> str:
    return load().dd_status_string(status).decode()


def check(status: int):
    if status != DD_OK:
        raise DDError(status, load().dd_last_error_detail().decode())
