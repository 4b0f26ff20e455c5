"""Tiled CPU dedispersion (the paper's CPU scheme, Algorithm 2): a labelled CPU
baseline for bench.py beside the plain oracle.  Not part of the GPU library
(which never falls back to the host) and not the parity authority."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_cpu_tiled.c")
_LIB = os.path.join(_HERE, "_build", "libdd_cpu_tiled.so")
_lock = threading.Lock()
_lib = None
_DTYPE = {np.dtype(np.uint8): 1, np.dtype(np.uint16): 2, np.dtype(np.float32): 3}


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_SRC) > os.path.getmtime(_LIB):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.dd_cpu_tiled.restype = ctypes.c_int
            lib.dd_cpu_tiled.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_int64, ctypes.c_void_p]
            _lib = lib
    return _lib


def forward(x: np.ndarray, shifts: np.ndarray, n_out: int) -> np.ndarray:
    """Y [n_dm][n_out] of one bin-1 range from int32 shifts [n_dm][n_chan]."""
    if x.dtype not in _DTYPE or x.strides[1] != x.itemsize:
        raise ValueError("x must be uint8/uint16/float32 [n_chan][stride], time contiguous")
    shifts = np.ascontiguousarray(shifts, dtype=np.int32)
    n_dm, n_chan = shifts.shape
    if x.shape[0] != n_chan or n_out + int(shifts.max()) > x.shape[1]:
        raise ValueError("input too short for the shifts")
    out = np.empty((n_dm, n_out), np.float32 if x.dtype == np.float32 else np.int32)
    stride = x.strides[0] // x.itemsize if n_chan > 1 else x.shape[1]
    rc = _load().dd_cpu_tiled(_DTYPE[x.dtype], x.ctypes.data, n_chan, stride, shifts.ctypes.data,
                              n_dm, int(n_out), out.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"dd_cpu_tiled failed ({rc})")
    return out
