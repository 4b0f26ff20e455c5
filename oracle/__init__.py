"""Plain CPU oracle for brute-force incoherent dedispersion (ctypes binding).

TEST INFRASTRUCTURE ONLY: the parity authority for the CUDA library.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
and never imports it.

The C source (``dd_oracle.c``) writes out the paper's definitions:
Eq. 1 (delay law), Eq. 3 / Algorithm 1 (direct transform, Sec. 2), the
per-range time binning of Sec. 5.3 and the transpose of the resulting linear
map.  This module only marshals numpy arrays into it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_HDR = os.path.join(_HERE, "dd_oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

DTYPE_U8, DTYPE_U16, DTYPE_F32, DTYPE_U4 = 1, 2, 3, 4
_NP_DTYPE = {np.dtype(np.uint8): DTYPE_U8, np.dtype(np.uint16): DTYPE_U16,
             np.dtype(np.float32): DTYPE_F32}


class Packed4:
    """4-bit samples packed two per byte: sample 2k of a row in the low nibble
    of byte k, sample 2k + 1 in the high nibble.  data is uint8
    [n_chan][row_bytes] (time contiguous); each row holds n_samp samples."""

    def __init__(self, data: np.ndarray, n_samp: int):
        if data.dtype != np.uint8 or data.ndim != 2 or data.strides[1] != 1:
            raise ValueError("packed 4-bit data must be uint8 [n_chan][row_bytes]")
        if n_samp > 2 * data.shape[1]:
            raise ValueError("n_samp exceeds the packed row")
        self.data = data
        self.shape = (data.shape[0], int(n_samp))

    @property
    def ctypes(self):
        return self.data.ctypes

_lock = threading.Lock()
_lib = None


class Range(ctypes.Structure):
    """One DM range: half-open [dm_lo, dm_hi) with a fixed step and a time bin."""

    _fields_ = [("dm_lo", ctypes.c_double), ("dm_hi", ctypes.c_double),
                ("dm_step", ctypes.c_double), ("bin", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (FP64 as written: no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            c_int64_p = ctypes.POINTER(ctypes.c_int64)
            c_double_p = ctypes.POINTER(ctypes.c_double)
            lib.oracle_c_dm.restype = ctypes.c_double
            lib.oracle_range_ndm.argtypes = [Range]
            lib.oracle_range_ndm.restype = ctypes.c_int64
            lib.oracle_range_dm.argtypes = [Range, ctypes.c_int64]
            lib.oracle_range_dm.restype = ctypes.c_double
            lib.oracle_delay_coeff.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.oracle_delay_coeff.restype = ctypes.c_double
            lib.oracle_shift.argtypes = [ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int32, ctypes.c_double]
            lib.oracle_shift.restype = ctypes.c_int64
            lib.oracle_shift_table.argtypes = [c_double_p, ctypes.c_int32, ctypes.c_double,
                                               ctypes.c_double, Range, c_int64_p]
            lib.oracle_range_extent.argtypes = [c_double_p, ctypes.c_int32, ctypes.c_double,
                                                ctypes.c_double, Range, ctypes.c_int64,
                                                c_int64_p, c_int64_p]
            lib.oracle_forward_rows.argtypes = [
                ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                ctypes.c_int64, c_double_p, ctypes.c_double, ctypes.c_double, Range,
                c_int64_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                c_double_p]
            lib.oracle_forward.argtypes = [
                ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                ctypes.c_int64, c_double_p, ctypes.c_double, ctypes.c_double,
                ctypes.POINTER(Range), ctypes.c_int32, ctypes.c_int, c_double_p]
            lib.oracle_adjoint.argtypes = [
                c_double_p, ctypes.c_int32, ctypes.c_int64, c_double_p, ctypes.c_double,
                ctypes.c_double, ctypes.POINTER(Range), ctypes.c_int32, c_double_p]
            lib.oracle_adjoint_channels.argtypes = [
                c_double_p, ctypes.c_int32, ctypes.c_int64, c_double_p, ctypes.c_double,
                ctypes.c_double, ctypes.POINTER(Range), ctypes.c_int32,
                ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, c_double_p]
            lib.oracle_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _range(r) -> Range:
    if isinstance(r, Range):
        return r
    lo, hi, step, b = r
    return Range(float(lo), float(hi), float(step), int(b))


def c_dm() -> float:
    return _load().oracle_c_dm()


def n_dm(r) -> int:
    return int(_load().oracle_range_ndm(_range(r)))


def dm_value(r, d: int) -> float:
    return float(_load().oracle_range_dm(_range(r), int(d)))


def delay_coeff(f_mhz: float, f_ref_mhz: float) -> float:
    return float(_load().oracle_delay_coeff(float(f_mhz), float(f_ref_mhz)))


def shift(dm: float, k_c: float, b: int, t_samp: float) -> int:
    return int(_load().oracle_shift(float(dm), float(k_c), int(b), float(t_samp)))


def shift_table(freqs, f_ref: float, t_samp: float, r) -> np.ndarray:
    """int64 [n_dm][n_chan] shift table of one range."""
    f = _f64(freqs)
    rr = _range(r)
    out = np.zeros((n_dm(rr), f.size), dtype=np.int64)
    rc = _load().oracle_shift_table(_dp(f), f.size, float(f_ref), float(t_samp), rr, _ip(out))
    if rc != 0:
        raise ValueError(f"oracle_shift_table failed ({rc})")
    return out


def extent(freqs, f_ref: float, t_samp: float, r, n_samp: int):
    """(S_max, N_out) of one range for n_samp raw samples."""
    f = _f64(freqs)
    smax = np.zeros(1, np.int64)
    nout = np.zeros(1, np.int64)
    rc = _load().oracle_range_extent(_dp(f), f.size, float(f_ref), float(t_samp), _range(r),
                                     int(n_samp), _ip(smax), _ip(nout))
    if rc != 0:
        raise ValueError(f"oracle_range_extent failed ({rc})")
    return int(smax[0]), int(nout[0])


def _input(x):
    if isinstance(x, Packed4):
        d = x.data
        row_bytes = d.strides[0] if d.shape[0] > 1 else d.shape[1]
        return DTYPE_U4, 2 * row_bytes
    if x.ndim != 2:
        raise ValueError("x must be [n_chan][n_samp]")
    if x.dtype not in _NP_DTYPE:
        raise ValueError(f"unsupported dtype {x.dtype}")
    if x.strides[1] != x.itemsize:
        raise ValueError("time axis must be contiguous")
    stride = x.strides[0] // x.itemsize if x.shape[0] > 1 else x.shape[1]
    return _NP_DTYPE[x.dtype], stride


def forward_rows(x: np.ndarray, freqs, f_ref: float, t_samp: float, r, rows,
                 t_begin: int = 0, t_end: int | None = None, take_abs: bool = False):
    """FP64 [len(rows)][t_end - t_begin] outputs of one range (Eq. 3)."""
    dt, stride = _input(x)
    f = _f64(freqs)
    rr = _range(r)
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    if t_end is None:
        t_end = extent(f, f_ref, t_samp, rr, x.shape[1])[1]
    out = np.zeros((rows.size, max(t_end - t_begin, 0)), dtype=np.float64)
    rc = _load().oracle_forward_rows(dt, x.ctypes.data, f.size, x.shape[1], stride, _dp(f),
                                     float(f_ref), float(t_samp), rr, _ip(rows), rows.size,
                                     int(t_begin), int(t_end), int(take_abs), _dp(out))
    if rc != 0:
        raise ValueError(f"oracle_forward_rows failed ({rc})")
    return out


def forward(x: np.ndarray, freqs, f_ref: float, t_samp: float, ranges,
            take_abs: bool = False):
    """List of FP64 [n_dm_r][N_out_r] planes, one per range (Eq. 3 per range)."""
    dt, stride = _input(x)
    f = _f64(freqs)
    rs = [_range(r) for r in ranges]
    shapes = []
    for rr in rs:
        shapes.append((n_dm(rr), extent(f, f_ref, t_samp, rr, x.shape[1])[1]))
    if any(s[1] <= 0 for s in shapes):
        raise ValueError("input too short for the plan")
    total = sum(a * b for a, b in shapes)
    out = np.zeros(total, dtype=np.float64)
    arr = (Range * len(rs))(*rs)
    rc = _load().oracle_forward(dt, x.ctypes.data, f.size, x.shape[1], stride, _dp(f),
                                float(f_ref), float(t_samp), arr, len(rs), int(take_abs),
                                _dp(out))
    if rc != 0:
        raise ValueError(f"oracle_forward failed ({rc})")
    planes, off = [], 0
    for a, b in shapes:
        planes.append(out[off:off + a * b].reshape(a, b))
        off += a * b
    return planes


def adjoint(ybar_planes, n_chan: int, n_samp: int, freqs, f_ref: float, t_samp: float,
            ranges) -> np.ndarray:
    """FP64 [n_chan][n_samp] transpose applied to the per-range cotangent planes."""
    f = _f64(freqs)
    rs = [_range(r) for r in ranges]
    flat = np.ascontiguousarray(np.concatenate([_f64(p).ravel() for p in ybar_planes]))
    out = np.zeros((n_chan, n_samp), dtype=np.float64)
    arr = (Range * len(rs))(*rs)
    rc = _load().oracle_adjoint(_dp(flat), int(n_chan), int(n_samp), _dp(f), float(f_ref),
                                float(t_samp), arr, len(rs), _dp(out))
    if rc != 0:
        raise ValueError(f"oracle_adjoint failed ({rc})")
    return out


def adjoint_channels(ybar_planes, n_chan: int, n_samp: int, freqs, f_ref: float, t_samp: float,
                     ranges, chans) -> np.ndarray:
    """FP64 [len(chans)][n_samp]: the transpose's rows for the listed channels."""
    f = _f64(freqs)
    rs = [_range(r) for r in ranges]
    flat = np.ascontiguousarray(np.concatenate([_f64(p).ravel() for p in ybar_planes]))
    ch = np.ascontiguousarray(np.asarray(chans, dtype=np.int32))
    out = np.zeros((ch.size, n_samp), dtype=np.float64)
    arr = (Range * len(rs))(*rs)
    rc = _load().oracle_adjoint_channels(_dp(flat), int(n_chan), int(n_samp), _dp(f),
                                         float(f_ref), float(t_samp), arr, len(rs),
                                         ch.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                         ch.size, _dp(out))
    if rc != 0:
        raise ValueError(f"oracle_adjoint_channels failed ({rc})")
    return out


def transpose(x_tm: np.ndarray) -> np.ndarray:
    """Front end of the paper's pipeline (Sec. 5.4): time-major samples
    x_tm[t][c] to channel-major rows x[c][t], the order Eq. 3 sums along.
    The definition written out: element (c, t) of the result is x_tm[t, c]."""
    n_samp, n_chan = x_tm.shape
    out = np.empty((n_chan, n_samp), dtype=x_tm.dtype)
    for c in range(n_chan):
        out[c, :] = x_tm[:, c]
    return out


def threads() -> int:
    return int(_load().oracle_threads())
