"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

Holds no dedispersion arithmetic: it draws noise (counter-based splitmix64 +
Box-Muller, see ``synth.c``), adds boxcar pulses along per-channel start
samples that the caller computes, lays out the channel centre frequencies of
an evenly channelised band and draws Poisson arrival times for the streaming
workload.  The workloads mirror the paper's synthetic filterbanks (SIGPROC
``fake`` data, Sec. 5): 8/16-bit integer samples or float32, channel-major.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None

_KIND = {np.dtype(np.uint8): 1, np.dtype(np.uint16): 2, np.dtype(np.float32): 3}
_LIMITS = {1: (0.0, 255.0), 2: (0.0, 65535.0), 3: (0.0, 0.0)}


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_SRC) > os.path.getmtime(_LIB):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                        "-ffp-contract=off", "-Wall", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.synth_splitmix64.restype = ctypes.c_uint64
            lib.synth_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.synth_normal.restype = ctypes.c_double
            lib.synth_fill.argtypes = [
                ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p,
                ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_fill.restype = ctypes.c_int
            _lib = lib
    return _lib


def splitmix64(seed: int, n: int) -> int:
    """Output number ``n`` (n >= 1) of a splitmix64 stream seeded with ``seed``."""
    return int(_load().synth_splitmix64(seed & (2**64 - 1), n & (2**64 - 1)))


def normal(seed: int, i: int) -> float:
    """Normal variate number ``i`` of stream ``seed`` (Box-Muller pair i // 2)."""
    return float(_load().synth_normal(seed & (2**64 - 1), i))


def channel_freqs(f_high_mhz: float, bandwidth_mhz: float, n_chan: int) -> np.ndarray:
    """Channel centres of a band [f_high - bw, f_high] split into equal channels.

    Channel 0 is the highest: f_c = f_high - (c + 1/2) * bw / n_chan.
    """
    c = np.arange(n_chan, dtype=np.float64)
    return f_high_mhz - (c + 0.5) * (bandwidth_mhz / n_chan)


def filterbank(dtype, n_chan: int, n_samp: int, seed: int, mean: float, sd: float,
               pulses=(), out: np.ndarray | None = None, row_stride: int | None = None):
    """Channel-major [n_chan][n_samp] noise plus boxcar pulses.

    ``pulses`` is a sequence of ``(starts, width, amplitude)`` where ``starts``
    holds one start sample per channel.  ``out`` may be a (pinned) buffer of
    shape [n_chan][row_stride] to fill in place.
    """
    dt = np.dtype(dtype)
    kind = _KIND[dt]
    stride = n_samp if row_stride is None else int(row_stride)
    if out is None:
        out = np.empty((n_chan, stride), dtype=dt)
    if out.dtype != dt or out.shape[0] != n_chan or out.shape[1] < stride \
            or not out.flags["C_CONTIGUOUS"]:
        raise ValueError("out must be C-contiguous [n_chan][row_stride] of the dtype")
    n_p = len(pulses)
    starts = np.zeros((max(n_p, 1), n_chan), dtype=np.int64)
    widths = np.zeros(max(n_p, 1), dtype=np.int64)
    amps = np.zeros(max(n_p, 1), dtype=np.float64)
    for k, (s, w, a) in enumerate(pulses):
        starts[k] = np.asarray(s, dtype=np.int64)
        widths[k] = int(w)
        amps[k] = float(a)
    lo, hi = _LIMITS[kind]
    rc = _load().synth_fill(kind, out.ctypes.data, n_chan, n_samp, stride, seed & (2**64 - 1),
                            float(mean), float(sd), lo, hi, n_p, starts.ctypes.data,
                            widths.ctypes.data, amps.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"synth_fill failed ({rc})")
    return out


def poisson_arrivals(seed: int, rate_hz: float, n: int, t0: float = 0.0) -> np.ndarray:
    """``n`` arrival times of a Poisson process of the given rate, from ``t0``."""
    rng = np.random.default_rng(seed)
    return t0 + np.cumsum(rng.exponential(1.0 / rate_hz, size=n))


def pick_pulses(seed: int, n_pulses: int, n_dm: int, n_out: int, w_lo: int = 1,
                w_hi: int = 32):
    """Random (dm_index, t0, width) triples for injected pulses.

    t0 is uniform in [0, n_out - 64), widths uniform in [w_lo, w_hi].
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_pulses):
        d = int(rng.integers(0, n_dm))
        t0 = int(rng.integers(0, max(n_out - 64, 1)))
        w = int(rng.integers(w_lo, w_hi + 1))
        out.append((d, t0, w))
    return out


def pack4(x: np.ndarray) -> np.ndarray:
    """Pack 4-bit samples (uint8 values 0..15, [n_chan][n], n even) two per
    byte: sample 2k in the low nibble of byte k, 2k + 1 in the high nibble."""
    if x.shape[1] % 2:
        raise ValueError("pack4 needs an even number of samples per row")
    lo = x[:, 0::2].astype(np.uint8) & 0x0F
    hi = x[:, 1::2].astype(np.uint8) & 0x0F
    return np.ascontiguousarray(lo | (hi << 4))


def filterbank4(n_chan: int, n_samp: int, seed: int, mean: float, sd: float, pulses=(),
                row_bytes: int | None = None) -> np.ndarray:
    """Packed 4-bit filterbank: the uint8 generator's samples clamped to 0..15,
    packed by pack4 into [n_chan][row_bytes] bytes (row_bytes >= n_samp / 2)."""
    n_even = n_samp + (n_samp % 2)
    x = filterbank(np.uint8, n_chan, n_even, seed, mean, sd, pulses=pulses)
    x = np.minimum(x, 15).astype(np.uint8)
    packed = pack4(x)
    if row_bytes is not None and row_bytes != packed.shape[1]:
        out = np.zeros((n_chan, row_bytes), np.uint8)
        out[:, : packed.shape[1]] = packed
        packed = out
    return packed
