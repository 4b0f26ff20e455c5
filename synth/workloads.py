"""Synthetic workloads shaped like the paper's telescopes and test plans.

Each workload is a plain description (band, sampling, DM plan, noise and
pulse recipe).  ``make_input`` draws its filterbank with ``synth.filterbank``;
pulse tracks need the per-channel shifts of the method, which the caller
supplies through ``shift_rows(range_index, dm_index) -> int array [n_chan]``
(the oracle in tests, the library's planner in the benchmark), so this module
holds none of the dedispersion arithmetic.

Recipes (seed = workload index * 1000 + beam index):
  tiny_u8      64 ch x 8192, 1500 MHz top, 300 MHz band, 64 us, DMs 0..63.5/0.5,
               N(128, 16) clipped to [0, 255], one boxcar (w=4, +40) at DM 30.
  paper_u8     8192 ch x 262144, 1670 MHz top, 320 MHz band, 64 us,
               DMs 0..409.5/0.1 (4096 trials), same noise, 3 pulses at random
               DMs, widths 1-32 (the 8-bit, 8192-channel case of Sec. 5.2).
  paper_u16    as paper_u8 with N(32768, 256) and +640 pulses (same S/N).
  batched      24 x u8 (1024 ch, 1210-1520 MHz, 64 us, 131072, 2048 DMs/0.1),
               8 x u16 (4096 ch, 1350-1670 MHz, 54.6 us, 65536, 3072 DMs/0.2),
               4 x f32 (336 ch, 300-400 MHz, 327.68 us, 32768, 1024 DMs/0.2).
  diff_f32     1024 ch, 1200-1500 MHz, 128 us, 65536, DMs 0..204.6/0.2, N(0, 1).
  stream_u8    64 beams u8 4096 ch, 1670 MHz top, 320 MHz band, 64 us, chunks of
               65536 + max-delay overlap; ranges 0-150/0.1 bin 1, 150-300/0.2
               bin 2, 300-1000/0.5 bin 4, 1000-2000/1.0 bin 8.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import channel_freqs, filterbank, pick_pulses


@dataclass
class Beam:
    name: str
    dtype: str                 # "u8", "u16", "f32"
    n_chan: int
    n_samp: int
    f_high: float              # MHz, top band edge (= reference frequency)
    bandwidth: float           # MHz
    t_samp: float              # s
    ranges: list               # [(lo, hi, step, bin)]
    mean: float
    sd: float
    seed: int
    pulse_amp: float
    pulses: list = field(default_factory=list)  # [(range, dm_index, t0, width)]
    n_random_pulses: int = 0

    @property
    def freqs(self) -> np.ndarray:
        return channel_freqs(self.f_high, self.bandwidth, self.n_chan)

    @property
    def np_dtype(self):
        """Element type of the sample buffer (packed bytes for "u4")."""
        return {"u8": np.uint8, "u16": np.uint16, "f32": np.float32, "u4": np.uint8}[self.dtype]


def tiny_u8() -> Beam:
    return Beam("tiny_u8", "u8", 64, 8192, 1500.0, 300.0, 64e-6, [(0.0, 64.0, 0.5, 1)],
                128.0, 16.0, 1000, 40.0, pulses=[(0, 60, 3000, 4)])


def paper_u8() -> Beam:
    return Beam("paper_u8", "u8", 8192, 262144, 1670.0, 320.0, 64e-6,
                [(0.0, 409.6, 0.1, 1)], 128.0, 16.0, 2000, 40.0, n_random_pulses=3)


def paper_u4() -> Beam:
    """The paper-scale plan on 4-bit samples (N(8, 2) clamped to 0..15)."""
    return Beam("paper_u4", "u4", 8192, 262144, 1670.0, 320.0, 64e-6,
                [(0.0, 409.6, 0.1, 1)], 8.0, 2.0, 2002, 5.0, n_random_pulses=3)


def paper_u16() -> Beam:
    return Beam("paper_u16", "u16", 8192, 262144, 1670.0, 320.0, 64e-6,
                [(0.0, 409.6, 0.1, 1)], 32768.0, 256.0, 2001, 640.0, n_random_pulses=3)


def batched() -> list:
    beams = []
    for i in range(24):
        beams.append(Beam(f"batched_u8_{i}", "u8", 1024, 131072, 1520.0, 310.0, 64e-6,
                          [(0.0, 204.8, 0.1, 1)], 128.0, 16.0, 3000 + i, 40.0,
                          n_random_pulses=1))
    for i in range(8):
        beams.append(Beam(f"batched_u16_{i}", "u16", 4096, 65536, 1670.0, 320.0, 54.6e-6,
                          [(0.0, 614.4, 0.2, 1)], 32768.0, 256.0, 3024 + i, 640.0,
                          n_random_pulses=1))
    for i in range(4):
        beams.append(Beam(f"batched_f32_{i}", "f32", 336, 32768, 400.0, 100.0, 327.68e-6,
                          [(0.0, 204.8, 0.2, 1)], 0.0, 1.0, 3032 + i, 2.5,
                          n_random_pulses=1))
    return beams


def diff_f32() -> Beam:
    return Beam("diff_f32", "f32", 1024, 65536, 1500.0, 300.0, 128e-6,
                [(0.0, 204.8, 0.2, 1)], 0.0, 1.0, 4000, 2.5)


STREAM_RANGES = [(0.0, 150.0, 0.1, 1), (150.0, 300.0, 0.2, 2), (300.0, 1000.0, 0.5, 4),
                 (1000.0, 2000.0, 1.0, 8)]


def stream_beam(i: int, n_samp: int) -> Beam:
    return Beam(f"stream_u8_{i}", "u8", 4096, n_samp, 1670.0, 320.0, 64e-6,
                list(STREAM_RANGES), 128.0, 16.0, 5000 + i, 40.0, n_random_pulses=1)


def resolve_pulses(beam: Beam, n_dm, n_out) -> list:
    """Fixed plus seeded random pulses as (range, dm_index, t0, width)."""
    out = list(beam.pulses)
    if beam.n_random_pulses:
        for d, t0, w in pick_pulses(beam.seed + 7919, beam.n_random_pulses, n_dm[0], n_out[0]):
            out.append((0, d, t0, w))
    return out


def make_input(beam: Beam, shift_rows, n_dm, n_out, out=None, row_stride=None):
    """Draw the beam's filterbank.  shift_rows(r, d) gives decimated shifts [n_chan].

    A pulse at decimated sample t0 of range r (bin b) covers raw samples
    [(t0 + s) * b, (t0 + s) * b + w * b) in each channel, so that it lands on
    output sample t0 of trial d with width w.
    """
    tracks = []
    for r, d, t0, w in resolve_pulses(beam, n_dm, n_out):
        b = beam.ranges[r][3]
        s = np.asarray(shift_rows(r, d), dtype=np.int64)
        tracks.append(((t0 + s) * b, w * b, beam.pulse_amp))
    if beam.dtype == "u4":  # 4-bit: 8-bit draws clamped to 0..15, packed two per byte
        from . import pack4
        n_even = beam.n_samp + (beam.n_samp % 2)
        x = filterbank(np.uint8, beam.n_chan, n_even, beam.seed, beam.mean, beam.sd,
                       pulses=tracks)
        packed = pack4(np.minimum(x, 15).astype(np.uint8))
        stride = n_even if row_stride is None else int(row_stride)
        res = np.zeros((beam.n_chan, stride // 2), np.uint8) if out is None else out
        res[:, : packed.shape[1]] = packed
        return res
    return filterbank(beam.np_dtype, beam.n_chan, beam.n_samp, beam.seed, beam.mean, beam.sd,
                      pulses=tracks, out=out, row_stride=row_stride)
