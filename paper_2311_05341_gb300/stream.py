"""Streaming dedispersion server: continuous batching of many beams on one GPU.

Each admitted beam keeps a device window of `overlap + chunk` raw samples per
channel.  A new chunk is copied into the window behind the overlap (the last
`overlap` samples of the previous step, kept on the device), the window is
dedispersed with dd_run, and the window's tail becomes the next overlap.  With
overlap >= max_r bin_r * S_max_r every step emits the next `chunk / bin_r`
output samples of every DM range, equal to the same samples of a one-shot
transform of the concatenated stream (the paper's real-time processing,
Sec. 5.4, done incrementally).

Serving is continuous batching: each beam has its own CUDA stream, chunks are
launched as soon as they arrive, so work of different beams overlaps on the
device; beams are admitted while their device memory (window, output planes)
fits an HBM budget and wait otherwise until another beam leaves.  Latency is
measured from a chunk's arrival to its outputs being ready on the device.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import Plan


def _torch():
    import torch
    return torch


@dataclass
class StreamSpec:
    """A beam's channelisation, sampling, DM plan and sample dtype."""

    freqs: np.ndarray
    f_ref: float
    t_samp: float
    ranges: list
    dtype: str = "u8"


@dataclass
class _Beam:
    spec: StreamSpec
    plan: Plan
    window: object          # device [n_chan][overlap + chunk]
    out: object             # device flat output of one window
    stream: object          # torch.cuda.Stream
    n_chunks: int = 0
    kept: list = field(default_factory=list)  # host copies of kept outputs per chunk
    bytes: int = 0


@dataclass
class _Job:
    beam: int
    chunk: object           # pinned host [n_chan][chunk]
    arrival: float
    event: object = None


def overlap_for(plan: Plan, ranges) -> int:
    """Raw samples of overlap so that each step emits chunk / bin new outputs."""
    info = plan.info(0)
    need = max(b * s for b, s in zip([r[3] for r in ranges], info["s_max"]))
    lcm = 1
    for r in ranges:
        lcm = np.lcm(lcm, int(r[3]))
    lcm = int(np.lcm(lcm, 16))
    return int((need + lcm - 1) // lcm * lcm)


class StreamServer:
    """Admits beams under an HBM budget and dedisperses their chunks as they arrive."""

    def __init__(self, chunk: int, hbm_budget_bytes: int, device="cuda", keep_outputs=False,
                 plan_cache: dict | None = None):
        torch = _torch()
        self.device = torch.device(device)
        self.chunk = int(chunk)
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.keep_outputs = keep_outputs
        self.beams: dict[int, _Beam] = {}
        self.waiting: collections.deque = collections.deque()  # (beam_id, spec) not yet admitted
        self.queue: collections.deque = collections.deque()    # jobs of admitted beams
        self.inflight: list[_Job] = []
        self.latencies: list[float] = []
        self.samples_done = 0
        self.rejected = 0
        self.plan_cache = {} if plan_cache is None else plan_cache

    # -- admission ---------------------------------------------------------
    def _plan(self, spec: StreamSpec) -> Plan:
        key = (spec.freqs.tobytes(), spec.f_ref, spec.t_samp, tuple(map(tuple, spec.ranges)),
               spec.dtype)
        if key not in self.plan_cache:
            self.plan_cache[key] = Plan(spec.freqs, spec.f_ref, spec.t_samp, spec.ranges,
                                        spec.dtype, device=self.device)
        return self.plan_cache[key]

    def beam_bytes(self, spec: StreamSpec) -> int:
        plan = self._plan(spec)
        ov = overlap_for(plan, spec.ranges)
        n = ov + self.chunk
        in_bytes = (n + 1) // 2 if spec.dtype == "u4" else n * {"u8": 1, "u16": 2, "f32": 4}[spec.dtype]
        return len(spec.freqs) * in_bytes + plan.info(n)["out_elems"] * 4

    def request(self, beam_id: int, spec: StreamSpec) -> bool:
        """Admit a beam now if its memory fits the budget, else queue it."""
        if beam_id in self.beams:
            return True
        need = self.beam_bytes(spec)
        if need > self.budget:
            self.rejected += 1
            return False
        if self.used + need <= self.budget and not self.waiting:
            self._admit(beam_id, spec, need)
            return True
        self.waiting.append((beam_id, spec))
        return False

    def _admit(self, beam_id: int, spec: StreamSpec, need: int):
        torch = _torch()
        from .batch import input_buffer
        plan = self._plan(spec)
        ov = overlap_for(plan, spec.ranges)
        n = ov + self.chunk
        window = input_buffer(spec.dtype, len(spec.freqs), n, self.device)
        out = plan.empty_output(n, self.device)
        self.beams[beam_id] = _Beam(spec, plan, window, out, torch.cuda.Stream(self.device),
                                    bytes=need)
        self.used += need

    def release(self, beam_id: int):
        """A beam's stream ended: free its memory and admit waiting beams."""
        beam = self.beams.pop(beam_id)
        beam.stream.synchronize()
        self.used -= beam.bytes
        while self.waiting:
            bid, spec = self.waiting[0]
            need = self.beam_bytes(spec)
            if self.used + need > self.budget:
                break
            self.waiting.popleft()
            self._admit(bid, spec, need)
        return beam

    def is_admitted(self, beam_id: int) -> bool:
        return beam_id in self.beams

    # -- work ----------------------------------------------------------------
    def submit(self, beam_id: int, chunk_host, arrival: float | None = None):
        """Queue one chunk ([n_chan][chunk] host tensor, ideally pinned)."""
        self.queue.append(_Job(beam_id, chunk_host, time.perf_counter() if arrival is None
                               else arrival))

    def _launch(self, job: _Job):
        torch = _torch()
        beam = self.beams[job.beam]
        plan, ov = beam.plan, overlap_for(beam.plan, beam.spec.ranges)
        n = ov + self.chunk
        # Column indices of the window buffer ("u4" packs two samples per byte;
        # the overlap and the chunk are even).
        spe = 2 if beam.spec.dtype == "u4" else 1
        with torch.cuda.stream(beam.stream):
            beam.window[:, ov // spe:n // spe].copy_(job.chunk, non_blocking=True)
            plan.run(beam.window, out=beam.out, n_samp=n, stream=beam.stream)
            if self.keep_outputs:
                beam.kept.append(self._kept(beam, n, ov))
            # The tail of this window is the next step's overlap.
            tail = beam.window[:, self.chunk // spe:n // spe]
            beam.window[:, :ov // spe].copy_(tail.clone() if ov > self.chunk else tail)
            ev = torch.cuda.Event()
            ev.record(beam.stream)
        job.event = ev
        beam.n_chunks += 1
        self.inflight.append(job)

    def _kept(self, beam: _Beam, n: int, ov: int):
        """Host copies of this step's new outputs: chunk / bin samples per range."""
        planes = beam.plan.split(beam.out, n)
        kept = []
        for (lo, hi, step, b), p in zip(beam.spec.ranges, planes):
            first = beam.n_chunks == 0
            start = ov // b if first else 0
            kept.append(p[:, start:self.chunk // b].cpu())
        return kept

    def pump(self, block: bool = False):
        """Launch queued chunks of admitted beams; retire finished ones."""
        keep = collections.deque()
        while self.queue:
            job = self.queue.popleft()
            if job.beam in self.beams:
                self._launch(job)
            else:
                keep.append(job)
        self.queue = keep
        self._retire(block)

    def _retire(self, block: bool):
        now_list = []
        for job in self.inflight:
            if block:
                job.event.synchronize()
            if job.event.query():
                t = time.perf_counter()
                self.latencies.append(t - job.arrival)
                self.samples_done += self.chunk
            else:
                now_list.append(job)
        self.inflight = now_list

    def drain(self):
        while self.queue or self.inflight:
            self.pump(block=True)

    def stats(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.array([np.nan])
        return {"chunks": len(self.latencies), "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "max_ms": float(np.max(lat) * 1e3), "admitted": len(self.beams),
                "waiting": len(self.waiting), "rejected": self.rejected,
                "hbm_used_bytes": self.used}

    def outputs(self, beam: _Beam):
        """Concatenated kept outputs per range (host) of a beam kept with keep_outputs."""
        return [np.concatenate([k[r].numpy() for k in beam.kept], axis=1)
                for r in range(len(beam.spec.ranges))]
