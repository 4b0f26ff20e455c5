"""Streaming dedispersion server: continuous batching of many beams on one GPU.

Each admitted beam keeps a device window of `overlap + chunk` raw samples per
channel.  A new chunk is copied into the window behind the overlap (the last
`overlap` samples of the previous step, kept on the device), and the window is
dedispersed with dd_run_window for the first `chunk / bin_r` outputs of every
DM range r only: with overlap >= max_r bin_r * S_max_r those are the next
`chunk / bin_r` outputs of the stream, equal to the same samples of a one-shot
transform of the concatenated stream (the paper's real-time processing,
Sec. 5.4, done incrementally), and no output is computed twice.  The window's
tail becomes the next overlap.  Ranges that the packed-input tile serves run
on it (uint8 at bins 1, 2, 4 and 8), from a packed copy of the window made in
one of a few scratch slots the server shares among its beams (a slot is
reused once the launch that last used it is done); the budget counts the
slots once and each beam's window and outputs.

Serving is continuous batching: each beam has its own CUDA stream, chunks are
launched as soon as they arrive, so work of different beams overlaps on the
device; beams are admitted while their device memory (window, packed copy,
output planes) fits an HBM budget and wait otherwise until another beam
leaves.  Latency is measured from a chunk's arrival to its outputs being ready
on the device.  snapshot() / restore() carry a beam's stream state (its
overlap and position) across a server restart.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import DDError, Plan


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
    out: object             # device: per range [n_dm_r][chunk / bin_r], concatenated
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
                 plan_cache: dict | None = None, packed: bool = True, scratch_slots: int = 4):
        """chunk: raw samples per chunk (a multiple of 16 and of every range's
        bin); packed: run the ranges the packed-input tile serves on it, with
        `scratch_slots` shared scratch buffers for the packed copies."""
        torch = _torch()
        self.device = torch.device(device)
        self.n_slots = max(1, int(scratch_slots))
        self.slots = []          # [buffer, event of its last use]
        self.slot_bytes = 0
        self._next_slot = 0
        self.chunk = int(chunk)
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.keep_outputs = keep_outputs
        self.packed = packed
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
               spec.dtype, self.packed)
        if key not in self.plan_cache:
            plan = Plan(spec.freqs, spec.f_ref, spec.t_samp, spec.ranges, spec.dtype,
                        device=self.device)
            if self.packed:
                for r in range(len(spec.ranges)):
                    try:
                        plan.set_tile(r, "packed")
                    except DDError:
                        pass  # this range stays on the plan's automatic tile
            self.plan_cache[key] = plan
        return self.plan_cache[key]

    def keep_counts(self, spec: StreamSpec) -> list:
        """New outputs per range per chunk: chunk / bin_r."""
        for r in spec.ranges:
            if self.chunk % int(r[3]):
                raise ValueError("the chunk must be a multiple of every range's bin")
        return [self.chunk // int(r[3]) for r in spec.ranges]

    def _sizes(self, spec: StreamSpec):
        plan = self._plan(spec)
        ov = overlap_for(plan, spec.ranges)
        n = ov + self.chunk
        out_elems = sum(a * b for a, b in zip(plan.info(0)["n_dm"], self.keep_counts(spec)))
        return plan, ov, n, out_elems, plan.input_scratch_bytes(n)

    def beam_bytes(self, spec: StreamSpec) -> int:
        """Device bytes of one admitted beam: window and outputs (the packed
        copies live in the server's shared scratch slots)."""
        plan, ov, n, out_elems, scratch = self._sizes(spec)
        in_bytes = (n + 1) // 2 if spec.dtype == "u4" else n * {"u8": 1, "u16": 2, "f32": 4}[spec.dtype]
        return len(spec.freqs) * in_bytes + out_elems * 4

    def slots_bytes(self, spec: StreamSpec) -> int:
        """Device bytes of the shared scratch slots a beam of `spec` needs
        (counted once for all beams)."""
        return self.n_slots * self._sizes(spec)[4]

    def _ensure_slots(self, scratch: int) -> bool:
        """Grow the shared scratch slots to `scratch` bytes each if the budget
        allows (with nothing in flight); False if it does not."""
        torch = _torch()
        if scratch <= self.slot_bytes:
            return True
        extra = self.n_slots * (scratch - self.slot_bytes)
        if self.used + extra > self.budget:
            return False
        for job in self.inflight:
            job.event.synchronize()
        self.slots = [[torch.empty(scratch, dtype=torch.uint8, device=self.device), None]
                      for _ in range(self.n_slots)]
        self.used += extra
        self.slot_bytes = scratch
        return True

    def request(self, beam_id: int, spec: StreamSpec) -> bool:
        """Admit a beam now if its memory fits the budget, else queue it."""
        if beam_id in self.beams:
            return True
        need = self.beam_bytes(spec)
        scratch = self._sizes(spec)[4]
        if need + self.n_slots * max(scratch, self.slot_bytes) > self.budget:
            self.rejected += 1
            return False
        if (self.used + need <= self.budget and not self.waiting and
                self._ensure_slots(scratch) and self.used + need <= self.budget):
            self._admit(beam_id, spec, need)
            return True
        self.waiting.append((beam_id, spec))
        return False

    def _admit(self, beam_id: int, spec: StreamSpec, need: int):
        torch = _torch()
        from .batch import input_buffer
        plan, ov, n, out_elems, scratch = self._sizes(spec)
        window = input_buffer(spec.dtype, len(spec.freqs), n, self.device)
        out = torch.empty(max(out_elems, 4), dtype=plan.out_dtype(), device=self.device)
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
            if (self.used + need > self.budget or not self._ensure_slots(self._sizes(spec)[4])
                    or self.used + need > self.budget):
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
        slot = None
        if plan.input_scratch_bytes(n):
            slot = self.slots[self._next_slot]
            self._next_slot = (self._next_slot + 1) % self.n_slots
        with torch.cuda.stream(beam.stream):
            beam.window[:, ov // spe:n // spe].copy_(job.chunk, non_blocking=True)
            if slot is not None and slot[1] is not None:
                beam.stream.wait_event(slot[1])  # the slot's last user is done with it
            plan.run_window(beam.window, self.keep_counts(beam.spec), out=beam.out, n_samp=n,
                            stream=beam.stream, scratch=None if slot is None else slot[0])
            if slot is not None:
                slot[1] = torch.cuda.Event()
                slot[1].record(beam.stream)
            if self.keep_outputs:
                beam.kept.append(self._kept(beam, ov))
            # The tail of this window is the next step's overlap.
            tail = beam.window[:, self.chunk // spe:n // spe]
            beam.window[:, :ov // spe].copy_(tail.clone() if ov > self.chunk else tail)
            ev = torch.cuda.Event()
            ev.record(beam.stream)
        job.event = ev
        beam.n_chunks += 1
        self.inflight.append(job)

    def planes(self, beam: _Beam):
        """Views of a beam's last window outputs: per range [n_dm_r][chunk / bin_r]."""
        n_dm = beam.plan.info(0)["n_dm"]
        out, off = [], 0
        for a, b in zip(n_dm, self.keep_counts(beam.spec)):
            out.append(beam.out[off:off + a * b].view(a, b))
            off += a * b
        return out

    def _kept(self, beam: _Beam, ov: int):
        """Host copies of this step's new outputs: chunk / bin samples per range.
        Output t of the k-th window is decimated sample (k chunk - ov) / bin + t
        of the stream; those before the stream's start read the zeroed overlap
        and are dropped."""
        kept = []
        for (lo, hi, step, b), p in zip(beam.spec.ranges, self.planes(beam)):
            start = max(0, (ov - beam.n_chunks * self.chunk) // b)
            kept.append(p[:, start:].cpu())
        return kept

    # -- checkpoint / resume -------------------------------------------------
    def snapshot(self, beam_id: int) -> dict:
        """State of an admitted beam between chunks, on the host: its spec, the
        overlap samples of its window and the number of chunks done.  A server
        that restores it continues the stream exactly where this one stopped.
        Chunks of the beam still queued here would be in neither, so they are
        refused: pump() or drain() first."""
        if any(j.beam == beam_id for j in self.queue):
            raise RuntimeError(f"beam {beam_id} has queued chunks: pump() or drain() before "
                               "snapshot()")
        beam = self.beams[beam_id]
        beam.stream.synchronize()
        ov = overlap_for(beam.plan, beam.spec.ranges)
        spe = 2 if beam.spec.dtype == "u4" else 1
        return {"spec": beam.spec, "chunk": self.chunk, "n_chunks": beam.n_chunks,
                "overlap": beam.window[:, :ov // spe].cpu()}

    def restore(self, beam_id: int, state: dict) -> bool:
        """Admit a beam from snapshot() state (same chunk size); False if the
        budget does not admit it now (then it is not queued)."""
        if state["chunk"] != self.chunk:
            raise ValueError("snapshot taken with another chunk size")
        spec = state["spec"]
        need = self.beam_bytes(spec)
        if (beam_id in self.beams or self.used + need > self.budget or
                not self._ensure_slots(self._sizes(spec)[4]) or self.used + need > self.budget):
            return False
        self._admit(beam_id, spec, need)
        beam = self.beams[beam_id]
        ov = overlap_for(beam.plan, spec.ranges)
        spe = 2 if spec.dtype == "u4" else 1
        beam.window[:, :ov // spe].copy_(state["overlap"].to(self.device))
        beam.n_chunks = int(state["n_chunks"])
        return True

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

    def has_work(self, beam_id: int) -> bool:
        """A chunk of the beam is queued or on the device."""
        return any(j.beam == beam_id for j in self.queue) or any(
            j.beam == beam_id for j in self.inflight)

    def drain(self):
        """Run every queued chunk of admitted beams to completion (chunks of
        beams still waiting for admission stay queued)."""
        while self.inflight or any(j.beam in self.beams for j in self.queue):
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
