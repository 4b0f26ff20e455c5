"""Batched dedispersion of many beams in one persistent launch (dd_batch_*).

Beams may differ in channel count, dtype, sampling time and DM plan.  Each
beam's plan gets a register tile chosen by the autotuner, which times every
feasible candidate on the beam's own shapes and caches the winner by plan
signature -- the per-telescope tuning of the paper's tile parameters
(Sec. 4.1) done automatically.  The candidates are the pattern tile and the
packed-input tile in each shape of the shape table (window words per lane H,
warps per CTA, channels per stage; dd_tile_shapes) and the offset tile with
4, 2 or 1 DMs per lane.  The batch then runs as persistent launches (one per
tile variant, after the packing launches of packed-tile beams) over
(beam range, DM block, time tile) work lists, optionally captured once in a
CUDA graph and replayed.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os
from dataclasses import dataclass

import numpy as np

from . import Plan, _lib
from ._lib import check

BATCH_SHAPES = ("pattern", 4, 2, 1)  # tile families the persistent kernels serve


def tile_candidates(plan: Plan, r: int, packed: bool = True):
    """Every (tile, shape) the batch can run range r of the plan on: the
    pattern tile (and, for bin-1 ranges of packable dtypes, the packed tile)
    in each shape that serves it, then the offset tiles.  Leaves the range on
    its automatic tile."""
    from . import tile_shapes
    out = []
    tiles = ["pattern"] + (["packed"] if packed and plan.dtype in ("u8", "u4", "u16", "f32")
                           and int(plan.ranges[r][3]) == 1 else [])
    for tile in tiles:
        for i, sh in enumerate(tile_shapes()):
            try:
                plan.set_tile_shape(r, tile, i)
                out.append((tile, i))
            except _lib.DDError:
                pass
    for dr in (4, 2, 1):
        try:
            plan.set_tile(r, dr)
            out.append((dr, -1))
        except _lib.DDError:
            pass
    plan.set_tile(r, 0)
    return out


def apply_tile(plan: Plan, r: int, cand):
    """Put range r on a candidate of tile_candidates ((tile, shape) or a bare
    tile as Plan.set_tile takes it)."""
    if isinstance(cand, (list, tuple)):
        tile, shape = cand
        if tile in ("pattern", "packed"):
            plan.set_tile_shape(r, tile, int(shape))
            return
        cand = tile
    plan.set_tile(r, cand)


@dataclass
class BeamSpec:
    """One beam: channel frequencies, sampling, DM plan, dtype and length."""

    freqs: np.ndarray
    f_ref: float
    t_samp: float
    ranges: list
    dtype: str
    n_samp: int


def _torch():
    import torch
    return torch


def input_buffer(dtype: str, n_chan: int, n_samp: int, device, n_cols: int | None = None):
    """Zeroed device input [n_chan][row] with 16-byte rows for n_samp samples
    (n_cols: samples per row instead).  "u4" rows hold packed bytes, two
    samples each (row stride in samples a multiple of 32)."""
    torch = _torch()
    esz = {"u8": 1, "u16": 2, "f32": 4, "u4": 1}[dtype]
    per = 32 if dtype == "u4" else 16 // esz
    n = n_samp if n_cols is None else n_cols
    stride = (n + per - 1) // per * per
    row_bytes = stride // 2 if dtype == "u4" else stride * esz
    raw = torch.zeros((n_chan, row_bytes), dtype=torch.uint8, device=device)
    return raw.view({"u8": torch.uint8, "u16": torch.uint16, "f32": torch.float32,
                     "u4": torch.uint8}[dtype])


def plan_signature(plan: Plan, n_samp: int) -> str:
    """Key of the autotune cache: everything that changes the tile's work."""
    h = hashlib.sha1(plan.freqs.tobytes()).hexdigest()[:16]
    return json.dumps([plan.dtype, plan.n_chan, h, plan.f_ref, plan.t_samp,
                       [list(r) for r in plan.ranges], int(n_samp)])


class Autotuner:
    """Times every feasible (tile, shape) of each range of a plan and keeps the
    fastest (each candidate timed with its own packing pass, if any)."""

    def __init__(self, shapes=None, reps: int = 3, cache_path: str | None = None,
                 packed: bool = True):
        self.shapes = None if shapes is None else tuple(shapes)  # restrict to these tiles
        self.reps = reps
        self.packed = packed
        self.cache_path = cache_path or os.environ.get("DD_AUTOTUNE_CACHE")
        self.cache = {}
        if self.cache_path and os.path.exists(self.cache_path):
            with open(self.cache_path) as fh:
                self.cache = json.load(fh)
        self.log = []

    def _feasible(self, plan: Plan, r: int):
        cands = tile_candidates(plan, r, packed=self.packed)
        if self.shapes is not None:
            cands = [c for c in cands if c[0] in self.shapes]
        return cands

    def choose(self, plan: Plan, n_samp: int, x, out):
        """Pick and set a (tile, shape) for every range of the plan; returns them."""
        torch = _torch()
        key = plan_signature(plan, n_samp) + ("|packed" if self.packed else "")
        if self.shapes is not None:  # a restricted tuner keeps its own entries
            key += "|tiles=" + json.dumps(list(self.shapes), default=str)
        if key in self.cache:
            choice = [tuple(c) if isinstance(c, list) else c for c in self.cache[key]]
            for r, c in enumerate(choice):
                apply_tile(plan, r, c)
            return choice
        choice = []
        for r in range(len(plan.ranges)):
            feas = self._feasible(plan, r)
            if not feas:
                raise _lib.DDError(_lib.DD_ERR_UNSUPPORTED,
                                   f"range {r} fits none of the batch tiles")
            best, best_ms = feas[0], float("inf")
            if len(feas) > 1:
                for cand in feas:
                    apply_tile(plan, r, cand)
                    # Full copies for packed candidates, as the batch runs them.
                    plan.run(x, out=out, n_samp=n_samp, segments=0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(self.reps):
                        plan.run(x, out=out, n_samp=n_samp, segments=0)
                    e1.record()
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / self.reps
                    self.log.append((key, r, cand, ms))
                    if ms < best_ms:
                        best, best_ms = cand, ms
            apply_tile(plan, r, best)
            choice.append(best)
        self.cache[key] = choice
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as fh:
                json.dump(self.cache, fh)
            os.replace(tmp, self.cache_path)
        return choice


class BatchRunner:
    """Owns per-beam device buffers and runs all beams as one persistent launch."""

    def __init__(self, beams, device="cuda", autotune: bool = True, graph: bool = True,
                 tuner: Autotuner | None = None, tiles=None):
        """tiles: optional per beam, a list of per-range tiles (as Plan.set_tile
        takes them) used instead of the autotuner or the first feasible tile."""
        torch = _torch()
        self.device = torch.device(device)
        self.beams = list(beams)
        self.plans, self.inputs, self.outputs = [], [], []
        self.tuner = tuner or (Autotuner() if autotune else None)
        self.shapes = []
        for b in self.beams:
            plan = Plan(b.freqs, b.f_ref, b.t_samp, b.ranges, b.dtype, device=self.device)
            x = input_buffer(b.dtype, plan.n_chan, b.n_samp, self.device)
            out = plan.empty_output(b.n_samp, self.device)
            if tiles is not None:
                self.shapes.append(list(tiles[len(self.plans)]))
            elif self.tuner is not None:
                self.shapes.append(self.tuner.choose(plan, b.n_samp, x, out))
            else:
                shp = []
                for r in range(len(b.ranges)):
                    for dr in BATCH_SHAPES:
                        try:
                            plan.set_tile(r, dr)
                            shp.append(dr)
                            break
                        except _lib.DDError:
                            continue
                self.shapes.append(shp)
            if tiles is not None:
                for r, t in enumerate(tiles[len(self.plans)]):
                    apply_tile(plan, r, t)
            self.plans.append(plan)
            self.inputs.append(x)
            self.outputs.append(out)
        lib = _lib.load()
        n = len(self.plans)
        handles = (ctypes.c_void_p * n)(*[p.handle.value for p in self.plans])
        n_samp = (ctypes.c_int64 * n)(*[b.n_samp for b in self.beams])
        h = ctypes.c_void_p()
        check(lib.dd_batch_create(handles, n_samp, n, ctypes.byref(h)))
        self._h = h
        self._lib = lib
        # Per-beam scratch of packed-tile beams (their packed copies).
        self.scratch = []
        for i in range(n):
            need = ctypes.c_size_t()
            check(lib.dd_batch_plan_scratch_bytes(h, i, ctypes.byref(need)))
            self.scratch.append(torch.empty(need.value, dtype=torch.uint8, device=self.device)
                                if need.value else None)
        nbytes = ctypes.c_size_t()
        check(lib.dd_batch_workspace_bytes(h, ctypes.byref(nbytes)))
        self.workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=self.device)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        check(lib.dd_batch_upload(h, self.workspace.data_ptr(), self.workspace.numel(), stream))
        self.bind()
        n_items, n_jobs = ctypes.c_int64(), ctypes.c_int32()
        check(lib.dd_batch_info(h, ctypes.byref(n_items), ctypes.byref(n_jobs)))
        self.n_items, self.n_jobs = n_items.value, n_jobs.value
        n_launch = ctypes.c_int32()
        check(lib.dd_batch_launches(h, ctypes.byref(n_launch)))
        self.n_launches = n_launch.value  # kernel launches per run
        self.graph = None
        if graph:
            self._capture()

    def bind(self):
        """Upload the job table (buffers and each plan's launch parameters,
        dd_batch_bind); again after a plan's wait limit changes."""
        torch = _torch()
        n = len(self.plans)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        d_in = (ctypes.c_void_p * n)(*[x.data_ptr() for x in self.inputs])
        strides = (ctypes.c_int64 * n)(*[x.stride(0) * (2 if b.dtype == "u4" else 1)
                                         for x, b in zip(self.inputs, self.beams)])
        d_out = (ctypes.c_void_p * n)(*[o.data_ptr() for o in self.outputs])
        d_sc = (ctypes.c_void_p * n)(*[None if t is None else t.data_ptr() for t in self.scratch])
        n_sc = (ctypes.c_size_t * n)(*[0 if t is None else t.numel() for t in self.scratch])
        check(self._lib.dd_batch_bind_scratch(self._h, d_in, strides, d_out, d_sc, n_sc, stream))

    def _launch(self):
        torch = _torch()
        check(self._lib.dd_batch_run(self._h, torch.cuda.current_stream(self.device).cuda_stream))

    def _capture(self):
        torch = _torch()
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self._launch()  # warm-up outside the graph
        torch.cuda.current_stream(self.device).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._launch()
        self.graph = g

    def run(self):
        """One persistent launch over every beam (graph replay if captured)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._launch()

    def status(self):
        torch = _torch()
        check(self._lib.dd_batch_status(self._h, torch.cuda.current_stream(self.device).cuda_stream))

    def planes(self, i: int):
        return self.plans[i].split(self.outputs[i], self.beams[i].n_samp)

    def run_per_beam(self):
        """The plain path: one dd_run per beam (dd_run_scratch with the full
        copies of its packed ranges), in order, on the current stream."""
        for p, x, o, b in zip(self.plans, self.inputs, self.outputs, self.beams):
            p.run(x, out=o, n_samp=b.n_samp, segments=0)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
