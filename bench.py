#!/usr/bin/env python3
"""Benchmark: brute-force dedispersion throughput on one GB300 (or N replicas).

Default workload: the paper-scale 8-bit case -- 8192 channels x 262144
samples of uint8 (16.8 s at 64 us), 4096 trial DMs 0..409.5 step 0.1,
1670 MHz top of a 320 MHz band.  One step = one dd_run over the whole input
(inputs resident in HBM; 2.1 GB in + 4.2 GB out, far larger than L2, so no
flush is needed between steps).

Prints ONE JSON line (rank 0).  Metric: DM-trial x output-samples per second.
Extra keys: channel-adds/s, real-time factor R = t_obs / t_step (Sec. 5.4),
the ALU roofline of the dominant kernel, the oracle's CPU baseline and an
end-to-end (host buffers through the C ABI) number.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference   # the CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "DM-trials x samples / s"
SM_MAX_MHZ = 2070.0   # GB300 maximum SM clock
def _measured_hbm_gbs(default=6800.0):
    """The machine's measured HBM copy bandwidth (MEASURED_PEAKS.json beside this
    file, written per machine pool), else the recipe's 6.8 TB/s fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return default


HBM_GBS = _measured_hbm_gbs()
# dram__bytes_read.sum + dram__bytes_write.sum of the transform launches the
# roofline times (ncu), keyed by workload, raw samples, tiles, input mode and
# segments; valid only for the kernel build it was taken on
# (profiles/fwd_pattern_u8_8192ch.md).
TRAFFIC = {("paper_u8", 262144, (0x104,), "packed ring", 8): 18.29e9 + 13.42e9}
UNIT = "DM*samples/s"


def _workload(name, n_samp=None):
    import dataclasses
    from synth import workloads
    beam = {"paper_u8": workloads.paper_u8, "paper_u16": workloads.paper_u16,
            "paper_u4": workloads.paper_u4, "tiny_u8": workloads.tiny_u8,
            "diff_f32": workloads.diff_f32}[name]()
    if n_samp:  # a shorter observation of the same plan (profiler captures)
        beam = dataclasses.replace(beam, n_samp=int(n_samp))
    return beam


def _describe(beam):
    r = beam.ranges
    plan = "; ".join(f"DM {lo:g}-{hi:g} step {st:g} bin {b}" for lo, hi, st, b in r)
    return (f"{beam.name}: {beam.dtype} {beam.n_chan} ch x {beam.n_samp} samples, "
            f"{beam.f_high:g} MHz top, {beam.bandwidth:g} MHz band, "
            f"{beam.t_samp * 1e6:g} us; {plan}")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_throughput(units: float, seconds: float, device) -> tuple:
    """Whole-job throughput of independent replicas: every rank processed
    `units` in `seconds`; the job took the slowest rank's time, so value =
    world_size * units / max(seconds).  Returns (value, max seconds)."""
    import torch
    ws = 1
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        ws = torch.distributed.get_world_size()
        t = torch.tensor([seconds], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        seconds = float(t.item())
    return units * ws / seconds, seconds


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names[1:], parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measure_alu_peak(torch, lib):
    """Measured 3-input integer add rate (lane-ops/s) from the register microbenchmark."""
    import ctypes
    sms, clk = ctypes.c_int32(), ctypes.c_int32()
    lib.dd_bench_device(ctypes.byref(sms), ctypes.byref(clk))
    blocks, threads, iters = int(sms.value) * 4, 512, 4096
    sink = torch.empty(blocks * threads, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    ops = ctypes.c_double()
    res = {}
    for kind, name in [(1, "iadd3"), (2, "iadd2"), (3, "fadd"), (4, "fadd2"), (5, "iadd3_imad"),
                       (6, "lds128")]:
        best = 0.0
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lib.dd_bench_launch(kind, blocks, threads, iters, sink.data_ptr(), stream.cuda_stream,
                                ctypes.byref(ops))
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            best = max(best, blocks * threads * iters * ops.value / sec)
        res[name] = best
    res["sm_count"] = int(sms.value)
    res["lds128_bytes_per_s"] = res["lds128"] * 16
    return res


def run_ours(args):
    import torch
    import paper_2311_05341_gb300 as dd
    from paper_2311_05341_gb300 import _lib
    from synth import workloads

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    lib = _lib.load()

    beam = _workload(args.workload, args.n_samp)
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, beam.dtype,
                   device=f"cuda:{local}")
    if args.tile != "auto":
        for r in range(len(beam.ranges)):
            plan.set_tile(r, args.tile if args.tile in ("pattern", "packed")
                          else int(args.tile))
    elif beam.dtype == "f32":
        # Float32's fastest tile (float pairs) reads a packed copy with other
        # tables than the automatic tile's, so it is asked for explicitly.
        for r in range(len(beam.ranges)):
            try:
                plan.set_tile(r, "packed")
            except dd.DDError:
                pass
    info = plan.info(beam.n_samp)
    # Caller-owned scratch (allocated once, like the output): the packed ring
    # of `segments` time segments for the ranges with a packed copy (the
    # automatic uint8 / 4-bit / uint16 tiles), the full copies for
    # --segments 1, none for 0.
    need = plan.input_scratch_bytes(beam.n_samp)
    mode = "input read directly"
    if any(info["packed_copy"]) and args.segments > 0:
        try:
            need = max(need, plan.packed_scratch_bytes(beam.n_samp, args.segments))
            mode = "packed ring" if args.segments > 1 else "packed full copy"
        except dd.DDError:
            need = max(need, plan.packed_scratch_bytes(beam.n_samp, 1))
            mode = "packed full copy"
    scratch = (torch.empty(int(need), dtype=torch.uint8, device=f"cuda:{local}")
               if need else None)
    tables = {}

    def shift_rows(r, d):
        if r not in tables:
            tables[r] = plan.shifts(r)
        return tables[r][d]

    # Rows start 16-byte aligned; strides count samples (two per byte for "u4").
    per = 32 if beam.dtype == "u4" else 16 // np.dtype(beam.np_dtype).itemsize
    row_stride = (beam.n_samp + per - 1) // per * per
    spe = 2 if beam.dtype == "u4" else 1  # samples per buffer element
    x_host = workloads.make_input(beam, shift_rows, info["n_dm"], info["n_out"],
                                  row_stride=row_stride)
    x = torch.from_numpy(x_host).cuda()
    out = plan.empty_output(beam.n_samp)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def step():
        """One pass: dd_run_scratch over the whole input (in ring mode it packs
        segment k + 1 while the kernels of segment k run, on the plan's side
        streams joined back into this one)."""
        plan.run_raw(x.data_ptr(), x.stride(0) * spe, beam.n_samp, out.data_ptr(), sp,
                     scratch=scratch)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    dm_samples = sum(a * b for a, b in zip(info["n_dm"], info["n_out"]))
    chan_adds = dm_samples * beam.n_chan
    launches_per_step = _launches_per_step(plan, info, mode, args.segments)

    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for i in range(args.steps):
        step()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    per = [evs[i].elapsed_time(evs[i + 1]) / 1e3 for i in range(args.steps)]
    value, total = replica_throughput(dm_samples * args.steps, sum(per), "cuda")
    ms_per_step = total / args.steps * 1e3
    # The same tables in one transform launch from the full packed copy (the
    # copy made first, outside the launch's events), and the unpacking kernel
    # without scratch: the dominant kernel timed alone, the ncu launch list's
    # per-launch figure.
    single = _single_launch_times(torch, lib, plan, info, x, spe, beam.n_samp, out, stream, args)
    # In ring mode the step's transform launches overlap each other and the
    # packing, so the roofline takes the whole step (a lower bound on the
    # kernels' own rate); with one launch per range the launch time.
    kern = (total / args.steps if mode != "packed full copy" or single is None
            else single["kernel_ms"] / 1e3)

    # End to end through the C ABI: pinned host in -> device -> pinned host out.
    e2e = None
    e2e_buffers = None
    if not args.no_e2e:
        h_in = torch.from_numpy(x_host).pin_memory()
        h_out = torch.empty(info["out_elems"], dtype=plan.out_dtype()).pin_memory()
        plan.run_host(h_in, h_out, x, out, n_samp=beam.n_samp)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(1, min(args.steps, 5))
        e0.record(stream)
        for _ in range(k):
            plan.run_host(h_in, h_out, x, out, n_samp=beam.n_samp)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / k
        e2e = {"value": dm_samples * ws / sec, "unit": UNIT,
               "h2d_bytes_per_step": int(h_in.numel() * h_in.element_size()),
               "d2h_bytes_per_step": int(h_out.numel() * h_out.element_size()),
               "ms_per_step": sec * 1e3}
        e2e_buffers = (h_in, h_out)

    peaks = measure_alu_peak(torch, lib)
    if rank != 0:
        return
    # Roofline of the dominant (only) kernel: sample-adds per launch / mean launch time,
    # against the add rate derived from the SM's integer units and clock (a
    # three-input add retires on the 16-lane integer pipe of each of the 4 SM
    # sub-partitions; float adds on both 16-lane float pipes).
    sample_adds_per_s = chan_adds / kern
    sms = peaks["sm_count"]
    per_lane = {"u8": 4, "u4": 4, "u16": 2, "f32": 1}[beam.dtype]
    lanes = 128 if beam.dtype == "f32" else 64  # lane-ops per clock per SM
    peak_adds = lanes * sms * SM_MAX_MHZ * 1e6 * per_lane
    algo_bytes = (beam.n_chan * beam.n_samp * np.dtype(beam.np_dtype).itemsize // spe
                  + info["out_elems"] * 4)
    traffic = TRAFFIC.get((args.workload, beam.n_samp, tuple(info["tile_dms"]), mode,
                           args.segments))
    roofline = {
        "bound": "alu", "achieved": sample_adds_per_s / 1e12, "peak": peak_adds / 1e12,
        "unit": "Tadd/s", "frac": sample_adds_per_s / peak_adds,
        "traffic": traffic,
        "kernel_ms": kern * 1e3,
        "timed": ("the whole step: %d transform launches on two streams with the packing "
                  "overlapped" % launches_per_step["transform"]) if mode == "packed ring"
                 else "the transform launch alone",
        "frac_whole_step": chan_adds / (total / args.steps) / peak_adds,
        "peak_source": ("%d lane-ops/clk/SM x %d SMs x %g MHz x %d sample-adds per lane-op"
                        % (lanes, sms, SM_MAX_MHZ, per_lane)),
        "alu_microbench": {k: v for k, v in peaks.items()},
        "frac_of_microbench": sample_adds_per_s / (
            peaks["iadd3"] * per_lane if beam.dtype != "f32" else peaks["fadd"]),
        # Against one sample per two-input add on both 16-lane pipes (no packing):
        # above 1 is the gain of the packed sample-adds.
        "frac_of_scalar_adds": sample_adds_per_s / (128 * sms * SM_MAX_MHZ * 1e6),
        "hbm": {"algorithmic_bytes": algo_bytes,
                "achieved_gbs": algo_bytes / (total / args.steps) / 1e9,
                "frac_of_measured": algo_bytes / (total / args.steps) / 1e9 / HBM_GBS},
    }
    t_obs = beam.n_samp * beam.t_samp
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"u8": "int32", "u4": "int32", "u16": "int32", "f32": "f32"}[beam.dtype],
        "data": "synthetic",
        "config": {"workload": _describe(beam), "n_dm": info["n_dm_total"],
                   "n_out": info["n_out"],
                   "tile": [{_lib.DD_TILE_PATTERN: "pattern",
                             _lib.DD_TILE_PACKED: "packed"}.get(t, t)
                            for t in info["tile_dms"]],
                   "input": mode + (f" ({args.segments} segments, "
                                    f"{need / 1e9:.2f} GB scratch)" if mode == "packed ring"
                                    else f" ({need / 1e9:.2f} GB scratch)" if need else ""),
                   "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{ws}"},
        "channel_adds_per_s": chan_adds * args.steps * ws / total,
        "real_time_factor": t_obs / (ms_per_step / 1e3),
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": args.steps * launches_per_step["total"],
        "clocks": clk,
    }
    if single is not None:
        single["frac"] = chan_adds / (single["kernel_ms"] / 1e3) / peak_adds
        if "unpacked_ms" in single:
            single["frac_unpacked_kernel"] = chan_adds / (single["unpacked_ms"] / 1e3) / peak_adds
        line["single_launch"] = single
    if beam.dtype == "f32":
        line["adjoint"] = _adjoint_timing(args, plan, x, info, beam, stream)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(beam, x_host, info, args.cpu_rows)
        if beam.dtype in ("u8", "u16", "f32") and len(beam.ranges) == 1 and beam.ranges[0][3] == 1:
            line["cpu_baseline_tiled"] = cpu_tiled_baseline(beam, x_host, plan.shifts(0), info,
                                                            args.cpu_tiled_rows)
    if ws == 1 and args.workload == "paper_u8" and not args.no_extras:
        # The rest of the headline metric on the same GPU: batched vs plain
        # (config 3), streamed vs plain with p50/p99 latency and the real-time
        # factor over an arrival-rate sweep (config 5), and the float32
        # forward / adjoint / training step (config 4).  Each carries its own
        # clock record.
        del x, out, scratch, e2e_buffers
        torch.cuda.empty_cache()
        line["batched"] = batched_result(args)
        line["stream"] = stream_result(args)
        line["diff_f32"] = diff_result(args)
    print(json.dumps(line))


def _launches_per_step(plan, info, mode, segments):
    """Kernel launches of one dd_run_scratch: per range one transform launch
    (plus one packing launch per copy); in ring mode one packing launch and
    one launch per ring range for every segment with outputs (the library's
    segment rule: boundaries k * ceil(n / segments) rounded down to each
    range's time tiles, n the longest ring range's outputs)."""
    shapes = None
    n_ranges = len(info["n_out"])
    if mode == "packed full copy":
        return {"transform": n_ranges, "total": n_ranges + 1}
    if mode != "packed ring":
        return {"transform": n_ranges, "total": n_ranges + (1 if plan.input_scratch_bytes(
            info["n_samp"]) else 0)}
    import paper_2311_05341_gb300 as dd
    shapes = dd.tile_shapes()
    ring = [r for r in range(n_ranges) if info["packed_copy"][r]]
    n_max = max(info["n_out"][r] for r in ring)
    seg = -(-n_max // segments)
    transform, packs = n_ranges - len(ring), 0
    for k in range(segments):
        busy = 0
        for r in ring:
            sh = shapes[info["tile_shape"][r]]
            ts = 32 * sh["words_per_lane"] * (1 if plan.dtype == "u16" else 2)
            n_out = info["n_out"][r]
            lo = min(n_out, k * seg // ts * ts)
            hi = n_out if k == segments - 1 else min(n_out, (k + 1) * seg // ts * ts)
            busy += hi > lo
        transform += busy
        packs += busy > 0
    return {"transform": transform, "total": transform + packs}


def _single_launch_times(torch, lib, plan, info, x, spe, n_samp, out, stream, args):
    """Ranges with a packed copy: the full copies (dd_pack_input), then one
    transform launch per range from them (dd_run_packed) timed alone with
    CUDA events; and dd_run without scratch (the automatic tiles unpacking
    the input themselves).  None without such a range."""
    if not any(info["packed_copy"]):
        return None
    from paper_2311_05341_gb300 import _lib
    full = plan.packed_scratch_bytes(n_samp, 1)
    sc = torch.empty(full, dtype=torch.uint8, device=x.device)
    sp = stream.cuda_stream
    args_in = (plan.handle, x.data_ptr(), x.stride(0) * spe, n_samp)

    def pack():
        _lib.check(lib.dd_pack_input(*args_in, sc.data_ptr(), full, sp))

    def run():
        _lib.check(lib.dd_run_packed(*args_in, out.data_ptr(), sc.data_ptr(), full, sp))

    pack_s = _timed(pack, args.steps, args.warmup, stream)
    pack()
    run_s = _timed(run, args.steps, args.warmup, stream)
    del sc
    res = {"what": "full packed copy (dd_pack_input), then the transform launch alone "
                   "(dd_run_packed)", "pack_ms": pack_s * 1e3, "kernel_ms": run_s * 1e3}
    if plan.input_scratch_bytes(n_samp) == 0:
        def unpacked():
            plan.run_raw(x.data_ptr(), x.stride(0) * spe, n_samp, out.data_ptr(), sp)
        res["unpacked_ms"] = _timed(unpacked, args.steps, args.warmup, stream) * 1e3
    torch.cuda.empty_cache()
    return res


def _adjoint_timing(args, plan, x, info, beam, stream):
    """Float32 plans: the adjoint gather (dd_run_adjoint) alone, and one
    training step through the autograd Function (forward, loss = sum Y * W,
    backward to the filterbank), each timed with CUDA events."""
    import torch
    from paper_2311_05341_gb300 import autograd as ddg

    n = beam.n_samp
    g = torch.Generator(device="cuda").manual_seed(4)
    w = torch.randn(info["out_elems"], device="cuda", generator=g)
    xbar = torch.empty((beam.n_chan, (n + 3) // 4 * 4), dtype=torch.float32, device="cuda")
    xr = x[:, :n].clone().requires_grad_(True)

    def adjoint():
        plan.run_adjoint(w, n, xbar=xbar, stream=stream)

    def step():
        xr.grad = None
        planes = ddg.dedisperse(xr, plan)
        loss = sum((p.reshape(-1) * wp).sum() for p, wp in
                   zip(planes, torch.split(w, [p.numel() for p in planes])))
        loss.backward()

    out = {}
    for name, fn in (("adjoint", adjoint), ("train_step", step)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out[name] = {"ms": ms,
                     "dm_samples_per_s": sum(a * b for a, b in zip(info["n_dm"], info["n_out"]))
                     / (ms / 1e3)}
    out["what"] = ("adjoint: Plan.run_adjoint of a random cotangent (dd_run_adjoint_scratch: "
                   "kernel %s); train_step: autograd forward + loss sum(Y W) + backward "
                   "(forward, adjoint, elementwise)" % info.get("adjoint_kernel"))
    return out


def cpu_baseline(beam, x_host, info, n_rows):
    """The oracle, as it stands, on a bounded sample: n_rows full-length DM rows."""
    import oracle
    rows = np.linspace(0, info["n_dm"][0] - 1, n_rows).astype(np.int64)
    t0 = time.perf_counter()
    x = oracle.Packed4(x_host, beam.n_samp) if beam.dtype == "u4" else x_host
    oracle.forward_rows(x, beam.freqs, beam.f_high, beam.t_samp, beam.ranges[0], rows)
    sec = time.perf_counter() - t0
    units = n_rows * info["n_out"][0]
    return {"value": units / sec, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{n_rows} of {info['n_dm'][0]} DM rows, full length "
                      f"({info['n_out'][0]} samples), range 0", "seconds": sec}


def cpu_tiled_baseline(beam, x_host, shifts, info, n_rows):
    """The tiled CPU scheme (cpu_baseline/, the paper's Algorithm 2) on a
    bounded sample: n_rows consecutive DM rows from the middle, full length."""
    import cpu_baseline
    d0 = max(0, info["n_dm"][0] // 2 - n_rows // 2)
    rows = shifts[d0:d0 + n_rows]
    cpu_baseline.forward(x_host, rows[:16], 4096)  # build / warm
    t0 = time.perf_counter()
    cpu_baseline.forward(x_host, rows, info["n_out"][0])
    sec = time.perf_counter() - t0
    import oracle
    return {"value": rows.shape[0] * info["n_out"][0] / sec, "unit": UNIT,
            "cores": oracle.threads(), "kind": "tiled CPU (Algorithm 2 scheme)",
            "sample": f"DM rows {d0}..{d0 + rows.shape[0] - 1} of {info['n_dm'][0]}, full length "
                      f"({info['n_out'][0]} samples)", "seconds": sec}


def run_reference(args):
    """The CPU oracle timed as it stands on a bounded sample of the workload."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    from synth import workloads
    import oracle
    beam = _workload(args.workload)
    tables = [oracle.shift_table(beam.freqs, beam.f_high, beam.t_samp, r) for r in beam.ranges]
    n_dm = [t.shape[0] for t in tables]
    n_out = [oracle.extent(beam.freqs, beam.f_high, beam.t_samp, r, beam.n_samp)[1]
             for r in beam.ranges]
    x = workloads.make_input(beam, lambda r, d: tables[r][d], n_dm, n_out)
    if beam.dtype == "u4":
        x = oracle.Packed4(x, beam.n_samp)
    n_rows = args.cpu_rows_reference
    rows = np.linspace(0, n_dm[0] - 1, n_rows).astype(np.int64)

    def step():
        oracle.forward_rows(x, beam.freqs, beam.f_high, beam.t_samp, beam.ranges[0], rows)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    sec = time.perf_counter() - t0
    value = n_rows * n_out[0] * args.steps / sec
    sample = f"{n_rows} of {n_dm[0]} DM rows, full length ({n_out[0]} samples) per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": _describe(beam), "n_dm": sum(n_dm), "n_out": n_out},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def _timed(fn, steps, warmup, stream=None):
    """Mean seconds per call of fn over `steps` calls after `warmup` calls
    (CUDA events on the current stream)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps / 1e3


def batched_result(args):
    """Config 3: 24 u8 + 8 u16 + 4 f32 beams in persistent launches (one per
    tile variant, autotuned tiles, CUDA graph) against the plain path (one
    dd_run per beam on each plan's tuned tile), same inputs, same outputs."""
    import torch
    import paper_2311_05341_gb300 as dd
    from paper_2311_05341_gb300 import batch as ddb
    from synth import workloads

    beams = workloads.batched()
    specs = [ddb.BeamSpec(b.freqs, b.f_high, b.t_samp, b.ranges, b.dtype, b.n_samp) for b in beams]
    t_setup = time.perf_counter()
    runner = ddb.BatchRunner(specs, autotune=True, graph=True)
    for b, x in zip(beams, runner.inputs):
        h = workloads.make_input(b, lambda r, d, b=b: _plan_shifts_cache(b)[r][d], *_sizes(b))
        x[:, : b.n_samp].copy_(torch.from_numpy(h).to(x.device))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    infos = [p.info(b.n_samp) for p, b in zip(runner.plans, beams)]
    units = sum(sum(a * c for a, c in zip(i["n_dm"], i["n_out"])) for i in infos)
    adds = sum(sum(a * c for a, c in zip(i["n_dm"], i["n_out"])) * b.n_chan
               for i, b in zip(infos, beams))
    # The plain per-beam path: one dd_run per beam on the plan's automatic
    # tile (what dd_plan_create gives, no scratch), one after another on one
    # stream; and Plan.run's default per beam (the automatic tiles from a
    # packed ring where they have a packed copy).
    plain = [dd.Plan(b.freqs, b.f_high, b.t_samp, b.ranges, b.dtype) for b in beams]
    plain_out = [p.empty_output(b.n_samp) for p, b in zip(plain, beams)]
    tuned_out = [torch.empty_like(o) for o in runner.outputs]
    ring_out = [torch.empty_like(o) for o in runner.outputs]

    def plain_step():
        for p, x, o, b in zip(plain, runner.inputs, plain_out, beams):
            p.run(x, out=o, n_samp=b.n_samp, segments=0)

    def ring_step():
        for p, x, o, b in zip(plain, runner.inputs, ring_out, beams):
            p.run(x, out=o, n_samp=b.n_samp)

    def tuned_step():  # per beam again, on the batch's tuned tiles
        for p, x, o, b, sc in zip(runner.plans, runner.inputs, tuned_out, beams, runner.scratch):
            p.run_raw(x.data_ptr(), x.stride(0), b.n_samp, o.data_ptr(),
                      torch.cuda.current_stream().cuda_stream, scratch=sc)

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t_plain = _timed(plain_step, args.steps, args.warmup)
    t_ring = _timed(ring_step, args.steps, args.warmup)
    t_tuned = _timed(tuned_step, args.steps, args.warmup)
    t_batch = _timed(runner.run, args.steps, args.warmup)
    clk = clocks.stop()
    runner.status()
    same = all(torch.equal(a, c) for a, c in zip(plain_out, runner.outputs))
    same_tuned = all(torch.equal(a, c) for a, c in zip(tuned_out, runner.outputs))
    same_ring = all(torch.equal(a, c) for a, c in zip(ring_out, runner.outputs))
    tiles = {}
    for b, shp in zip(beams, runner.shapes):
        tiles.setdefault(b.dtype, [str(t) for t in shp])
    res = {
        "workload": "24 x u8 1024 ch x 131072 (2048 DMs step 0.1), 8 x u16 4096 ch x 65536 "
                    "at 54.6 us (3072 DMs step 0.2), 4 x f32 336 ch x 32768 at 327.68 us "
                    "(1024 DMs step 0.2)",
        "value": units / t_batch, "unit": UNIT, "ms_per_step": t_batch * 1e3,
        "channel_adds_per_s": adds / t_batch,
        "plain_per_beam": {"value": units / t_plain, "ms_per_step": t_plain * 1e3,
                           "what": "one dd_run per beam, automatic tiles, one stream"},
        "batched_over_plain": t_plain / t_batch,
        "outputs_identical_to_plain": bool(same),
        "per_beam_ring": {"value": units / t_ring, "ms_per_step": t_ring * 1e3,
                          "what": "Plan.run per beam (automatic tiles from a 8-segment "
                                  "packed ring where they have a packed copy), one stream",
                          "outputs_identical": bool(same_ring)},
        "batched_over_per_beam_ring": t_ring / t_batch,
        "per_beam_same_tiles": {"value": units / t_tuned, "ms_per_step": t_tuned * 1e3,
                                "what": "one run per beam on the batch's tuned tiles"},
        "batched_over_same_tiles": t_tuned / t_batch,
        "outputs_identical_same_tiles": bool(same_tuned),
        "beams": len(beams), "work_items": runner.n_items, "tiles": tiles,
        "launches_per_step": runner.n_launches, "setup_s": t_setup, "clocks": clk,
    }
    del runner, plain_out, tuned_out, ring_out, plain
    torch.cuda.empty_cache()
    return res


def run_batched(args):
    res = batched_result(args)
    line = {"metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "mixed",
            "data": "synthetic", "config": {"workload": "batched: " + res["workload"]},
            "gpu_launches": args.steps * res["launches_per_step"], "clocks": res["clocks"],
            "batched": res}
    print(json.dumps(line))


def stream_result(args):
    """Config 5: 64 u8 beams of 4096 channels, chunks of 65536 samples, the
    4-range decimated plan.  (1) Saturated: the server (windowed outputs,
    packed tile, one stream per beam) against the plain per-beam path (dd_run
    over the whole overlap + chunk window, one stream), on the same chunks,
    with identical outputs.  (2) Poisson arrivals at each rate (multiples of
    real time): p50/p99 chunk latency and the aggregate real-time factor
    (Sec. 5.4's R); the knee is the highest rate whose p99 stays within one
    chunk's duration."""
    import torch
    from paper_2311_05341_gb300 import stream as dds
    from synth import filterbank, poisson_arrivals, workloads

    chunk, n_beams = 65536, 64
    beam0 = workloads.stream_beam(0, chunk)
    spec = dds.StreamSpec(beam0.freqs, beam0.f_high, beam0.t_samp, beam0.ranges, "u8")
    pool = [torch.from_numpy(filterbank(np.uint8, beam0.n_chan, chunk, 5000 + i, 128, 16))
            .pin_memory() for i in range(4)]
    chunk_s = chunk * beam0.t_samp
    budget = int(args.hbm_budget_gb * 2**30)
    plan_cache = {}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    sat = _stream_saturated(args, spec, pool, chunk, plan_cache)
    sweep = []
    for m in args.stream_rates:
        srv = dds.StreamServer(chunk, budget, plan_cache=plan_cache)
        # Every beam streams for the whole window: Poisson arrivals at m times
        # its real-time chunk rate (64 m / 4.19 s chunks per second offered).
        n_max = int(np.ceil(args.stream_seconds * m / chunk_s * 3)) + 8
        sched = []
        for b in range(n_beams):
            ts = poisson_arrivals(7000 + b + int(m * 100), m / chunk_s, n_max)
            sched += [(float(t), b) for t in ts if t < args.stream_seconds]
        sched.sort()
        last = {}
        for k, (_, b) in enumerate(sched):
            last[b] = k  # a beam's stream ends with its last scheduled chunk
        for b in range(n_beams):
            srv.request(b, spec)
        t0 = time.perf_counter()
        i = 0
        ended = set()
        while i < len(sched) or srv.queue or srv.inflight:
            now = time.perf_counter() - t0
            while i < len(sched) and sched[i][0] <= now:
                _, b = sched[i]
                srv.submit(b, pool[(b + i) % len(pool)], arrival=t0 + sched[i][0])
                if last[b] == i:
                    ended.add(b)
                i += 1
            srv.pump()
            for b in list(ended):  # streams that ended leave and free their memory
                if srv.is_admitted(b) and not srv.has_work(b):
                    srv.release(b)
                    ended.discard(b)
            if now > 4 * args.stream_seconds:
                break  # far over capacity: stop waiting
            time.sleep(0.0005)
        srv.drain()
        wall = time.perf_counter() - t0
        st = srv.stats()
        dm_samples_per_chunk = sum(
            n * (chunk // r[3]) for n, r in zip(srv._plan(spec).info(0)["n_dm"], spec.ranges))
        sweep.append({"rate_x_realtime": m, "chunks_offered": len(sched),
                      "chunks": st["chunks"], "p50_ms": st["p50_ms"],
                      "p99_ms": st["p99_ms"], "max_ms": st["max_ms"], "wall_s": wall,
                      "admitted": st["admitted"], "waiting": st["waiting"],
                      "real_time_factor_aggregate": st["chunks"] * chunk_s / wall,
                      "dm_samples_per_s": st["chunks"] * dm_samples_per_chunk / wall})
        del srv
    clk = clocks.stop()
    # The knee: the highest swept rate the server keeps up with -- it serves
    # at least 97 % of the offered real-time factor (n_beams x rate), so no
    # queue builds up over the window.
    ok = [r for r in sweep
          if r["real_time_factor_aggregate"] >= 0.97 * n_beams * r["rate_x_realtime"]]
    knee = max(ok, key=lambda r: r["rate_x_realtime"]) if ok else None
    res = {"workload": "64 beams u8 4096 ch, 1670 MHz top, 320 MHz band, 64 us, chunks 65536 "
                       "+ overlap; DM 0-150/0.1 b1, 150-300/0.2 b2, 300-1000/0.5 b4, "
                       "1000-2000/1.0 b8",
           "chunk_s": chunk_s, "hbm_budget_gb": args.hbm_budget_gb,
           "saturated": sat, "sweep": sweep,
           "knee_x_realtime": knee["rate_x_realtime"] if knee else None,
           "knee_p50_ms": knee["p50_ms"] if knee else None,
           "knee_p99_ms": knee["p99_ms"] if knee else None,
           "knee_rule": "highest swept rate whose served real-time factor is >= 97 % of the "
                        "offered one (64 beams x rate)",
           "capacity_x_realtime": sat["real_time_factor_server"] / n_beams,
           "clocks": clk}
    torch.cuda.empty_cache()
    return res


def run_stream(args):
    res = stream_result(args)
    print(json.dumps({"metric": "p50/p99 chunk latency, real-time factor", **res}))


def _stream_saturated(args, spec, pool, chunk, plan_cache):
    """Server against the plain per-beam path on the same chunks, all queued at
    once: the plain path runs every beam's chunks one after another on one
    stream (copy in, dd_run of the whole window on the plan's automatic tiles
    without scratch, keep the overlap); the server launches them on per-beam streams and
    computes each range's chunk / bin new outputs only (dd_run_window).  Both
    end with each beam's last window outputs, which depend on every earlier
    chunk through the overlap; they must be equal."""
    import torch
    import paper_2311_05341_gb300 as dd
    from paper_2311_05341_gb300 import stream as dds
    from paper_2311_05341_gb300.batch import input_buffer

    n_beams, per_beam = args.stream_sat_beams, args.stream_sat_chunks
    srv = dds.StreamServer(chunk, int(args.hbm_budget_gb * 2**30), plan_cache=plan_cache)
    plan = dd.Plan(spec.freqs, spec.f_ref, spec.t_samp, spec.ranges, spec.dtype)
    ov = dds.overlap_for(plan, spec.ranges)
    n = ov + chunk
    keep = srv.keep_counts(spec)
    dm_samples_per_chunk = sum(k * c for k, c in zip(plan.info(0)["n_dm"], keep))
    jobs = [(b, pool[(b + j) % len(pool)]) for j in range(per_beam) for b in range(n_beams)]

    # Plain: one stream, beam after beam.
    windows = [input_buffer(spec.dtype, len(spec.freqs), n, "cuda") for _ in range(n_beams)]
    outs = [plan.empty_output(n) for _ in range(n_beams)]

    def plain():
        for b in range(n_beams):
            for j in range(per_beam):
                windows[b][:, ov:n].copy_(pool[(b + j) % len(pool)], non_blocking=True)
                plan.run(windows[b], out=outs[b], n_samp=n, segments=0)
                tail = windows[b][:, chunk:n]
                windows[b][:, :ov].copy_(tail.clone() if ov > chunk else tail)

    def server():
        for b in range(n_beams):
            srv.request(b, spec)
        for b, c in jobs:
            srv.submit(b, c)
        srv.drain()

    for w in windows:
        w.zero_()
    plain()  # warm-up (plans, allocator)
    torch.cuda.synchronize()
    for w in windows:
        w.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain()
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0

    server()  # warm-up: the beams stay admitted; reset their windows
    torch.cuda.synchronize()
    for b in range(n_beams):
        srv.beams[b].window.zero_()
    srv.latencies.clear()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    server()
    torch.cuda.synchronize()
    t_srv = time.perf_counter() - t0
    same = True
    for b in range(n_beams):
        for k, p_srv, p_plain in zip(keep, srv.planes(srv.beams[b]), plan.split(outs[b], n)):
            same = same and torch.equal(p_srv, p_plain[:, :k])
    total = len(jobs) * dm_samples_per_chunk
    st = srv.stats()
    res = {"beams": n_beams, "chunks": len(jobs),
           "server_dm_samples_per_s": total / t_srv, "server_s": t_srv,
           "plain_per_beam_dm_samples_per_s": total / t_plain, "plain_s": t_plain,
           "server_over_plain": t_plain / t_srv,
           "real_time_factor_server": len(jobs) * chunk * spec.t_samp / t_srv,
           "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
           "outputs_identical_to_plain": bool(same)}
    for b in list(srv.beams):
        srv.release(b)
    del windows, outs, srv
    return res


def diff_result(args):
    """Config 4: float32 1024 ch x 65536 at 128 us, 1024 DMs: forward,
    adjoint and one training step (forward, loss sum(Y W), backward through
    the autograd Function), CUDA events, against the float add roofline."""
    import torch
    import paper_2311_05341_gb300 as dd
    from paper_2311_05341_gb300 import _lib
    from synth import workloads

    beam = _workload("diff_f32")
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, beam.dtype)
    plan.set_tile(0, "packed")  # float pairs: two adds per instruction
    info = plan.info(beam.n_samp)
    x_host = workloads.make_input(beam, lambda r, d: plan.shifts(r)[d], info["n_dm"],
                                  info["n_out"], row_stride=(beam.n_samp + 3) // 4 * 4)
    x = torch.from_numpy(x_host).cuda()
    out = plan.empty_output(beam.n_samp)
    scratch = torch.empty(plan.input_scratch_bytes(beam.n_samp), dtype=torch.uint8, device="cuda")
    sp = torch.cuda.current_stream().cuda_stream
    lib = plan._lib
    stream = torch.cuda.current_stream()

    def pack():
        _lib.check(lib.dd_pack_input(plan.handle, x.data_ptr(), x.stride(0), beam.n_samp,
                                     scratch.data_ptr(), scratch.numel(), sp))

    def transform():
        _lib.check(lib.dd_run_packed(plan.handle, x.data_ptr(), x.stride(0), beam.n_samp,
                                     out.data_ptr(), scratch.data_ptr(), scratch.numel(), sp))

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t_fwd = _timed(lambda: (pack(), transform()), args.steps, args.warmup)
    # The transform launch alone (CUDA events around it, the packing outside).
    ks = []
    for _ in range(args.steps):
        pack()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        transform()
        e1.record(stream)
        ks.append((e0, e1))
    torch.cuda.synchronize()
    t_kern = sum(a.elapsed_time(b) for a, b in ks) / len(ks) / 1e3
    adj = _adjoint_timing(args, plan, x, info, beam, torch.cuda.current_stream())
    clk = clocks.stop()
    dm_samples = sum(a * b for a, b in zip(info["n_dm"], info["n_out"]))
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = 128 * sms * SM_MAX_MHZ * 1e6  # FP32 add lanes per clock per SM x SMs x clock
    adds = dm_samples * beam.n_chan
    res = {"workload": _describe(beam), "tile": "packed (float pairs)",
           "forward": {"ms": t_fwd * 1e3, "dm_samples_per_s": dm_samples / t_fwd,
                       "adds_per_s": adds / t_fwd, "frac_with_packing": adds / t_fwd / peak,
                       "kernel_ms": t_kern * 1e3, "frac": adds / t_kern / peak},
           "adjoint": {**adj["adjoint"], "frac": adds / (adj["adjoint"]["ms"] / 1e3) / peak,
                       "kernel": info["adjoint_kernel"]},
           "train_step": adj["train_step"],
           "adjoint_over_forward": adj["adjoint"]["ms"] / (t_fwd * 1e3),
           "peak": {"value": peak / 1e12, "unit": "Tadd/s",
                    "source": "128 FP32 lanes/clk/SM x %d SMs x %g MHz" % (sms, SM_MAX_MHZ)},
           "clocks": clk}
    del x, out, plan, scratch
    torch.cuda.empty_cache()
    return res


def run_frontend(args):
    """Time-major (receiver / SIGPROC order) input of the paper-scale uint8
    workload: the transpose kernel alone against HBM bandwidth, and the whole
    host-to-host pipeline (copy in, transpose, dedisperse, copy out)."""
    import torch
    import paper_2311_05341_gb300 as dd
    from synth import workloads

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    beam = _workload("paper_u8", args.n_samp)
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, beam.dtype)
    info = plan.info(beam.n_samp)
    x_cm = workloads.make_input(beam, lambda r, d: plan.shifts(r)[d], info["n_dm"], info["n_out"])
    x_tm = np.ascontiguousarray(x_cm[:, : beam.n_samp].T)
    h_in = torch.from_numpy(x_tm).pin_memory()
    h_out = torch.empty(info["out_elems"], dtype=torch.int32).pin_memory()
    d_tm = h_in.to("cuda")
    d_cm = torch.empty((beam.n_chan, (beam.n_samp + 15) // 16 * 16), dtype=torch.uint8,
                       device="cuda")
    out = plan.empty_output(beam.n_samp)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / args.steps

    clocks = ClockSampler(local)
    clocks.start()
    t_tr = timed(lambda: dd.transpose(d_tm, out=d_cm))
    t_e2e = timed(lambda: plan.run_host_tmajor(h_in, h_out, d_tm, d_cm, out,
                                               n_samp=beam.n_samp))
    clk = clocks.stop()
    # Parity of the transposed input on sampled rows.
    same = all(np.array_equal(d_cm[c, : beam.n_samp].cpu().numpy(), x_cm[c, : beam.n_samp])
               for c in (0, beam.n_chan // 2, beam.n_chan - 1))
    units = sum(a * b for a, b in zip(info["n_dm"], info["n_out"]))
    tr_bytes = 2 * beam.n_chan * beam.n_samp
    line = {
        "metric": METRIC, "value": units / t_e2e, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_e2e * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "frontend: " + _describe(beam) + "; time-major host input",
                   "path": "pinned host -> device, transpose, dedisperse, device -> pinned host"},
        "transpose": {"ms": t_tr * 1e3, "bytes": tr_bytes,
                      "roofline": {"bound": "hbm", "achieved": tr_bytes / t_tr / 1e9,
                                   "peak": HBM_GBS, "unit": "GB/s",
                                   "frac": tr_bytes / t_tr / 1e9 / HBM_GBS,
                                   "traffic": None},
                      "rows_equal_definition": bool(same)},
        "gpu_launches": None, "clocks": clk,
    }
    print(json.dumps(line))


_SHIFT_CACHE = {}


def _plan_shifts_cache(beam):
    import paper_2311_05341_gb300 as dd
    key = beam.name.rsplit("_", 1)[0]
    if key not in _SHIFT_CACHE:
        p = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, beam.dtype, upload=False)
        _SHIFT_CACHE[key] = ([p.shifts(r) for r in range(len(beam.ranges))], p.info(beam.n_samp))
    return _SHIFT_CACHE[key][0]


def _sizes(beam):
    _plan_shifts_cache(beam)
    inf = _SHIFT_CACHE[beam.name.rsplit("_", 1)[0]][1]
    return inf["n_dm"], inf["n_out"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper_u8",
                    choices=["paper_u8", "paper_u16", "paper_u4", "tiny_u8", "diff_f32", "batched",
                             "stream", "frontend"])
    ap.add_argument("--stream-rates", type=float, nargs="+",
                    default=[1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0])
    ap.add_argument("--stream-seconds", type=float, default=8.0)
    ap.add_argument("--stream-sat-beams", type=int, default=16)
    ap.add_argument("--stream-sat-chunks", type=int, default=4)
    ap.add_argument("--hbm-budget-gb", type=float, default=170.0)
    ap.add_argument("--cpu-rows", type=int, default=96)
    ap.add_argument("--cpu-rows-reference", type=int, default=16)
    ap.add_argument("--cpu-tiled-rows", type=int, default=256)
    ap.add_argument("--n-samp", type=int, default=None,
                    help="raw samples per channel instead of the workload's (smaller "
                         "cases for profiler captures)")
    ap.add_argument("--tile", default="auto",
                    help="register tile of every range: auto (packed where it serves), "
                         "pattern, packed or the offset tile's DMs per lane "
                         "(8, 6, 4, 2, 1)")
    ap.add_argument("--segments", type=int, default=8,
                    help="ranges with a packed copy: time segments of the packed ring "
                         "(1: the full copy, 0: no packed copy)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="paper_u8 only: skip the batched, streaming and float32 results "
                         "that the default line carries")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "stream":
        run_stream(args)
    elif args.workload == "frontend":
        run_frontend(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
