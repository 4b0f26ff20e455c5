"""Host-side checks of the C-ABI library (no GPU needed).

The library must load, export every entry point the public headers declare,
plan exactly the oracle's shift tables for every workload, and reject bad
arguments with the documented status codes.
"""
import ctypes
import glob
import json
import os
import re

import numpy as np
import pytest

import paper_2311_05341_gb300 as dd
from paper_2311_05341_gb300 import _lib
from synth import channel_freqs, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(dd_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    declared = _declared_functions()
    assert {"dd_plan_create", "dd_run", "dd_run_adjoint"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(_lib.SIGNATURES) >= declared


def test_status_strings():
    lib = _lib.load()
    for code, name in [(0, "DD_OK"), (1, "DD_ERR_INVALID_ARG"), (2, "DD_ERR_UNSUPPORTED"),
                       (3, "DD_ERR_SHAPE"), (4, "DD_ERR_BUDGET"), (5, "DD_ERR_CUDA"),
                       (6, "DD_ERR_TIMEOUT")]:
        assert lib.dd_status_string(code).decode() == name


def _beams():
    return [workloads.tiny_u8(), workloads.paper_u8(), workloads.diff_f32(),
            workloads.batched()[0], workloads.batched()[24], workloads.batched()[32],
            workloads.stream_beam(0, 65536 + 24632)]


@pytest.mark.parametrize("beam", _beams(), ids=lambda b: b.name)
def test_plan_tables_equal_oracle(oracle_mod, beam):
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, beam.dtype, upload=False)
    info = plan.info(beam.n_samp)
    for r, rng in enumerate(beam.ranges):
        ref = oracle_mod.shift_table(beam.freqs, beam.f_high, beam.t_samp, rng)
        got = plan.shifts(r)
        assert got.shape == ref.shape
        assert np.array_equal(got, ref), f"range {r}"
        s_max, n_out = oracle_mod.extent(beam.freqs, beam.f_high, beam.t_samp, rng, beam.n_samp)
        assert info["s_max"][r] == s_max
        assert info["n_out"][r] == n_out
        assert info["n_dm"][r] == oracle_mod.n_dm(rng)


def test_plan_info_layout():
    beam = workloads.stream_beam(0, 65536 + 24632)
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, beam.dtype, upload=False)
    info = plan.info(beam.n_samp)
    off = 0
    for r in range(4):
        assert info["out_offset"][r] == off
        off += info["n_dm"][r] * info["n_out"][r]
    assert info["out_elems"] == off
    assert info["n_dm"] == [1500, 750, 1400, 1000]
    raw = max((s + 1) * rr[3] - 1 for s, rr in zip(info["s_max"], beam.ranges))
    assert info["max_delay_raw"] == raw


def _create(freqs, f_ref, ts, ranges, dtype=_lib.DD_U8):
    lib = _lib.load()
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    arr = (_lib.Range * max(len(ranges), 1))(*[_lib.Range(*r) for r in ranges])
    h = ctypes.c_void_p()
    st = lib.dd_plan_create(f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), f.size, f_ref, ts,
                            arr, len(ranges), dtype, ctypes.byref(h))
    if st == 0:
        lib.dd_plan_destroy(h)
    return st


@pytest.mark.parametrize("args", [
    ([1400.0, 1300.0], 1400.0, 0.0, [(0.0, 10.0, 1.0, 1)]),        # t_samp = 0
    ([1400.0, 1500.0], 1400.0, 1e-4, [(0.0, 10.0, 1.0, 1)]),       # f > f_ref
    ([1400.0, -1.0], 1400.0, 1e-4, [(0.0, 10.0, 1.0, 1)]),         # f <= 0
    ([1400.0], 1400.0, 1e-4, [(0.0, 10.0, 0.0, 1)]),               # step 0
    ([1400.0], 1400.0, 1e-4, [(10.0, 10.0, 1.0, 1)]),              # empty range
    ([1400.0], 1400.0, 1e-4, [(0.0, 10.0, 1.0, 0)]),               # bin 0
    ([1400.0], 1400.0, 1e-4, [(-5.0, 10.0, 1.0, 1)]),              # negative DM
    ([1400.0], 1400.0, 1e-4, []),                                  # no ranges
    ([1400.0], 1400.0, 1e-4, [(0.0, 1.0, 1.0, 1)] * 17),           # too many ranges
])
def test_plan_create_rejects_bad_arguments(args):
    assert _create(*args) == _lib.DD_ERR_INVALID_ARG


def test_plan_create_rejects_bad_dtype():
    assert _create([1400.0], 1400.0, 1e-4, [(0.0, 1.0, 1.0, 1)], dtype=9) == _lib.DD_ERR_INVALID_ARG


def test_null_and_shape_errors():
    lib = _lib.load()
    assert lib.dd_plan_query(None, 10, None) == _lib.DD_ERR_INVALID_ARG
    assert lib.dd_run(None, None, 0, 0, None, None) == _lib.DD_ERR_INVALID_ARG
    plan = dd.Plan([1400.0, 1300.0], 1400.0, 1e-4, [(0.0, 10.0, 1.0, 1)], "u8", upload=False)
    # No workspace bound yet.
    assert lib.dd_run(plan.handle, 16, 64, 64, 16, None) == _lib.DD_ERR_INVALID_ARG
    # Workspace too small / misaligned (checked before any device call).
    assert lib.dd_plan_upload(plan.handle, 16, 0, None) == _lib.DD_ERR_BUDGET
    nb = plan.info(0)["workspace_bytes"]
    assert lib.dd_plan_upload(plan.handle, 8, nb, None) == _lib.DD_ERR_SHAPE
    assert lib.dd_plan_shifts(plan.handle, 3, None) == _lib.DD_ERR_INVALID_ARG
    u16 = dd.Plan([1400.0], 1400.0, 1e-4, [(0.0, 10.0, 1.0, 1)], "u16", upload=False)
    assert lib.dd_run_adjoint(u16.handle, 16, 16, 64, 64, None) == _lib.DD_ERR_UNSUPPORTED
    msg = lib.dd_last_error_detail().decode()
    assert "float32" in msg


def test_too_short_input_is_reported():
    plan = dd.Plan(workloads.tiny_u8().freqs, 1500.0, 64e-6, [(0.0, 64.0, 0.5, 1)], "u8",
                   upload=False)
    info = plan.info(100)
    assert info["n_out"][0] <= 0


def test_kernel_selection():
    paper = workloads.paper_u8()
    plan = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, "u8", upload=False)
    info = plan.info(paper.n_samp)
    # At most 1.23 samples of delay per DM step: the pattern tile.
    assert info["kernel"] == ["tiled"] and info["tile_dms"] == [_lib.DD_TILE_PATTERN]
    # Bins with bin * sample bytes dividing 16 are tiled (decimation fused)
    # while their raw windows fit shared memory; other bins run on the generic
    # kernel.
    stream = workloads.stream_beam(0, 90168)
    plan = dd.Plan(stream.freqs, stream.f_high, stream.t_samp, stream.ranges, "u8", upload=False)
    assert plan.info(stream.n_samp)["kernel"] == ["tiled"] * 4
    odd = [(0.0, 10.0, 0.5, 3), (10.0, 20.0, 1.0, 4)]
    plan = dd.Plan(stream.freqs, stream.f_high, stream.t_samp, odd, "u8", upload=False)
    assert plan.info(stream.n_samp)["kernel"] == ["generic", "tiled"]
    plan = dd.Plan(stream.freqs, stream.f_high, stream.t_samp, [(0.0, 10.0, 0.5, 8)], "f32",
                   upload=False)
    assert plan.info(stream.n_samp)["kernel"] == ["generic"]  # 8 * 4 bytes > 16
    # 8 samples of delay per DM step: only 2 DMs per lane fit the 4-bit offsets.
    tiny = workloads.tiny_u8()
    plan = dd.Plan(tiny.freqs, tiny.f_high, tiny.t_samp, tiny.ranges, "u8", upload=False)
    assert plan.info(tiny.n_samp)["tile_dms"] == [2]
    with pytest.raises(dd.DDError) as ei:
        plan.set_tile(0, 4)
    assert ei.value.status == _lib.DD_ERR_UNSUPPORTED
    assert plan.info(tiny.n_samp)["tile_dms"] == [2]
    f32 = workloads.diff_f32()
    plan = dd.Plan(f32.freqs, f32.f_high, f32.t_samp, f32.ranges, "f32", upload=False)
    assert plan.info(f32.n_samp)["kernel"] == ["tiled"]
    # 2.9 samples of delay per DM step: increments 2 or 3, base increment 2 of
    # the pattern tile (0..3).
    u16 = workloads.batched()[24]
    plan = dd.Plan(u16.freqs, u16.f_high, u16.t_samp, u16.ranges, "u16", upload=False)
    assert plan.info(u16.n_samp)["tile_dms"] == [_lib.DD_TILE_PATTERN]
    plan.set_tile(0, 0)
    plan.set_tile(0, 4)
    assert plan.info(u16.n_samp)["tile_dms"] == [4]
    fb = workloads.batched()[32]  # 12.3 samples of delay per DM step
    plan = dd.Plan(fb.freqs, fb.f_high, fb.t_samp, fb.ranges, "f32", upload=False)
    assert plan.info(fb.n_samp)["tile_dms"] == [1]


def test_pattern_tile_selection():
    """The pattern tile serves plans whose per-DM shift increments are 0, 1 or 2."""
    paper = workloads.paper_u8()  # at most 1.23 samples per DM step
    plan = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, "u8", upload=False)
    plan.set_tile(0, 6)
    ws_offset = plan.info(paper.n_samp)["workspace_bytes"]
    assert plan.info(paper.n_samp)["tile_dms"] == [6]
    plan.set_tile(0, "pattern")
    info = plan.info(paper.n_samp)
    assert info["kernel"] == ["tiled"] and info["tile_dms"] == [_lib.DD_TILE_PATTERN]
    # Per-warp pair lists against 64-byte offset records: other table sizes.
    assert info["workspace_bytes"] != ws_offset
    plan.set_tile(0, 6)
    plan.set_tile(0, 0)  # automatic: the pattern tile
    assert plan.info(paper.n_samp)["tile_dms"] == [_lib.DD_TILE_PATTERN]
    tiny = workloads.tiny_u8()  # 8 samples per DM step at the lowest channel
    plan = dd.Plan(tiny.freqs, tiny.f_high, tiny.t_samp, tiny.ranges, "u8", upload=False)
    with pytest.raises(dd.DDError) as ei:
        plan.set_tile(0, "pattern")
    assert ei.value.status == _lib.DD_ERR_UNSUPPORTED
    assert plan.info(tiny.n_samp)["tile_dms"] == [2]
    with pytest.raises(dd.DDError) as ei:
        plan.set_tile(0, 3)
    assert ei.value.status == _lib.DD_ERR_INVALID_ARG


def test_tile_shape_table_and_explicit_shapes():
    """dd_tile_shapes lists the pattern shapes (the automatic ones first, then
    the tuning entries); dd_plan_set_tile_shape puts a range on one of them,
    refuses shapes that cannot serve it (keeping the previous choice) and bad
    arguments; dd_plan_info reports the shape in use."""
    shapes = dd.tile_shapes()
    assert len(shapes) >= 12
    auto = [s["automatic"] for s in shapes]
    assert auto == sorted(auto, reverse=True) and 0 in auto and 1 in auto
    assert all(s["dms_per_lane"] == 4 and s["words_per_lane"] % 2 == 1 for s in shapes)
    paper = workloads.paper_u8()
    paper.n_chan, paper.ranges = 512, [(0.0, 51.2, 0.1, 1)]
    plan = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, "u8", upload=False)
    first = plan.info(paper.n_samp)["tile_shape"][0]
    assert shapes[first]["automatic"] and shapes[first]["channel_pairs"]
    served = 0
    for i, sh in enumerate(shapes):
        if sh["channel_pairs"] and not sh["float_pairs"]:
            plan.set_tile_shape(0, "pattern", i)
            info = plan.info(paper.n_samp)
            assert info["tile_shape"] == [i] and info["tile_dms"] == [_lib.DD_TILE_PATTERN]
            served += 1
        else:
            with pytest.raises(dd.DDError) as ei:
                plan.set_tile_shape(0, "pattern", i)
            assert ei.value.status == _lib.DD_ERR_UNSUPPORTED
            assert plan.info(paper.n_samp)["tile_shape"] != [i]
    assert served >= 5
    plan.set_tile_shape(0, "packed", -1)
    assert plan.info(paper.n_samp)["tile_dms"] == [_lib.DD_TILE_PACKED]
    f2 = [i for i, s in enumerate(shapes) if s["float_pairs"]]
    f32 = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, "f32", upload=False)
    for i in f2:
        # A window that does not fit shared memory (32 channels of float-pair
        # words on this plan) is refused; the automatic shapes all fit.
        try:
            f32.set_tile_shape(0, "packed", i)
        except dd.DDError as e:
            assert e.status == _lib.DD_ERR_UNSUPPORTED and not shapes[i]["automatic"]
            continue
        assert f32.info(paper.n_samp)["tile_shape"] == [i]
    lib = _lib.load()
    assert lib.dd_plan_set_tile_shape(plan.handle, 0, 6, 0) == _lib.DD_ERR_INVALID_ARG
    assert lib.dd_plan_set_tile_shape(plan.handle, 0, _lib.DD_TILE_PATTERN, len(shapes)) == \
        _lib.DD_ERR_INVALID_ARG
    assert lib.dd_plan_set_tile_shape(plan.handle, 5, _lib.DD_TILE_PATTERN, 0) == \
        _lib.DD_ERR_INVALID_ARG
    plan.set_tile(0, 6)
    assert plan.info(paper.n_samp)["tile_shape"] == [-1]


def test_u4_plan_selection_and_refusals():
    """4-bit plans take the pattern tile or the generic kernel (no offset
    tiles); the transpose front end refuses them."""
    paper = workloads.paper_u8()
    plan = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, "u4", upload=False)
    assert plan.info(paper.n_samp)["tile_dms"] == [_lib.DD_TILE_PATTERN]
    with pytest.raises(dd.DDError) as ei:
        plan.set_tile(0, 6)
    assert ei.value.status == _lib.DD_ERR_UNSUPPORTED
    lib = _lib.load()
    st = lib.dd_transpose(_lib.DD_U4, 16, 32, 1, 16, 32, 0, 1, None)
    assert st == _lib.DD_ERR_UNSUPPORTED


def test_adjoint_scratch_bytes():
    """dd_adjoint_scratch_bytes: the pattern adjoint's scratch by its formula
    (padded cotangent rows as float pairs, per-range results; no result
    buffer for one range at bin 1), 0 where the plan's adjoint is the gather,
    errors for bad arguments."""
    import ctypes
    lib = _lib.load()
    freqs = channel_freqs(1500.0, 2.6, 130)
    ranges = [(0.0, 25.6, 0.4, 1), (25.6, 51.2, 0.8, 2)]
    plan = dd.Plan(freqs, 1500.0, 64e-6, ranges, "f32", upload=False)
    n_samp = 6001
    info = plan.info(n_samp)
    assert info["adjoint_kernel"] == "pattern"
    got = ctypes.c_size_t(0)
    assert lib.dd_adjoint_scratch_bytes(plan.handle, n_samp, ctypes.byref(got)) == _lib.DD_OK
    r4 = lambda n: (n + 3) // 4 * 4
    u = [(n_samp - 1) // r[3] + 1 for r in ranges]
    pad_in = max(2 * nd * r4(uu + s) for nd, uu, s in zip(info["n_dm"], u, info["s_max"]))
    want = 4 * (pad_in + sum(130 * r4(uu) for uu in u))
    assert got.value == want
    one = dd.Plan(freqs, 1500.0, 64e-6, ranges[:1], "f32", upload=False)
    i1 = one.info(n_samp)
    assert lib.dd_adjoint_scratch_bytes(one.handle, n_samp, ctypes.byref(got)) == _lib.DD_OK
    assert got.value == 4 * 2 * i1["n_dm"][0] * r4(n_samp + i1["s_max"][0])
    wide = dd.Plan(channel_freqs(1500.0, 600.0, 17), 1500.0, 64e-6, [(0.0, 80.0, 0.4, 1)], "f32",
                   upload=False)
    assert wide.info(n_samp)["adjoint_kernel"] == "gather"
    assert lib.dd_adjoint_scratch_bytes(wide.handle, n_samp, ctypes.byref(got)) == _lib.DD_OK
    assert got.value == 0
    u8 = dd.Plan(freqs, 1500.0, 64e-6, ranges, "u8", upload=False)
    assert u8.info(n_samp)["adjoint_kernel"] is None
    assert lib.dd_adjoint_scratch_bytes(u8.handle, n_samp, ctypes.byref(got)) == \
        _lib.DD_ERR_UNSUPPORTED
    assert lib.dd_adjoint_scratch_bytes(plan.handle, 0, ctypes.byref(got)) == _lib.DD_ERR_SHAPE
    assert lib.dd_adjoint_scratch_bytes(plan.handle, n_samp, None) == _lib.DD_ERR_INVALID_ARG


def test_packed_tile_selection_and_scratch_bytes():
    """DD_TILE_PACKED serves uint8, 4-bit, uint16 and float32 ranges at bin 1
    and uint8 at bins 2, 4 and 8; it is never the automatic choice; the input
    scratch is n_chan x ceil4(n_samp / bin) words (32-bit; float32: 64-bit
    pairs) per distinct packed copy."""
    lib = _lib.load()
    paper = workloads.paper_u8()
    # The paper band and DM step on fewer channels and DMs (quick to plan).
    paper.n_chan, paper.ranges = 1024, [(0.0, 51.2, 0.1, 1)]
    need = ctypes.c_size_t(0)
    for dtype in ("u8", "u4", "u16"):
        plan = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, dtype,
                       upload=False)
        assert plan.info(paper.n_samp)["tile_dms"] == [_lib.DD_TILE_PATTERN], dtype
        assert lib.dd_plan_input_scratch_bytes(plan.handle, 1001, ctypes.byref(need)) == \
            _lib.DD_OK
        assert need.value == 0
        plan.set_tile(0, "packed")
        assert plan.info(paper.n_samp)["tile_dms"] == [_lib.DD_TILE_PACKED], dtype
        assert lib.dd_plan_input_scratch_bytes(plan.handle, 1001, ctypes.byref(need)) == \
            _lib.DD_OK
        assert need.value == paper.n_chan * 1004 * 4
    f32 = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, "f32", upload=False)
    assert f32.info(paper.n_samp)["tile_dms"] == [_lib.DD_TILE_PATTERN]
    f32.set_tile(0, "packed")
    assert f32.info(paper.n_samp)["tile_dms"] == [_lib.DD_TILE_PACKED]
    assert lib.dd_plan_input_scratch_bytes(f32.handle, 1001, ctypes.byref(need)) == _lib.DD_OK
    assert need.value == paper.n_chan * 1004 * 8
    # uint8 decimated by 2, 4 or 8: a packed copy of decimated pair words (one
    # per distinct bin); other bins and other dtypes at bin > 1 are refused.
    binned = dd.Plan(paper.freqs, paper.f_high, paper.t_samp,
                     [(0.0, 40.0, 0.2, 2), (40.0, 80.0, 0.4, 4), (80.0, 120.0, 0.8, 3)], "u8",
                     upload=False)
    binned.set_tile(0, "packed")
    binned.set_tile(1, "packed")
    with pytest.raises(dd.DDError):
        binned.set_tile(2, "packed")
    assert lib.dd_plan_input_scratch_bytes(binned.handle, 1001, ctypes.byref(need)) == _lib.DD_OK
    copy2 = paper.n_chan * ((1001 // 2 + 3) // 4 * 4) * 4
    copy4 = paper.n_chan * ((1001 // 4 + 3) // 4 * 4) * 4
    assert need.value == (copy2 + 255) // 256 * 256 + copy4
    u16b = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, [(0.0, 40.0, 0.2, 2)], "u16",
                   upload=False)
    with pytest.raises(dd.DDError):
        u16b.set_tile(0, "packed")
    plan = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, "u8", upload=False)
    assert lib.dd_plan_input_scratch_bytes(plan.handle, 0, ctypes.byref(need)) == \
        _lib.DD_ERR_SHAPE
    assert lib.dd_plan_input_scratch_bytes(plan.handle, 10, None) == _lib.DD_ERR_INVALID_ARG


def test_packed_copy_flags_and_ring_sizes():
    """The automatic pattern tile of uint8, 4-bit and uint16 input at bin 1 can
    run from a packed copy (float32's automatic tile, binned uint8 and offset
    tiles cannot); the full copies are n_chan x ceil4(n_samp) words and a ring
    of n segments holds two slots of about n_out / n + the largest delay words
    per channel (plus a time tile and alignment)."""
    paper = workloads.paper_u8()
    n_samp = paper.n_samp
    for dtype in ("u8", "u4", "u16"):
        plan = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, dtype,
                       upload=False)
        info = plan.info(n_samp)
        assert info["packed_copy"] == [True], dtype
        assert plan.input_scratch_bytes(n_samp) == 0  # nothing is required
        full = plan.packed_scratch_bytes(n_samp, 1)
        assert full == paper.n_chan * n_samp * 4
        n_out, s_max = info["n_out"][0], info["s_max"][0]
        ts = 2 * 32 * 23 if dtype != "u16" else 32 * 23  # samples per time tile
        prev = 2 * full  # two slots of half the outputs each exceed the full copy
        for n in (2, 4, 16, 64):
            ring = plan.packed_scratch_bytes(n_samp, n)
            lo = 2 * paper.n_chan * 4 * (n_out // n + s_max - ts)
            hi = 2 * paper.n_chan * 4 * (-(-n_out // n) + ts + s_max + 64) + 512
            assert lo <= ring <= hi, (dtype, n, lo, ring, hi)
            assert ring <= prev
            prev = ring
        assert plan.packed_scratch_bytes(n_samp, 16) < full / 4
    f32 = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, "f32", upload=False)
    assert f32.info(n_samp)["packed_copy"] == [False]
    assert f32.packed_scratch_bytes(n_samp, 16) == 0
    # Binned uint8 and an explicit pattern or offset tile: no packed copy (nor
    # a tile whose packed kernel's two staging buffers would not fit).
    multi = dd.Plan(paper.freqs, paper.f_high, paper.t_samp,
                    [(0.0, 40.0, 0.1, 1), (40.0, 80.0, 0.2, 2), (80.0, 120.0, 0.1, 1)], "u8",
                    upload=False)
    assert multi.info(n_samp)["packed_copy"] == [True, False, True]
    multi.set_tile(2, "pattern")
    assert multi.info(n_samp)["packed_copy"] == [True, False, False]
    multi.set_tile(2, 4)
    assert multi.info(n_samp)["packed_copy"] == [True, False, False]
    multi.set_tile(2, 0)
    assert multi.info(n_samp)["packed_copy"] == [True, False, True]
    # Two pair distances would need two copies: no ring, full copies only.
    mixed = dd.Plan(paper.freqs, paper.f_high, paper.t_samp,
                    [(0.0, 40.0, 0.1, 1), (40.0, 80.0, 0.1, 1)], "u8", upload=False)
    mixed.set_tile_shape(1, "packed", 15)  # H = 19: pair distance 608
    with pytest.raises(dd.DDError) as ei:
        mixed.packed_scratch_bytes(n_samp, 8)
    assert ei.value.status == _lib.DD_ERR_UNSUPPORTED
    assert mixed.packed_scratch_bytes(n_samp, 1) > 0


def test_workspace_holds_widening_slots():
    """Plans with uint8 or 4-bit pattern tiles reserve 320 widening slots of
    DMs-per-CTA x 32 H 64-bit words after their tables (slot flags uploaded,
    slots not); uint16 plans, whose 32-bit lanes never widen, none."""
    paper = workloads.paper_u8()
    slot = 4 * 16 * 32 * 23 * 8  # 4 DMs x 16 warps, H = 23, 8 bytes
    sizes = {}
    for dtype in ("u8", "u4", "u16"):
        plan = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, dtype,
                       upload=False)
        sizes[dtype] = plan.info(paper.n_samp)["workspace_bytes"]
    tables = sizes["u16"]  # same shape of tables, no slots
    for dtype in ("u8", "u4"):
        extra = sizes[dtype] - tables
        assert 320 * slot <= extra <= 320 * slot + 320 * 4 + 512, (dtype, extra)


def test_run_scratch_choice():
    """Plan.run's scratch for the packed copies: the ring of `segments`, the
    full copies for segments == 1 (and where the plan has no ring), none for
    segments == 0; a segment count outside [1, 256] is an error, not a silent
    fall back to the full copies."""
    pytest.importorskip("torch")
    freqs = channel_freqs(1500.0, 300.0, 64)
    n = 20000
    plan = dd.Plan(freqs, 1500.0, 64e-6, [(0.0, 6.4, 0.1, 1)], "u8", upload=False)
    assert plan.info(n)["packed_copy"] == [True]
    full = plan.packed_scratch_bytes(n, 1)
    ring = plan.packed_scratch_bytes(n, 8)
    assert 0 < ring < full
    assert plan._input_scratch(n, "cpu", 8).numel() == ring
    assert plan._input_scratch(n, "cpu", 1).numel() == full
    assert plan._input_scratch(n, "cpu", 0) is None
    with pytest.raises(dd.DDError) as err:
        plan._input_scratch(n, "cpu", 300)
    assert err.value.status == _lib.DD_ERR_INVALID_ARG
    # A binned packed copy has no ring: the full copy it needs anyway.
    binned = dd.Plan(freqs, 1500.0, 64e-6, [(0.0, 6.4, 0.1, 2)], "u8", upload=False)
    binned.set_tile(0, "packed")
    with pytest.raises(dd.DDError) as err:
        binned.packed_scratch_bytes(n, 8)
    assert err.value.status == _lib.DD_ERR_UNSUPPORTED
    assert binned._input_scratch(n, "cpu", 8).numel() == binned.input_scratch_bytes(n) > 0


def test_stream_snapshot_refuses_queued_chunks():
    """A snapshot holds the overlap and the chunks already launched; a chunk
    still queued for the beam would be lost between the two servers, so
    snapshot() refuses until it has run (host logic, no device call)."""
    torch = pytest.importorskip("torch")
    from paper_2311_05341_gb300 import stream as dds
    server = dds.StreamServer(4096, 1 << 30)
    server.submit(3, torch.zeros((8, 4096), dtype=torch.uint8))
    with pytest.raises(RuntimeError, match="queued chunks"):
        server.snapshot(3)


def test_autotune_cache_keeps_restricted_tuners_apart(tmp_path):
    """A tuner restricted to some tiles never takes a cached choice made
    without that restriction (or the other way round): the cache key names
    the restriction.  A one-candidate tuner times nothing, so this runs on
    the CPU."""
    pytest.importorskip("torch")
    from paper_2311_05341_gb300 import batch
    freqs = channel_freqs(1500.0, 300.0, 64)
    plan = dd.Plan(freqs, 1500.0, 64e-6, [(0.0, 6.4, 0.1, 1)], "u8", upload=False)
    n = 20000
    cache = tmp_path / "tune.json"
    free_key = batch.plan_signature(plan, n) + "|packed"
    cache.write_text(json.dumps({free_key: [["pattern", 0]]}))
    restricted = batch.Autotuner(shapes=[4], cache_path=str(cache))
    assert restricted.choose(plan, n, None, None) == [(4, -1)]
    assert plan.info(n)["tile_dms"] == [4]
    stored = json.loads(cache.read_text())
    assert stored[free_key] == [["pattern", 0]] and len(stored) == 2
    free = batch.Autotuner(cache_path=str(cache))
    assert free.choose(plan, n, None, None) == [("pattern", 0)]
    assert plan.info(n)["tile_dms"] == [_lib.DD_TILE_PATTERN]
