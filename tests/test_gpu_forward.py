"""Parity of the CUDA forward transform (through the C ABI) with the oracle.

Integer inputs: bit-exact.  Float inputs: |err| <= 1e-5 * sum_c |X| per
output against the FP64 oracle.  Small cases compare every output (several
CTA tiles, ragged tails, odd channel counts, bins, several ranges); the
paper-scale workloads compare sampled rows and windows plus properties that
hold at any size.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from paper_2311_05341_gb300._lib import DD_TILE_PACKED as TILE_PACKED
from paper_2311_05341_gb300._lib import DD_TILE_PATTERN as TILE_PATTERN
from synth import workloads, channel_freqs, filterbank

from gpu_util import assert_float_parity, oracle_input

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def padded_device(x_np):
    """Copy to the device with the row stride rounded up to 16 bytes."""
    per = 16 // x_np.itemsize
    stride = (x_np.shape[1] + per - 1) // per * per
    x = torch.zeros((x_np.shape[0], stride), dtype=getattr(torch, str(x_np.dtype)),
                    device="cuda")
    x[:, : x_np.shape[1]] = torch.from_numpy(x_np).cuda()
    return x


def gpu_planes(beam_like, x_np, ranges=None, dtype=None):
    b = beam_like
    plan = dd.Plan(b.freqs, b.f_high, b.t_samp, ranges or b.ranges, dtype or b.dtype)
    planes = plan.run(padded_device(x_np), n_samp=x_np.shape[1])
    torch.cuda.synchronize()
    return [p.cpu().numpy() for p in planes]


def test_tiny_u8_full_plane():
    beam = workloads.tiny_u8()
    x, tables, n_dm, n_out = oracle_input(beam)
    ref = oracle.forward(x, beam.freqs, beam.f_high, beam.t_samp, beam.ranges)
    got = gpu_planes(beam, x)
    assert got[0].dtype == np.int32
    np.testing.assert_array_equal(got[0], ref[0])
    # The injected DM = 30 pulse peaks at its trial.
    d, t0 = 60, 3000
    assert np.argmax(got[0][:, t0:t0 + 4].sum(1)) == d


class _Beam:
    def __init__(self, freqs, f_high, t_samp, ranges, dtype, n_samp):
        self.freqs, self.f_high, self.t_samp = freqs, f_high, t_samp
        self.ranges, self.dtype, self.n_samp = ranges, dtype, n_samp


def _random_case(seed):
    rng = np.random.default_rng(seed)
    n_chan = int(rng.choice([1, 3, 31, 33, 64, 130, 257]))
    f_high = float(rng.uniform(300, 1700))
    bw = float(rng.uniform(0.05, 0.4)) * f_high
    freqs = channel_freqs(f_high, bw, n_chan)
    t_samp = float(rng.choice([64e-6, 128e-6, 327.68e-6, 1e-3]))
    dtype = ["u8", "u16", "f32"][seed % 3]
    ranges, lo = [], 0.0
    for _ in range(int(rng.integers(1, 4))):
        step = float(rng.choice([0.05, 0.1, 0.5, 2.0]))
        n = int(rng.integers(1, 70))
        ranges.append((lo, lo + n * step, step, int(rng.choice([1, 2, 3, 4, 8]))))
        lo += n * step
    smax = 0
    for r in ranges:
        s, _ = oracle.extent(freqs, f_high, t_samp, r, 10 ** 9)
        smax = max(smax, (s + 1) * r[3])
    n_samp = int(smax + rng.integers(1, 3000))
    return _Beam(freqs, f_high, t_samp, ranges, dtype, n_samp), rng


@pytest.mark.parametrize("seed", range(18))
def test_random_cases_full_planes(seed):
    b, rng = _random_case(seed)
    npdt = {"u8": np.uint8, "u16": np.uint16, "f32": np.float32}[b.dtype]
    mean, sd = {"u8": (128, 40), "u16": (32768, 9000), "f32": (0.0, 1.0)}[b.dtype]
    x = filterbank(npdt, len(b.freqs), b.n_samp, 7000 + seed, mean, sd)
    ref = oracle.forward(x, b.freqs, b.f_high, b.t_samp, b.ranges)
    got = gpu_planes(b, x)
    assert len(got) == len(ref)
    for r, (g, o) in enumerate(zip(got, ref)):
        assert g.shape == o.shape
        if b.dtype == "f32":
            ab = oracle.forward(x, b.freqs, b.f_high, b.t_samp, b.ranges, take_abs=True)[r]
            assert_float_parity(g, o, ab, f"range {r}")
        else:
            np.testing.assert_array_equal(g, o, err_msg=f"range {r}")


def _tiled_case(seed, dtype="u8"):
    """Plans on the register-tiled kernel: shallow DM steps, ragged sizes."""
    rng = np.random.default_rng(seed)
    n_chan = int(rng.choice([1, 15, 17, 255, 256, 257, 300, 513]))
    f_high = float(rng.uniform(800, 1700))
    freqs = channel_freqs(f_high, float(rng.uniform(0.05, 0.25)) * f_high, n_chan)
    t_samp = 64e-6
    k_low = oracle.delay_coeff(freqs[-1], f_high) / t_samp  # samples per unit DM
    step = float(rng.uniform(0.2, 1.7)) / max(k_low, 1e-9)  # <= 1.7 samples per step
    n_dm = int(rng.choice([1, 7, 63, 64, 65, 130]))
    lo = float(rng.uniform(0, 50)) * step
    r = (lo, lo + n_dm * step, step, 1)
    s_max, _ = oracle.extent(freqs, f_high, t_samp, r, 10 ** 9)
    n_samp = int(s_max + rng.choice([1, 639, 640, 1279, 1280, 1281, 5000]))
    return _Beam(freqs, f_high, t_samp, [r], dtype, n_samp), rng


_NOISE = {"u8": (np.uint8, 200, 80), "u16": (np.uint16, 40000, 12000), "f32": (np.float32, 0.0, 1.0)}


@pytest.mark.parametrize("dtype,seed", [("u8", s) for s in range(16)] +
                         [("u16", s) for s in range(8)] + [("f32", s) for s in range(8)])
def test_tiled_full_planes_every_shape(dtype, seed):
    b, rng = _tiled_case(seed, dtype)
    npdt, mean, sd = _NOISE[dtype]
    # uint8 values up to 255 in every channel exercise the 16-bit lane bound.
    x = filterbank(npdt, len(b.freqs), b.n_samp, 8000 + seed, mean, sd)
    ref = oracle.forward(x, b.freqs, b.f_high, b.t_samp, b.ranges)
    ref_abs = oracle.forward(x, b.freqs, b.f_high, b.t_samp, b.ranges, take_abs=True)
    xd = padded_device(x)
    # Steps of at most 1.7 samples keep every per-DM increment in {0, 1, 2}:
    # the pattern tile serves all these plans too (uint8 and float32: also on
    # the packed copy).
    tiles = (8, 6, 4, 2, 1, "pattern") + (("packed",) if dtype in ("u8", "f32") else ())
    for dms in tiles:
        plan = dd.Plan(b.freqs, b.f_high, b.t_samp, b.ranges, dtype)
        plan.set_tile(0, dms)
        info = plan.info(b.n_samp)
        code = {"pattern": TILE_PATTERN, "packed": TILE_PACKED}.get(dms, dms)
        assert info["kernel"] == ["tiled"] and info["tile_dms"] == [code]
        got = plan.run(xd, n_samp=b.n_samp)[0].cpu().numpy()
        if dtype == "f32":
            assert_float_parity(got, ref[0], ref_abs[0], f"tile {dms}")
        else:
            np.testing.assert_array_equal(got, ref[0], err_msg=f"tile {dms}")


@pytest.mark.parametrize("dtype,seed", [("u8", s) for s in range(6)] +
                         [("u16", s) for s in range(4)] + [("f32", s) for s in range(4)])
def test_pattern_steep_plans(dtype, seed):
    """Pattern tile on plans with 1.7 to 3.9 samples of delay per DM step (base
    increments 1 to 3), against the oracle and the 1-DM offset tile."""
    rng = np.random.default_rng(7000 + seed)
    n_chan = int(rng.choice([15, 96, 257, 300]))
    f_high = float(rng.uniform(800, 1700))
    freqs = channel_freqs(f_high, float(rng.uniform(0.05, 0.25)) * f_high, n_chan)
    k_low = oracle.delay_coeff(freqs[-1], f_high) / 64e-6
    step = float(rng.uniform(1.7, 3.9)) / k_low
    n_dm = int(rng.choice([5, 64, 67, 129]))
    r = (float(rng.uniform(0, 20)) * step, 0.0, step, 1)
    r = (r[0], r[0] + n_dm * step, step, 1)
    s_max, _ = oracle.extent(freqs, f_high, 64e-6, r, 10 ** 9)
    n_samp = int(s_max + rng.choice([1, 735, 1472, 3001]))
    npdt, mean, sd = _NOISE[dtype]
    x = filterbank(npdt, n_chan, n_samp, 7100 + seed, mean, sd)
    ref = oracle.forward(x, freqs, f_high, 64e-6, [r])[0]
    ref_abs = oracle.forward(x, freqs, f_high, 64e-6, [r], take_abs=True)[0]
    xd = padded_device(x)
    for tile in ("pattern", 1) + (("packed",) if dtype in ("u8", "f32") else ()):
        plan = dd.Plan(freqs, f_high, 64e-6, [r], dtype)
        plan.set_tile(0, tile)
        got = plan.run(xd, n_samp=n_samp)[0].cpu().numpy()
        if dtype == "f32":
            assert_float_parity(got, ref, ref_abs, f"tile {tile}")
        else:
            np.testing.assert_array_equal(got, ref, err_msg=f"tile {tile}")


@pytest.mark.parametrize("dtype,b", [("u8", 2), ("u8", 4), ("u8", 8), ("u16", 2), ("u16", 4),
                                     ("f32", 2)])
def test_tiled_decimation_every_shape(dtype, b):
    """Time binning fused into the tiled kernel's staging, every feasible shape."""
    rng = np.random.default_rng(900 + b)
    n_chan = 77
    freqs = channel_freqs(1400.0, 300.0, n_chan)
    r = (2.0, 2.0 + 33 * 0.05 * b, 0.05 * b, b)
    s_max, _ = oracle.extent(freqs, 1400.0, 64e-6, r, 10 ** 9)
    n_samp = int((s_max + 700) * b + rng.integers(0, b))  # ragged tail of the bin
    npdt, mean, sd = _NOISE[dtype]
    x = filterbank(npdt, n_chan, n_samp, 9000 + b, mean, sd)
    ref = oracle.forward(x, freqs, 1400.0, 64e-6, [r])[0]
    ref_abs = oracle.forward(x, freqs, 1400.0, 64e-6, [r], take_abs=True)[0]
    xd = padded_device(x)
    ran = 0
    for dms in (8, 6, 4, 2, 1, "pattern"):
        plan = dd.Plan(freqs, 1400.0, 64e-6, [r], dtype)
        try:
            plan.set_tile(0, dms)
        except dd.DDError:
            continue  # this shape's staging does not fit shared memory at this bin
        ran += 1
        got = plan.run(xd, n_samp=n_samp)[0].cpu().numpy()
        if dtype == "f32":
            assert_float_parity(got, ref, ref_abs, f"tile {dms}")
        else:
            np.testing.assert_array_equal(got, ref, err_msg=f"tile {dms}")
    assert ran >= 1


def test_u8_tiled_saturated_input():
    """All samples 255: every 16-bit lane reaches 255 * 256 before widening."""
    freqs = channel_freqs(1670.0, 320.0, 1000)
    r = (0.0, 12.8, 0.1, 1)
    s_max, _ = oracle.extent(freqs, 1670.0, 64e-6, r, 10 ** 9)
    n_samp = s_max + 3000
    x = np.full((1000, n_samp), 255, np.uint8)
    b = _Beam(freqs, 1670.0, 64e-6, [r], "u8", n_samp)
    got = gpu_planes(b, x)[0]
    assert np.all(got == 255 * 1000)


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_minimal_output_length(dtype):
    """n_samp = S_max + 1: exactly one output sample per trial."""
    freqs = channel_freqs(1400.0, 300.0, 40)
    r = (0.0, 25.0, 0.5, 1)
    s_max, _ = oracle.extent(freqs, 1400.0, 64e-6, r, 10 ** 6)
    n_samp = s_max + 1
    npdt = {"u8": np.uint8, "u16": np.uint16, "f32": np.float32}[dtype]
    x = filterbank(npdt, 40, n_samp, 11, 100, 30)
    b = _Beam(freqs, 1400.0, 64e-6, [r], dtype, n_samp)
    ref = oracle.forward(x, freqs, 1400.0, 64e-6, [r])[0]
    got = gpu_planes(b, x)[0]
    assert got.shape == (50, 1)
    if dtype == "f32":
        ab = oracle.forward(x, freqs, 1400.0, 64e-6, [r], take_abs=True)[0]
        assert_float_parity(got, ref, ab)
    else:
        np.testing.assert_array_equal(got, ref)


def test_padded_row_stride_ignores_padding():
    freqs = channel_freqs(1400.0, 300.0, 48)
    r = (0.0, 30.0, 0.25, 2)
    n_samp, stride = 3001, 3072
    x = filterbank(np.uint8, 48, n_samp, 5, 128, 16, row_stride=stride)
    x[:, n_samp:] = 255  # garbage the transform must never read
    ref = oracle.forward(np.ascontiguousarray(x[:, :n_samp]), freqs, 1400.0, 64e-6, [r])[0]
    plan = dd.Plan(freqs, 1400.0, 64e-6, [r], "u8")
    xt = torch.from_numpy(x).cuda()
    got = plan.run(xt, n_samp=n_samp)[0].cpu().numpy()
    np.testing.assert_array_equal(got, ref)


def test_too_short_input_raises():
    freqs = channel_freqs(1400.0, 300.0, 16)
    plan = dd.Plan(freqs, 1400.0, 64e-6, [(0.0, 500.0, 1.0, 1)], "u8")
    x = torch.zeros((16, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(dd.DDError) as ei:
        plan.run(x)
    assert ei.value.status == 3  # DD_ERR_SHAPE


# Oracle rows of the paper-scale workloads, computed once per workload and
# shared by the tile variants that run the same input.
_PAPER_REF = {}


def _paper_reference(beam, x, n_dm, n_out, pulse_rows):
    """Every 16th DM row (plus the last and the pulse rows) at full length, and
    96 random rows on three windows (the first, a random and the ragged last
    tile), from the oracle."""
    if beam.name not in _PAPER_REF:
        r = 0
        rows_full = sorted(set(range(0, n_dm[r], 16)) | {n_dm[r] - 1} | set(pulse_rows))
        full = oracle.forward_rows(x, beam.freqs, beam.f_high, beam.t_samp, beam.ranges[r],
                                   rows_full)
        rng = np.random.default_rng(9)
        rows = rng.integers(0, n_dm[r], 96)
        wins = []
        for t_lo in [0, int(rng.integers(0, n_out[r] - 2048)), n_out[r] - 1500]:
            t_hi = min(t_lo + 2048, n_out[r])
            wins.append((t_lo, t_hi, oracle.forward_rows(x, beam.freqs, beam.f_high, beam.t_samp,
                                                         beam.ranges[r], rows, t_lo, t_hi)))
        _PAPER_REF.clear()  # one workload's rows at a time (host memory)
        _PAPER_REF[beam.name] = (rows_full, full, rows, wins)
    return _PAPER_REF[beam.name]


def _sampled_parity(beam, x, planes_gpu, n_dm, n_out, pulse_rows):
    """Compare sampled full rows and windows of a large plane with the oracle."""
    rows_full, full, rows, wins = _paper_reference(beam, x, n_dm, n_out, pulse_rows)
    got = planes_gpu[0][torch.tensor(rows_full, device="cuda")].cpu().numpy()
    np.testing.assert_array_equal(got, full)
    for t_lo, t_hi, o in wins:
        g = planes_gpu[0][torch.tensor(rows, device="cuda"), t_lo:t_hi].cpu().numpy()
        np.testing.assert_array_equal(g, o)


# (workload, tile, segments): the automatic tile from the packed ring (the
# default of Plan.run) and unpacking the input itself (no scratch), the
# explicit pattern tile, the packed tile from its full copy, an offset tile.
@pytest.mark.parametrize("make,tile,segments",
                         [(workloads.paper_u8, 0, 8), (workloads.paper_u8, 0, 0),
                          (workloads.paper_u8, "pattern", 16), (workloads.paper_u8, "packed", 1),
                          (workloads.paper_u8, 6, 16), (workloads.paper_u16, 0, 16)],
                         ids=["paper_u8_ring", "paper_u8_unpacked", "paper_u8_pattern",
                              "paper_u8_packed_full", "paper_u8_offset6", "paper_u16_ring"])
def test_paper_scale_sampled(make, tile, segments):
    beam = make()
    x, tables, n_dm, n_out = oracle_input(beam)
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, beam.dtype)
    if tile:
        plan.set_tile(0, tile)
    xt = torch.from_numpy(x).cuda()
    planes = plan.run(xt, segments=segments)
    torch.cuda.synchronize()
    assert planes[0].shape == (n_dm[0], n_out[0])
    pulses = workloads.resolve_pulses(beam, n_dm, n_out)
    _sampled_parity(beam, x, planes, n_dm, n_out, [p[1] for p in pulses])
    # DM 0 is the plain channel sum at any size.
    dm0 = xt.to(torch.int64).sum(0)[: n_out[0]].to(torch.int32)
    assert torch.equal(planes[0][0], dm0)
    # Every injected pulse peaks at its own trial among its neighbours.
    for _, d, t0, w in pulses:
        lo, hi = max(d - 20, 0), min(d + 21, n_dm[0])
        seg = planes[0][lo:hi, t0:t0 + w].to(torch.int64).sum(1)
        assert int(torch.argmax(seg)) + lo == d


@pytest.mark.slow
@pytest.mark.skipif(os.environ.get("DD_FULL_PLANE") != "1",
                    reason="the full paper-scale comparison takes minutes of oracle time; "
                           "set DD_FULL_PLANE=1 to run it")
def test_paper_u8_full_plane():
    """Every output of the paper-scale uint8 plane (4096 x 257097) against the
    oracle: the automatic tile from the packed ring (what the benchmark runs)
    and unpacking the input itself, and the packed tile from its full copy."""
    beam = workloads.paper_u8()
    x, _, n_dm, n_out = oracle_input(beam)
    xt = torch.from_numpy(x).cuda()
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, beam.dtype)
    planes = {"ring": plan.run(xt, segments=8)[0], "unpacked": plan.run(xt, segments=0)[0]}
    plan.set_tile(0, "packed")
    planes["packed full copy"] = plan.run(xt, segments=1)[0]
    torch.cuda.synchronize()
    for p in planes.values():
        assert p.shape == (n_dm[0], n_out[0])
    block = 256
    for d0 in range(0, n_dm[0], block):
        rows = list(range(d0, min(d0 + block, n_dm[0])))
        ref = oracle.forward_rows(x, beam.freqs, beam.f_high, beam.t_samp, beam.ranges[0], rows)
        for name, p in planes.items():
            np.testing.assert_array_equal(p[d0:d0 + len(rows)].cpu().numpy(), ref,
                                          err_msg=f"{name}, rows {d0}..")
