"""4-bit packed input (two samples per byte, the earlier in the low nibble):
pattern tiles with fused binning, the generic kernel for steep plans, the
widening bound, the host path, and a paper-scale plan on sampled rows -- all
bit-exact against the oracle's 4-bit path."""
import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from paper_2311_05341_gb300._lib import DD_TILE_PATTERN as TILE_PATTERN
from synth import channel_freqs, filterbank4, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _packed(n_chan, n_samp, seed, mean=8.0, sd=4.0):
    """Packed rows padded to a 16-byte multiple (32 samples)."""
    row_bytes = (n_samp + 31) // 32 * 16
    return filterbank4(n_chan, n_samp, seed, mean, sd, row_bytes=row_bytes)


def _check(freqs, f_ref, t_samp, ranges, n_samp, data, want_kernel=None):
    plan = dd.Plan(freqs, f_ref, t_samp, ranges, "u4")
    info = plan.info(n_samp)
    if want_kernel:
        assert info["kernel"] == want_kernel
    planes = plan.run(torch.from_numpy(data).cuda(), n_samp=n_samp)
    ref = oracle.forward(oracle.Packed4(data, n_samp), freqs, f_ref, t_samp, ranges)
    for r, (g, o) in enumerate(zip(planes, ref)):
        np.testing.assert_array_equal(g.cpu().numpy(), o, err_msg=f"range {r}")
    return plan, info


@pytest.mark.parametrize("seed", range(8))
def test_u4_pattern_random_plans(seed):
    rng = np.random.default_rng(6000 + seed)
    n_chan = int(rng.choice([1, 17, 96, 257, 300]))
    f_high = float(rng.uniform(800, 1700))
    freqs = channel_freqs(f_high, float(rng.uniform(0.05, 0.25)) * f_high, n_chan)
    k_low = oracle.delay_coeff(freqs[-1], f_high) / 64e-6
    step = float(rng.uniform(0.3, 3.5)) / k_low
    n_dm = int(rng.choice([3, 64, 65, 130]))
    lo = float(rng.uniform(0, 30)) * step
    r = (lo, lo + n_dm * step, step, 1)
    s_max, _ = oracle.extent(freqs, f_high, 64e-6, r, 10 ** 9)
    n_samp = int(s_max + rng.choice([1, 1471, 1472, 2945, 6000]))
    data = _packed(n_chan, n_samp, 6100 + seed)
    plan, info = _check(freqs, f_high, 64e-6, [r], n_samp, data, ["tiled"])
    assert info["tile_dms"] == [TILE_PATTERN]


@pytest.mark.parametrize("b", [2, 4, 8, 16])
def test_u4_binned_ranges(b):
    freqs = channel_freqs(1400.0, 300.0, 77)
    r = (2.0, 2.0 + 40 * 0.05 * b, 0.05 * b, b)
    s_max, _ = oracle.extent(freqs, 1400.0, 64e-6, r, 10 ** 9)
    n_samp = (s_max + 900) * b + 3  # a ragged tail of the bin
    _check(freqs, 1400.0, 64e-6, [r], n_samp, _packed(77, n_samp, 6200 + b), ["tiled"])


def test_u4_steep_plan_generic_kernel():
    """12 samples of delay per DM step: outside the pattern tile's increments."""
    freqs = channel_freqs(400.0, 100.0, 64)
    k_low = oracle.delay_coeff(freqs[-1], 400.0) / 64e-6
    step = 12.0 / k_low
    r = (0.0, 40 * step, step, 1)
    s_max, _ = oracle.extent(freqs, 400.0, 64e-6, r, 10 ** 9)
    n_samp = s_max + 3001
    _check(freqs, 400.0, 64e-6, [r], n_samp, _packed(64, n_samp, 6300), ["generic"])


def test_u4_saturated_widening():
    """All samples 15 over 5000 channels: the 16-bit lanes are widened every
    4369 channels (15 * 4369 = 65535)."""
    freqs = channel_freqs(1670.0, 320.0, 5000)
    r = (0.0, 6.4, 0.1, 1)
    s_max, _ = oracle.extent(freqs, 1670.0, 64e-6, r, 10 ** 9)
    n_samp = s_max + 4000
    row_bytes = (n_samp + 31) // 32 * 16
    data = np.full((5000, row_bytes), 0xFF, np.uint8)
    plan = dd.Plan(freqs, 1670.0, 64e-6, [r], "u4")
    got = plan.run(torch.from_numpy(data).cuda(), n_samp=n_samp)[0]
    assert bool((got == 15 * 5000).all())


def test_u4_host_path_equals_device_path():
    freqs = channel_freqs(1500.0, 300.0, 40)
    ranges = [(0.0, 10.0, 0.1, 1), (10.0, 30.0, 0.4, 4)]
    n_samp = 30001
    data = _packed(40, n_samp, 6400)
    plan = dd.Plan(freqs, 1500.0, 64e-6, ranges, "u4")
    info = plan.info(n_samp)
    h_in = torch.from_numpy(data).pin_memory()
    h_out = torch.full((info["out_elems"],), -1, dtype=torch.int32).pin_memory()
    d_in = torch.empty_like(h_in, device="cuda")
    d_out = plan.empty_output(n_samp)
    plan.run_host(h_in, h_out, d_in, d_out, n_samp=n_samp)
    torch.cuda.synchronize()
    ref = torch.cat([p.reshape(-1) for p in plan.run(h_in.cuda(), n_samp=n_samp)]).cpu()
    assert torch.equal(h_out, ref)


def test_u4_paper_scale_sampled():
    """8192 channels x 262144 samples (1 GB packed), 4096 DMs: every 16th DM
    row at full length, on the plain pattern tile and on the packed tile."""
    beam = workloads.paper_u8()
    n_samp = beam.n_samp
    data = _packed(beam.n_chan, n_samp, 6500)
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, "u4")
    assert plan.info(n_samp)["tile_dms"] == [TILE_PATTERN]
    xd = torch.from_numpy(data).cuda()
    plane = plan.run(xd, n_samp=n_samp)[0]
    plan.set_tile(0, "packed")
    plane_packed = plan.run(xd, n_samp=n_samp)[0]
    torch.cuda.synchronize()
    x = oracle.Packed4(data, n_samp)
    n_dm = plane.shape[0]
    rows = sorted(set(range(0, n_dm, 16)) | {n_dm - 1, 1, 3333})
    ref = oracle.forward_rows(x, beam.freqs, beam.f_high, beam.t_samp, beam.ranges[0], rows)
    idx = torch.tensor(rows, device="cuda")
    np.testing.assert_array_equal(plane[idx].cpu().numpy(), ref)
    np.testing.assert_array_equal(plane_packed[idx].cpu().numpy(), ref)


@pytest.mark.parametrize("seed", range(6))
def test_u4_packed_tile(seed):
    """4-bit input through the packed tile (the same packed words, nibbles
    zero-extended; widened every 65535 / 15 channels), alone and beside a
    binned range, against the oracle; saturated samples (15) on 4500
    channels cross a widening."""
    from paper_2311_05341_gb300._lib import DD_TILE_PACKED
    rng = np.random.default_rng(6300 + seed)
    n_chan = int(rng.choice([1, 17, 96, 257, 4500 if seed == 5 else 300]))
    f_high = float(rng.uniform(800, 1700))
    freqs = channel_freqs(f_high, float(rng.uniform(0.05, 0.25)) * f_high, n_chan)
    k_low = oracle.delay_coeff(freqs[-1], f_high) / 64e-6
    step = float(rng.uniform(0.3, 2.9)) / k_low
    n_dm = int(rng.choice([3, 64, 65, 130]))
    ranges = [(0.0, n_dm * step, step, 1)]
    if seed % 2:
        ranges.append((n_dm * step, 2 * n_dm * step, 2 * step, 4))
    s_max = max((oracle.extent(freqs, f_high, 64e-6, r, 10 ** 9)[0] + 1) * r[3] for r in ranges)
    n_samp = int(s_max + rng.choice([1, 735, 1472, 2945]))
    data = _packed(n_chan, n_samp, 6400 + seed, mean=15.0 if seed == 5 else 8.0,
                   sd=0.0 if seed == 5 else 4.0)
    plan = dd.Plan(freqs, f_high, 64e-6, ranges, "u4")
    plan.set_tile(0, "packed")
    assert plan.info(n_samp)["tile_dms"][0] == DD_TILE_PACKED
    planes = plan.run(torch.from_numpy(data).cuda(), n_samp=n_samp)
    ref = oracle.forward(oracle.Packed4(data, n_samp), freqs, f_high, 64e-6, ranges)
    for r, (g, o) in enumerate(zip(planes, ref)):
        np.testing.assert_array_equal(g.cpu().numpy(), o, err_msg=f"range {r}")
