"""The pattern tile on a packed copy of uint8 input (DD_TILE_PACKED): the copy
written by dd_run_scratch, bit-exact outputs against the oracle, input
padding never read, and the calls that refuse such plans."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from paper_2311_05341_gb300 import _lib
from synth import channel_freqs, filterbank

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _plan(freqs, f_high, ranges, tiles):
    plan = dd.Plan(freqs, f_high, 64e-6, ranges, "u8")
    for r, t in enumerate(tiles):
        plan.set_tile(r, t)
    return plan


@pytest.mark.parametrize("segments", [1, 16])
@pytest.mark.parametrize("seed", range(8))
def test_packed_random_plans(seed, segments):
    """Ragged channel counts, DM counts and lengths (the last packed words of
    a row pair a sample with zeros past n_samp), mixed with a plain range."""
    rng = np.random.default_rng(5200 + seed)
    n_chan = int(rng.choice([1, 17, 64, 257, 300]))
    f_high = float(rng.uniform(900, 1700))
    freqs = channel_freqs(f_high, float(rng.uniform(0.05, 0.25)) * f_high, n_chan)
    k_low = oracle.delay_coeff(freqs[-1], f_high) / 64e-6
    step = float(rng.uniform(0.2, 1.9)) / k_low
    n_dm = int(rng.choice([1, 7, 64, 65, 130]))
    ranges = [(0.0, n_dm * step, step, 1)]
    tiles = ["packed"]
    if seed % 2:
        ranges.append((n_dm * step, 2 * n_dm * step, 2 * step, 2))
        tiles.append(0)
    s_max = max((oracle.extent(freqs, f_high, 64e-6, r, 10 ** 9)[0] + 1) * r[3] for r in ranges)
    n_samp = int(s_max + rng.choice([1, 735, 736, 737, 1472, 3001]))
    stride = (n_samp + 15) // 16 * 16
    x = filterbank(np.uint8, n_chan, n_samp, 5300 + seed, 200, 80, row_stride=stride)
    x[:, n_samp:] = 255  # padding the transform must not read
    ref = oracle.forward(np.ascontiguousarray(x[:, :n_samp]), freqs, f_high, 64e-6, ranges)
    plan = _plan(freqs, f_high, ranges, tiles)
    assert plan.info(n_samp)["tile_dms"][0] == _lib.DD_TILE_PACKED
    # The full copy, or the ring of 16 time segments.
    got = plan.run(torch.from_numpy(x).cuda(), n_samp=n_samp, segments=segments)
    for r, (g, o) in enumerate(zip(got, ref)):
        np.testing.assert_array_equal(g.cpu().numpy(), o, err_msg=f"range {r}")


def test_packed_saturated_input():
    """Every sample 255: each 16-bit lane reaches 255 x 256 before widening."""
    freqs = channel_freqs(1670.0, 320.0, 1000)
    r = [(0.0, 12.8, 0.1, 1)]
    s_max = oracle.extent(freqs, 1670.0, 64e-6, r[0], 10 ** 9)[0]
    n_samp = s_max + 3000
    x = np.full((1000, (n_samp + 15) // 16 * 16), 255, np.uint8)
    plan = _plan(freqs, 1670.0, r, ["packed"])
    got = plan.run(torch.from_numpy(x).cuda(), n_samp=n_samp)[0]
    assert bool(torch.all(got == 255 * 1000))


def test_packed_api_refusals_and_scratch():
    freqs = channel_freqs(1500.0, 300.0, 64)
    r = [(0.0, 6.4, 0.1, 1)]
    plan = _plan(freqs, 1500.0, r, ["packed"])
    n_samp = 4000
    lib = _lib.load()
    need = ctypes.c_size_t(0)
    assert lib.dd_plan_input_scratch_bytes(plan.handle, n_samp, ctypes.byref(need)) == _lib.DD_OK
    assert need.value == 64 * 4000 * 4
    x = torch.zeros((64, 4000), dtype=torch.uint8, device="cuda")
    out = plan.empty_output(n_samp)
    # dd_run cannot make the packed copy; too little scratch is refused.
    assert lib.dd_run(plan.handle, x.data_ptr(), 4000, n_samp, out.data_ptr(), None) == \
        _lib.DD_ERR_UNSUPPORTED
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    assert lib.dd_run_scratch(plan.handle, x.data_ptr(), 4000, n_samp, out.data_ptr(),
                              small.data_ptr(), 16, None) == _lib.DD_ERR_BUDGET
    # The host pipeline without scratch refuses such plans.
    h_in = torch.zeros((64, 4000), dtype=torch.uint8).pin_memory()
    h_out = torch.empty(plan.info(n_samp)["out_elems"], dtype=torch.int32).pin_memory()
    assert lib.dd_run_host(plan.handle, h_in.data_ptr(), 4000, n_samp, h_out.data_ptr(),
                           x.data_ptr(), out.data_ptr(), None) == _lib.DD_ERR_UNSUPPORTED
    plain = dd.Plan(freqs, 1500.0, 64e-6, r, "u8", upload=False)
    assert lib.dd_plan_input_scratch_bytes(plain.handle, n_samp, ctypes.byref(need)) == _lib.DD_OK
    assert need.value == 0


def test_packed_host_pipeline():
    """dd_run_host_scratch: segments packed 736 samples behind the copies; the
    output equals dd_run's and the oracle's, with a plain range beside."""
    n_chan = 300
    freqs = channel_freqs(1500.0, 300.0, n_chan)
    k_low = oracle.delay_coeff(freqs[-1], 1500.0) / 64e-6
    step = 1.1 / k_low
    ranges = [(0.0, 96 * step, step, 1), (96 * step, 192 * step, 2 * step, 2)]
    s_max = max((oracle.extent(freqs, 1500.0, 64e-6, r, 10 ** 9)[0] + 1) * r[3] for r in ranges)
    n_samp = int(s_max + 50001)
    stride = (n_samp + 15) // 16 * 16
    x = filterbank(np.uint8, n_chan, n_samp, 91, 128, 40, row_stride=stride)
    plan = _plan(freqs, 1500.0, ranges, ["packed", 0])
    info = plan.info(n_samp)
    assert info["tile_dms"][0] == _lib.DD_TILE_PACKED
    h_in = torch.from_numpy(x).pin_memory()
    h_out = torch.full((info["out_elems"],), -5, dtype=torch.int32).pin_memory()
    d_in = torch.empty_like(h_in, device="cuda")
    plan.run_host(h_in, h_out, d_in, plan.empty_output(n_samp), n_samp=n_samp)
    torch.cuda.synchronize()
    dev = plan.run(h_in.cuda(), n_samp=n_samp)
    flat = torch.cat([p.reshape(-1) for p in dev]).cpu()
    assert torch.equal(h_out, flat)
    ref = oracle.forward(np.ascontiguousarray(x[:, :n_samp]), freqs, 1500.0, 64e-6, ranges)
    for r, (g, o) in enumerate(zip(plan.split(h_out, n_samp), ref)):
        np.testing.assert_array_equal(g.numpy(), o, err_msg=f"range {r}")


@pytest.mark.parametrize("seed", range(4))
def test_packed_uint16(seed):
    """uint16 through the packed tile (the input widened to 32-bit words),
    beside a binned range, on the device and through the host pipeline."""
    rng = np.random.default_rng(5400 + seed)
    n_chan = int(rng.choice([1, 33, 257]))
    f_high = float(rng.uniform(900, 1700))
    freqs = channel_freqs(f_high, float(rng.uniform(0.05, 0.25)) * f_high, n_chan)
    k_low = oracle.delay_coeff(freqs[-1], f_high) / 64e-6
    step = float(rng.uniform(0.2, 2.9)) / k_low
    n_dm = int(rng.choice([7, 64, 130]))
    ranges = [(0.0, n_dm * step, step, 1), (n_dm * step, 2 * n_dm * step, 2 * step, 2)]
    s_max = max((oracle.extent(freqs, f_high, 64e-6, r, 10 ** 9)[0] + 1) * r[3] for r in ranges)
    n_samp = int(s_max + rng.choice([1, 1471, 30001]))
    stride = (n_samp + 7) // 8 * 8
    x = filterbank(np.uint16, n_chan, n_samp, 5500 + seed, 40000, 12000, row_stride=stride)
    x[:, n_samp:] = 65535
    ref = oracle.forward(np.ascontiguousarray(x[:, :n_samp]), freqs, f_high, 64e-6, ranges)
    plan = dd.Plan(freqs, f_high, 64e-6, ranges, "u16")
    plan.set_tile(0, "packed")
    info = plan.info(n_samp)
    assert info["tile_dms"][0] == _lib.DD_TILE_PACKED
    # The full copy (odd seeds) or the ring of 16 time segments.
    got = plan.run(torch.from_numpy(x).cuda(), n_samp=n_samp, segments=1 if seed % 2 else 16)
    for r, (g, o) in enumerate(zip(got, ref)):
        np.testing.assert_array_equal(g.cpu().numpy(), o, err_msg=f"range {r}")
    h_in = torch.from_numpy(x).pin_memory()
    h_out = torch.full((info["out_elems"],), -5, dtype=torch.int32).pin_memory()
    plan.run_host(h_in, h_out, torch.empty_like(h_in, device="cuda"), plan.empty_output(n_samp),
                  n_samp=n_samp)
    torch.cuda.synchronize()
    for r, (g, o) in enumerate(zip(plan.split(h_out, n_samp), ref)):
        np.testing.assert_array_equal(g.numpy(), o, err_msg=f"host range {r}")


@pytest.mark.parametrize("seed", range(4))
def test_packed_float32(seed):
    """float32 through the packed tile (64-bit words of two floats, added two
    at a time with add.f32x2), beside a binned range, on the device and
    through the host pipeline, against the FP64 oracle within 1e-5 sum |X|."""
    from gpu_util import assert_float_parity
    rng = np.random.default_rng(5600 + seed)
    n_chan = int(rng.choice([1, 33, 257, 300]))
    f_high = float(rng.uniform(900, 1700))
    freqs = channel_freqs(f_high, float(rng.uniform(0.05, 0.25)) * f_high, n_chan)
    k_low = oracle.delay_coeff(freqs[-1], f_high) / 64e-6
    step = float(rng.uniform(0.2, 2.9)) / k_low
    n_dm = int(rng.choice([7, 64, 130]))
    ranges = [(0.0, n_dm * step, step, 1), (n_dm * step, 2 * n_dm * step, 2 * step, 2)]
    s_max = max((oracle.extent(freqs, f_high, 64e-6, r, 10 ** 9)[0] + 1) * r[3] for r in ranges)
    n_samp = int(s_max + rng.choice([1, 703, 704, 705, 30001]))
    stride = (n_samp + 3) // 4 * 4
    x = filterbank(np.float32, n_chan, n_samp, 5700 + seed, 0.0, 1.0, row_stride=stride)
    x[:, n_samp:] = 1e30  # padding the transform must not read
    xs = np.ascontiguousarray(x[:, :n_samp])
    ref = oracle.forward(xs, freqs, f_high, 64e-6, ranges)
    ref_abs = oracle.forward(xs, freqs, f_high, 64e-6, ranges, take_abs=True)
    plan = dd.Plan(freqs, f_high, 64e-6, ranges, "f32")
    xd = torch.from_numpy(x).cuda()
    # Every float-pair shape (single channels and channel pairs, 16 and 12
    # warps) that fits the plan.
    ran = 0
    for i, sh in enumerate(dd.tile_shapes()):
        if not sh["float_pairs"]:
            continue
        try:
            plan.set_tile_shape(0, "packed", i)
        except dd.DDError:
            continue
        ran += 1
        got = plan.run(xd, n_samp=n_samp)
        for r, (g, o, a) in enumerate(zip(got, ref, ref_abs)):
            assert_float_parity(g.cpu().numpy(), o, a, f"shape {i} range {r}")
    assert ran >= 3
    plan.set_tile(0, "packed")
    info = plan.info(n_samp)
    assert info["tile_dms"][0] == _lib.DD_TILE_PACKED
    h_in = torch.from_numpy(x).pin_memory()
    h_out = torch.full((info["out_elems"],), -5.0, dtype=torch.float32).pin_memory()
    plan.run_host(h_in, h_out, torch.empty_like(h_in, device="cuda"), plan.empty_output(n_samp),
                  n_samp=n_samp)
    torch.cuda.synchronize()
    for r, (g, o, a) in enumerate(zip(plan.split(h_out, n_samp), ref, ref_abs)):
        assert_float_parity(g.numpy(), o, a, f"host range {r}")


@pytest.mark.parametrize("seed", range(6))
def test_packed_binned_uint8(seed):
    """uint8 ranges at bins 2, 4 and 8 on the packed tile (copies of decimated
    pair words, widened every 65535 / (255 bin) channels) beside a bin-1 packed
    range and a plain range, against the oracle; saturated samples (255) on
    every channel cross every widening at its lane bound."""
    rng = np.random.default_rng(5800 + seed)
    n_chan = int(rng.choice([33, 96, 257, 300]))
    f_high = float(rng.uniform(900, 1700))
    freqs = channel_freqs(f_high, float(rng.uniform(0.05, 0.25)) * f_high, n_chan)
    k_low = oracle.delay_coeff(freqs[-1], f_high) / 64e-6
    step = float(rng.uniform(0.2, 1.5)) / k_low
    n_dm = int(rng.choice([7, 64, 130]))
    ranges, lo, tiles = [], 0.0, []
    for b in (1, 2, 4, 8, 3):
        ranges.append((lo, lo + n_dm * step * b, step * b, b))
        lo += n_dm * step * b
        tiles.append("packed" if b != 3 else 0)
    s_max = max((oracle.extent(freqs, f_high, 64e-6, r, 10 ** 9)[0] + 1) * r[3] for r in ranges)
    n_samp = int(s_max + rng.choice([1, 1471, 12001]))
    stride = (n_samp + 15) // 16 * 16
    saturated = seed == 0
    if saturated:
        x = np.zeros((n_chan, stride), np.uint8)
        x[:, :n_samp] = 255
    else:
        x = filterbank(np.uint8, n_chan, n_samp, 5900 + seed, 200, 80, row_stride=stride)
    x[:, n_samp:] = 255
    ref = oracle.forward(np.ascontiguousarray(x[:, :n_samp]), freqs, f_high, 64e-6, ranges)
    plan = dd.Plan(freqs, f_high, 64e-6, ranges, "u8")
    for r, t in enumerate(tiles):
        plan.set_tile(r, t)
    info = plan.info(n_samp)
    assert info["tile_dms"][:4] == [_lib.DD_TILE_PACKED] * 4
    # Binned copies have no ring: the full copies.
    got = plan.run(torch.from_numpy(x).cuda(), n_samp=n_samp)
    for r, (g, o) in enumerate(zip(got, ref)):
        np.testing.assert_array_equal(g.cpu().numpy(), o, err_msg=f"range {r}")
    # The same through a windowed run (the streaming server's call).
    keep = [max(1, o.shape[1] // 2) for o in ref]
    win = plan.run_window(torch.from_numpy(x).cuda(), keep, n_samp=n_samp)
    for r, (w, o) in enumerate(zip(win, ref)):
        np.testing.assert_array_equal(w.cpu().numpy(), o[:, : keep[r]], err_msg=f"window {r}")
