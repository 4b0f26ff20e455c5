"""Parity of the pattern tile with channel classes (DD_TILE_MERGE) with the
oracle, bit-exact: stages whose classes take one to several rounds, classes
of up to a whole stage of channels at the 16-bit lane bound, ragged channel
counts and DM counts, and the same plans on the pattern tile without
classes."""
import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from paper_2311_05341_gb300._lib import DD_TILE_MERGE
from synth import channel_freqs, filterbank

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _device(x):
    stride = (x.shape[1] + 15) // 16 * 16
    xd = torch.zeros((x.shape[0], stride), dtype=torch.uint8, device="cuda")
    xd[:, : x.shape[1]] = torch.from_numpy(x).cuda()
    return xd


def _run(freqs, f_high, r, x, tile):
    plan = dd.Plan(freqs, f_high, 64e-6, [r], "u8")
    plan.set_tile(0, tile)
    out = plan.run(_device(x), n_samp=x.shape[1])[0].cpu().numpy()
    return out, plan.info(x.shape[1])


@pytest.mark.parametrize("seed", range(10))
def test_merge_random_plans(seed):
    """Channel widths from 0.02 to 1.2 MHz and 0.2 to 1.9 samples of delay per
    DM step: from nearly every channel in one class to one class per channel
    (several rounds per stage)."""
    rng = np.random.default_rng(4400 + seed)
    n_chan = int(rng.choice([1, 31, 33, 96, 257, 512, 700]))
    f_high = float(rng.uniform(1000, 1700))
    bw = float(rng.uniform(0.02, 1.2)) * n_chan
    freqs = channel_freqs(f_high, min(bw, 0.4 * f_high), n_chan)
    k_low = oracle.delay_coeff(freqs[-1], f_high) / 64e-6
    step = float(rng.uniform(0.2, 1.9)) / max(k_low, 1e-9)
    n_dm = int(rng.choice([1, 15, 16, 17, 64, 65, 150]))
    lo = float(rng.uniform(0, 400)) * step
    r = (lo, lo + n_dm * step, step, 1)
    s_max, _ = oracle.extent(freqs, f_high, 64e-6, r, 10 ** 9)
    n_samp = int(s_max + rng.choice([1, 1471, 1472, 1473, 4000]))
    x = filterbank(np.uint8, n_chan, n_samp, 4500 + seed, 200, 80)
    ref = oracle.forward(x, freqs, f_high, 64e-6, [r])[0]
    got, info = _run(freqs, f_high, r, x, "merge")
    assert info["tile_dms"] == [DD_TILE_MERGE]
    np.testing.assert_array_equal(got, ref)
    got_p, _ = _run(freqs, f_high, r, x, "pattern")
    np.testing.assert_array_equal(got_p, ref)


def test_merge_whole_stage_classes_saturated():
    """Low DMs on narrow channels: classes of up to 32 channels, every sample
    255, so each 16-bit lane holds 255 x 256 before it is widened."""
    n_chan = 1024
    freqs = channel_freqs(1670.0, 20.0, n_chan)
    r = (0.0, 6.4, 0.1, 1)
    s_max, _ = oracle.extent(freqs, 1670.0, 64e-6, r, 10 ** 9)
    x = np.full((n_chan, s_max + 3000), 255, np.uint8)
    got, info = _run(freqs, 1670.0, r, x, "merge")
    assert info["tile_dms"] == [DD_TILE_MERGE]
    assert np.all(got == 255 * n_chan)
    rng = np.random.default_rng(3)
    x = rng.integers(0, 256, x.shape).astype(np.uint8)
    ref = oracle.forward(x, freqs, 1670.0, 64e-6, [r])[0]
    got, _ = _run(freqs, 1670.0, r, x, "merge")
    np.testing.assert_array_equal(got, ref)


def test_merge_time_windows_and_host_path():
    """The host pipeline (launch windows over time tiles) on a merged plan."""
    n_chan = 300
    freqs = channel_freqs(1500.0, 300.0, n_chan)
    k_low = oracle.delay_coeff(freqs[-1], 1500.0) / 64e-6
    step = 1.1 / k_low
    r = (0.0, 96 * step, step, 1)
    s_max, _ = oracle.extent(freqs, 1500.0, 64e-6, r, 10 ** 9)
    n_samp = int(s_max + 40000)
    stride = (n_samp + 15) // 16 * 16
    x = filterbank(np.uint8, n_chan, n_samp, 77, 128, 40, row_stride=stride)
    ref = oracle.forward(np.ascontiguousarray(x[:, :n_samp]), freqs, 1500.0, 64e-6, [r])[0]
    plan = dd.Plan(freqs, 1500.0, 64e-6, [r], "u8")
    plan.set_tile(0, "merge")
    info = plan.info(n_samp)
    assert info["tile_dms"] == [DD_TILE_MERGE]
    h_in = torch.from_numpy(x).pin_memory()
    h_out = torch.full((info["out_elems"],), -5, dtype=torch.int32).pin_memory()
    d_in = torch.empty_like(h_in, device="cuda")
    plan.run_host(h_in, h_out, d_in, plan.empty_output(n_samp), n_samp=n_samp)
    torch.cuda.synchronize()
    got = plan.split(h_out, n_samp)[0].numpy()
    np.testing.assert_array_equal(got, ref)
