"""Front end: time-major samples to channel-major rows (dd_transpose), and the
host pipeline that takes time-major input (dd_run_host_tmajor).  A transpose
is a permutation, so results are compared bit for bit."""
import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from synth import channel_freqs, filterbank

from gpu_util import assert_float_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


_NP = {"u8": np.uint8, "u16": np.uint16, "f32": np.float32}


def _tm(dtype, n_samp, n_chan, seed):
    """Time-major host array [n_samp][stride] (16-byte rows), random samples."""
    per = 16 // np.dtype(_NP[dtype]).itemsize
    stride = (n_chan + per - 1) // per * per
    rng = np.random.default_rng(seed)
    if dtype == "f32":
        x = rng.standard_normal((n_samp, stride)).astype(np.float32)
    else:
        x = rng.integers(0, np.iinfo(_NP[dtype]).max + 1, (n_samp, stride)).astype(_NP[dtype])
    return x


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
@pytest.mark.parametrize("n_samp,n_chan", [(1, 1), (5, 3), (130, 129), (1000, 257), (4099, 64),
                                           (333, 1024)])
def test_transpose_equals_definition(dtype, n_samp, n_chan):
    x = _tm(dtype, n_samp, n_chan, n_samp * 7 + n_chan)
    got = dd.transpose(torch.from_numpy(x).cuda(), n_chan=n_chan).cpu().numpy()
    np.testing.assert_array_equal(got[:, :n_samp], oracle.transpose(x[:, :n_chan]))


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_transpose_window_writes_only_its_samples(dtype):
    n_samp, n_chan = 2000, 200
    x = _tm(dtype, n_samp, n_chan, 3)
    xd = torch.from_numpy(x).cuda()
    per = 16 // x.itemsize
    out = torch.full((n_chan, (n_samp + per - 1) // per * per), 7, dtype=xd.dtype, device="cuda")
    dd.transpose(xd, n_chan=n_chan, out=out, t_begin=512, t_end=1501)
    got = out.cpu().numpy()
    ref = oracle.transpose(x[:, :n_chan])
    np.testing.assert_array_equal(got[:, 512:1501], ref[:, 512:1501])
    assert np.all(got[:, :512] == 7) and np.all(got[:, 1501:] == 7)


@pytest.mark.parametrize("dtype", ["u8", "u16", "f32"])
def test_time_major_host_pipeline(dtype):
    freqs = channel_freqs(1500.0, 300.0, 77)
    ranges = [(0.0, 8.0, 0.05, 1), (8.0, 20.0, 0.2, 2)]
    n_samp = 30011
    plan = dd.Plan(freqs, 1500.0, 64e-6, ranges, dtype)
    x_tm = _tm(dtype, n_samp, 77, 21)
    h_in = torch.from_numpy(x_tm).pin_memory()
    info = plan.info(n_samp)
    out_dt = torch.float32 if dtype == "f32" else torch.int32
    h_out = torch.full((info["out_elems"],), -3, dtype=out_dt).pin_memory()
    per = 16 // x_tm.itemsize
    d_tm = torch.empty_like(h_in, device="cuda")
    d_cm = torch.empty((77, (n_samp + per - 1) // per * per), dtype=d_tm.dtype, device="cuda")
    d_out = plan.empty_output(n_samp)
    plan.run_host_tmajor(h_in, h_out, d_tm, d_cm, d_out, n_samp=n_samp)
    torch.cuda.synchronize()
    # The oracle's transform of the oracle's transpose of the same samples.
    x_cm = np.ascontiguousarray(oracle.transpose(x_tm[:, :77]))
    ref = oracle.forward(x_cm, freqs, 1500.0, 64e-6, ranges)
    got = plan.split(h_out, n_samp)
    for r, (g, o) in enumerate(zip(got, ref)):
        g = g.numpy()
        if dtype == "f32":
            ab = oracle.forward(x_cm, freqs, 1500.0, 64e-6, ranges, take_abs=True)[r]
            assert_float_parity(g, o, ab, f"range {r}")
        else:
            np.testing.assert_array_equal(g, o, err_msg=f"range {r}")
