"""The bounded-wait timeout path of the register-tiled kernels, on the GPU.

Every pipeline wait of the tiled kernels polls its mbarrier a bounded number of
times (dd_plan_set_wait_limit).  With the copies of one channel stage withheld
(the test hook of that call) the wait on that stage can never complete: the
kernels must give up after the bound, record DD_ERR_TIMEOUT in the plan's status
word, let the copies they did issue land and return -- no trap, no hang -- and
the context must stay usable: the next run at the default bound is bit-exact
against the oracle.
"""
import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from paper_2311_05341_gb300 import _lib
from paper_2311_05341_gb300 import batch as ddb
from synth import channel_freqs, filterbank

from gpu_util import assert_float_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

POLLS = 2000  # a short bound: each CTA gives up after this many polls


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(dtype, n_chan=300):
    freqs = channel_freqs(1400.0, 300.0, n_chan)
    r = (0.0, 12.8, 0.1, 1)  # about 2 samples of delay per DM step: every tile serves it
    s_max, _ = oracle.extent(freqs, 1400.0, 64e-6, r, 10 ** 9)
    n_samp = s_max + 3001
    npdt, mean, sd = {"u8": (np.uint8, 128, 40), "f32": (np.float32, 0.0, 1.0)}[dtype]
    x = filterbank(npdt, n_chan, n_samp, 77, mean, sd)
    per = 16 // x.itemsize
    stride = (n_samp + per - 1) // per * per
    xd = torch.zeros((n_chan, stride), dtype=getattr(torch, str(x.dtype)), device="cuda")
    xd[:, :n_samp] = torch.from_numpy(x).cuda()
    return freqs, r, x, xd, n_samp


def _timeout_status(plan):
    with pytest.raises(dd.DDError) as ei:
        plan.device_status()
    return ei.value.status


@pytest.mark.parametrize("dtype,tile,hold", [("u8", "pattern", 3), ("u8", "packed", 4),
                                             ("u8", 4, 2), ("u8", "pattern", 0),
                                             ("f32", "pattern", 5)])
def test_withheld_stage_times_out_then_recovers(dtype, tile, hold):
    freqs, r, x, xd, n_samp = _case(dtype)
    plan = dd.Plan(freqs, 1400.0, 64e-6, [r], dtype)
    plan.set_tile(0, tile)
    out = plan.empty_output(n_samp)
    plan.set_wait_limit(POLLS, hold)
    plan.run(xd, out=out, n_samp=n_samp)
    torch.cuda.synchronize()  # the kernels returned
    assert _timeout_status(plan) == _lib.DD_ERR_TIMEOUT
    plan.device_status()  # the flag was cleared by the read
    # The same context, the default bound, no withheld stage: exact again.
    plan.set_wait_limit(0, -1)
    got = plan.run(xd, out=out, n_samp=n_samp)[0].cpu().numpy()
    plan.device_status()
    ref = oracle.forward(x, freqs, 1400.0, 64e-6, [r])[0]
    if dtype == "f32":
        ab = oracle.forward(x, freqs, 1400.0, 64e-6, [r], take_abs=True)[0]
        assert_float_parity(got, ref, ab, f"tile {tile}")
    else:
        np.testing.assert_array_equal(got, ref)


def test_hold_past_the_last_stage_changes_nothing():
    freqs, r, x, xd, n_samp = _case("u8")
    plan = dd.Plan(freqs, 1400.0, 64e-6, [r], "u8")
    plan.set_wait_limit(POLLS, 1000)  # 300 channels have 10 stages
    got = plan.run(xd, n_samp=n_samp)[0].cpu().numpy()
    plan.device_status()
    np.testing.assert_array_equal(got, oracle.forward(x, freqs, 1400.0, 64e-6, [r])[0])


def test_batch_reports_timeout_then_recovers():
    freqs = channel_freqs(1400.0, 300.0, 200)
    beams = [ddb.BeamSpec(freqs, 1400.0, 64e-6, [(0.0, 12.8, 0.1, 1)], "u8", 9000),
             ddb.BeamSpec(freqs, 1400.0, 64e-6, [(0.0, 6.4, 0.1, 1)], "u8", 7000)]
    runner = ddb.BatchRunner(beams, autotune=False, graph=False)
    hosts = []
    for i, (b, xd) in enumerate(zip(runner.beams, runner.inputs)):
        h = filterbank(np.uint8, 200, b.n_samp, 300 + i, 128, 40)
        xd[:, : b.n_samp].copy_(torch.from_numpy(h).cuda())
        hosts.append(h)
    runner.plans[1].set_wait_limit(POLLS, 2)
    runner.bind()
    runner.run()
    torch.cuda.synchronize()
    with pytest.raises(dd.DDError) as ei:
        runner.status()
    assert ei.value.status == _lib.DD_ERR_TIMEOUT
    runner.plans[1].set_wait_limit(0, -1)
    runner.bind()
    runner.run()
    runner.status()
    for i, b in enumerate(runner.beams):
        got = runner.planes(i)[0].cpu().numpy()
        np.testing.assert_array_equal(got, oracle.forward(hosts[i], b.freqs, b.f_ref, b.t_samp,
                                                          b.ranges)[0])
