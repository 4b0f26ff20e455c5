"""dd_run_u8_noalloc: the uint8 forward transform for callers that cannot
allocate device memory (a real-time pipeline that must not call cudaMalloc
mid-observation, a plug-in whose host framework owns every device
allocation).  Its tables live in a fixed array inside the library.

Its output must equal dd_run's and the oracle's (bit for bit, as every integer
path here) on two calls in a row, for one range and for several ranges at
different time bins; it must refuse plans that do not fit its array or do not
run on the uint8 tiled kernel; and a bounded wait that gives up must be
reported by dd_run_u8_noalloc_status.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from paper_2311_05341_gb300 import _lib
from synth import channel_freqs, filterbank, workloads

from gpu_util import oracle_input

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _noalloc(plan, x, n_samp, out, stride=None):
    stream = torch.cuda.current_stream().cuda_stream
    stride = x.stride(0) if stride is None else stride
    return _lib.load().dd_run_u8_noalloc(plan.handle, x.data_ptr(), stride, n_samp,
                                         out.data_ptr(), stream)


def _noalloc_status():
    return _lib.load().dd_run_u8_noalloc_status(torch.cuda.current_stream().cuda_stream)


def _twice_against_dd_run_and_oracle(plan, x_np, n_samp):
    info = plan.info(n_samp)
    assert set(info["kernel"]) == {"tiled"}
    x = torch.from_numpy(x_np).cuda()
    ref = plan.empty_output(n_samp)
    plan.run(x, out=ref, n_samp=n_samp)
    outs = []
    for _ in range(2):
        out = torch.full_like(ref, -7)
        st = _noalloc(plan, x, n_samp, out)
        assert st == _lib.DD_OK, _lib.load().dd_last_error_detail().decode()
        outs.append(out)
    torch.cuda.synchronize()
    assert _noalloc_status() == _lib.DD_OK
    n = info["out_elems"]
    for out in outs:
        assert torch.equal(out[:n], ref[:n])
    orc = oracle.forward(x_np, plan.freqs, plan.f_ref, plan.t_samp, plan.ranges)
    for r, (o, g) in enumerate(zip(orc, plan.split(outs[1], n_samp))):
        np.testing.assert_array_equal(g.cpu().numpy(), o, err_msg=f"range {r}")


def test_noalloc_matches_dd_run_and_oracle_twice():
    beam = workloads.batched()[0]  # 1024 ch x 131072 samples, 2048 DMs, uint8
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, "u8")
    x, _, _, _ = oracle_input(beam)
    _twice_against_dd_run_and_oracle(plan, x, beam.n_samp)


def test_noalloc_several_ranges_and_bins():
    """Two tiled ranges at bins 1 and 2 and an offset-tile range: the
    per-range table layout of the array and the output offsets."""
    freqs = channel_freqs(1670.0, 320.0, 1000)
    ranges = [(0.0, 15.0, 0.1, 1), (15.0, 30.0, 0.2, 2), (30.0, 40.0, 0.2, 1)]
    n_samp = 40000
    plan = dd.Plan(freqs, 1670.0, 64e-6, ranges, "u8")
    plan.set_tile(2, 4)
    x = filterbank(np.uint8, 1000, n_samp, 41, 128, 40)
    _twice_against_dd_run_and_oracle(plan, x, n_samp)


def test_noalloc_reports_a_wait_that_gave_up():
    freqs = channel_freqs(1400.0, 300.0, 300)
    r = (0.0, 12.8, 0.1, 1)
    n_samp = 9008  # rows of a multiple of 16 bytes
    plan = dd.Plan(freqs, 1400.0, 64e-6, [r], "u8", upload=False)
    x_np = filterbank(np.uint8, 300, n_samp, 43, 128, 40)
    x = torch.from_numpy(x_np).cuda()
    out = torch.zeros(plan.info(n_samp)["out_elems"], dtype=torch.int32, device="cuda")
    plan.set_wait_limit(2000, 3)  # stage 3's copies are withheld: its wait runs out
    assert _noalloc(plan, x, n_samp, out) == _lib.DD_OK
    torch.cuda.synchronize()
    assert _noalloc_status() == _lib.DD_ERR_TIMEOUT
    assert _noalloc_status() == _lib.DD_OK  # read and cleared
    plan.set_wait_limit(0, -1)
    assert _noalloc(plan, x, n_samp, out) == _lib.DD_OK
    assert _noalloc_status() == _lib.DD_OK
    ref = oracle.forward(x_np, freqs, 1400.0, 64e-6, [r])[0]
    np.testing.assert_array_equal(out.cpu().numpy().reshape(ref.shape), ref)


def test_noalloc_rejects_plans_it_cannot_serve():
    x = torch.zeros((16, 4096), dtype=torch.uint8, device="cuda")
    out = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    # Paper-scale tables (8192 channels x 4096 DMs) exceed the fixed array; the
    # call refuses before touching device memory, so small buffers suffice.
    paper = workloads.paper_u8()
    big = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, "u8", upload=False)
    assert _noalloc(big, x, paper.n_samp, out, stride=paper.n_samp) == _lib.DD_ERR_BUDGET
    assert "at most" in _lib.load().dd_last_error_detail().decode()
    # A plan with a range on the generic kernel (time bin 3), a packed-tile
    # plan and a float32 plan are refused.
    tiny = workloads.tiny_u8()
    binned = dd.Plan(tiny.freqs, tiny.f_high, tiny.t_samp, [(0.0, 8.0, 0.5, 3)], "u8",
                     upload=False)
    assert _noalloc(binned, x, 8192, out, stride=8192) == _lib.DD_ERR_UNSUPPORTED
    packed = dd.Plan(tiny.freqs, tiny.f_high, tiny.t_samp, [(0.0, 8.0, 0.025, 1)], "u8",
                     upload=False)
    packed.set_tile(0, "packed")
    assert _noalloc(packed, x, 4096, out) == _lib.DD_ERR_UNSUPPORTED
    f32 = dd.Plan(tiny.freqs, tiny.f_high, tiny.t_samp, tiny.ranges, "f32", upload=False)
    assert _noalloc(f32, x, 4096, out) == _lib.DD_ERR_UNSUPPORTED
