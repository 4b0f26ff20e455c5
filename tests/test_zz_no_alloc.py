"""dd_run_u8_noalloc: the uint8 forward transform for callers that cannot
allocate device memory (its tables live in a fixed array inside the library).

Its output must equal dd_run's (bit for bit, as every integer path here) on
two calls in a row, and it must refuse plans that do not fit its array or do
not run on the uint8 tiled kernel.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import paper_2311_05341_gb300 as dd
from paper_2311_05341_gb300 import _lib
from synth import filterbank, workloads

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


def test_noalloc_matches_dd_run_twice():
    beam = workloads.batched()[0]  # 1024 ch x 131072 samples, 2048 DMs, uint8
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, "u8")
    info = plan.info(beam.n_samp)
    assert info["kernel"] == ["tiled"]
    x_np = filterbank(np.uint8, beam.n_chan, beam.n_samp, beam.seed, 200, 80)
    x = torch.from_numpy(x_np).cuda()
    ref = plan.empty_output(beam.n_samp)
    plan.run(x, out=ref)
    outs = []
    for _ in range(2):
        out = torch.full_like(ref, -7)
        st = _noalloc(plan, x, beam.n_samp, out)
        assert st == _lib.DD_OK, _lib.load().dd_last_error_detail().decode()
        outs.append(out)
    torch.cuda.synchronize()
    n = info["out_elems"]
    for out in outs:
        assert torch.equal(out[:n], ref[:n])


def test_noalloc_rejects_plans_it_cannot_serve():
    x = torch.zeros((16, 4096), dtype=torch.uint8, device="cuda")
    out = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    # Paper-scale tables (8192 channels x 4096 DMs) exceed the fixed array; the
    # call refuses before touching device memory, so small buffers suffice.
    paper = workloads.paper_u8()
    big = dd.Plan(paper.freqs, paper.f_high, paper.t_samp, paper.ranges, "u8", upload=False)
    assert _noalloc(big, x, paper.n_samp, out, stride=paper.n_samp) == _lib.DD_ERR_BUDGET
    assert "at most" in _lib.load().dd_last_error_detail().decode()
    # A plan with a range on the generic kernel (time bin 3) and a float32
    # plan are refused.
    tiny = workloads.tiny_u8()
    binned = dd.Plan(tiny.freqs, tiny.f_high, tiny.t_samp, [(0.0, 8.0, 0.5, 3)], "u8",
                     upload=False)
    assert _noalloc(binned, x, 8192, out, stride=8192) == _lib.DD_ERR_UNSUPPORTED
    f32 = dd.Plan(tiny.freqs, tiny.f_high, tiny.t_samp, tiny.ranges, "f32", upload=False)
    assert _noalloc(f32, x, 4096, out) == _lib.DD_ERR_UNSUPPORTED
