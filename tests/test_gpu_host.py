"""dd_run_host: host buffers in and out, the raw time axis in segments whose
copies overlap the kernels.  Its output must equal dd_run's on the same input
(the same kernels compute every output once) and the oracle's."""
import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from synth import channel_freqs, filterbank, workloads

from gpu_util import assert_float_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


_NP = {"u8": np.uint8, "u16": np.uint16, "f32": np.float32}
_NOISE = {"u8": (128, 30), "u16": (32768, 3000), "f32": (0.0, 1.0)}


def _host_vs_device(freqs, f_ref, t_samp, ranges, dtype, n_samp, seed, packed=True):
    plan = dd.Plan(freqs, f_ref, t_samp, ranges, dtype)
    per = 16 // np.dtype(_NP[dtype]).itemsize
    stride = (n_samp + per - 1) // per * per
    mean, sd = _NOISE[dtype]
    x = filterbank(_NP[dtype], len(freqs), n_samp, seed, mean, sd, row_stride=stride)
    h_in = torch.from_numpy(x).pin_memory()
    info = plan.info(n_samp)
    out_dt = torch.float32 if dtype == "f32" else torch.int32
    h_out = torch.full((info["out_elems"],), -5, dtype=out_dt).pin_memory()
    d_in = torch.empty_like(h_in, device="cuda")
    d_out = plan.empty_output(n_samp)
    plan.run_host(h_in, h_out, d_in, d_out, n_samp=n_samp, packed=packed)
    torch.cuda.synchronize()
    ref_dev = plan.run(h_in.cuda(), n_samp=n_samp)
    flat = torch.cat([p.reshape(-1) for p in ref_dev]).cpu()
    assert torch.equal(h_out, flat)
    return plan, x, h_out, info


# packed: the automatic uint8 and uint16 tiles at bin 1 read the packed copy
# the pipeline makes as the input arrives, or unpack the input themselves.
@pytest.mark.parametrize("dtype,packed", [("u8", True), ("u8", False), ("u16", True),
                                          ("u16", False), ("f32", True)])
def test_host_path_equals_device_path_and_oracle(dtype, packed):
    freqs = channel_freqs(1500.0, 300.0, 97)
    # Four ranges: pattern and offset tiles, decimation, and a time bin (3)
    # that only the generic kernel takes.
    ranges = [(0.0, 6.0, 0.05, 1), (6.0, 12.0, 0.1, 2), (12.0, 30.0, 0.3, 3),
              (30.0, 60.0, 1.0, 4)]
    n_samp = 40001
    plan, x, h_out, info = _host_vs_device(freqs, 1500.0, 64e-6, ranges, dtype, n_samp, 11,
                                           packed)
    ref = oracle.forward(x[:, :n_samp], freqs, 1500.0, 64e-6, ranges)
    planes = plan.split(h_out, n_samp)
    for r, (g, o) in enumerate(zip(planes, ref)):
        g = g.numpy()
        if dtype == "f32":
            ab = oracle.forward(x[:, :n_samp], freqs, 1500.0, 64e-6, ranges, take_abs=True)[r]
            assert_float_parity(g, o, ab, f"range {r}")
        else:
            np.testing.assert_array_equal(g, o, err_msg=f"range {r}")


def test_host_path_short_input():
    """Fewer raw samples than segments' worth of tiles: most segments add nothing."""
    freqs = channel_freqs(1400.0, 300.0, 33)
    _host_vs_device(freqs, 1400.0, 64e-6, [(0.0, 3.2, 0.1, 1)], "u8", 3001, 12)


def test_host_path_paper_scale():
    beam = workloads.paper_u8()
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, "u8")
    x = filterbank(np.uint8, beam.n_chan, beam.n_samp, 13, 128, 16)
    h_in = torch.from_numpy(x).pin_memory()
    info = plan.info(beam.n_samp)
    h_out = torch.full((info["out_elems"],), -5, dtype=torch.int32).pin_memory()
    d_in = torch.empty_like(h_in, device="cuda")
    d_out = plan.empty_output(beam.n_samp)
    plan.run_host(h_in, h_out, d_in, d_out, n_samp=beam.n_samp)
    torch.cuda.synchronize()
    ref = plan.run(d_in, n_samp=beam.n_samp)[0].reshape(-1).cpu()
    assert torch.equal(h_out, ref)
