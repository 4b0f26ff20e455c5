"""DedispFn: autograd through the forward kernel and the adjoint gather kernel.

Checked on the differentiable workload (1024 channels x 65536 samples, 1024
DMs): loss = sum(Y * W); the autograd gradient equals the oracle transpose
applied to W (sampled channels), agrees with central finite differences of
the loss on 64 random entries, and satisfies the dot-product identity.
"""
import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from paper_2311_05341_gb300.autograd import DedispFn, dedisperse
from synth import channel_freqs, filterbank, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_autograd_matches_oracle_transpose_small():
    freqs = channel_freqs(1400.0, 300.0, 37)
    ranges = [(0.0, 10.0, 0.5, 1), (10.0, 20.0, 1.0, 2)]
    n_samp = 3001  # ragged: the binding pads rows to a 16-byte stride
    plan = dd.Plan(freqs, 1400.0, 64e-6, ranges, "f32")
    x = torch.from_numpy(filterbank(np.float32, 37, n_samp, 21, 0, 1)).cuda().requires_grad_()
    planes = dedisperse(x, plan)
    rng = np.random.default_rng(5)
    ws = [torch.from_numpy(rng.standard_normal(p.shape).astype(np.float32)).cuda() for p in planes]
    loss = sum((p * w).sum() for p, w in zip(planes, ws))
    loss.backward()
    ref = oracle.adjoint([w.cpu().numpy().astype(np.float64) for w in ws], 37, n_samp, freqs,
                         1400.0, 64e-6, ranges)
    ref_abs = oracle.adjoint([np.abs(w.cpu().numpy().astype(np.float64)) for w in ws], 37, n_samp,
                             freqs, 1400.0, 64e-6, ranges)
    got = x.grad.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-5 * ref_abs + 1e-30)


def test_autograd_diff_workload():
    beam = workloads.diff_f32()
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, "f32")
    x0 = torch.from_numpy(filterbank(np.float32, beam.n_chan, beam.n_samp, beam.seed, 0, 1)).cuda()
    x = x0.clone().requires_grad_()
    flat = DedispFn.apply(x, plan)
    info = plan.info(beam.n_samp)
    n = info["out_elems"]
    w = torch.randn(flat.numel(), generator=torch.Generator().manual_seed(4000)).cuda()
    loss = (flat[:n].double() * w[:n].double()).sum()
    loss.backward()
    flat = flat.detach()
    g = x.grad.double()

    # Dot-product identity <A x, w> = <x, A^T w>.
    rhs = float((x0.double() * g).sum())
    scale = float((flat[:n].double().abs() * w[:n].double().abs()).sum())
    assert abs(float(loss) - rhs) <= 1e-6 * scale

    # Sampled channels against the oracle transpose.
    wn = w[:n].cpu().numpy().reshape(info["n_dm"][0], info["n_out"][0]).astype(np.float64)
    chans = [0, 511, 1023]
    sub = oracle.adjoint_channels([wn], beam.n_chan, beam.n_samp, beam.freqs, beam.f_high,
                                  beam.t_samp, beam.ranges, chans)
    sub_abs = oracle.adjoint_channels([np.abs(wn)], beam.n_chan, beam.n_samp, beam.freqs,
                                      beam.f_high, beam.t_samp, beam.ranges, chans)
    got = g[chans].cpu().numpy()
    assert np.all(np.abs(got - sub) <= 1e-5 * sub_abs + 1e-30)

    # Central finite differences of the loss on 64 random entries.
    rng = np.random.default_rng(4001)
    h = 4.0
    with torch.no_grad():
        for _ in range(64):
            c, t = int(rng.integers(0, beam.n_chan)), int(rng.integers(0, beam.n_samp))
            vals = []
            for sgn in (1.0, -1.0):
                xp = x0.clone()
                xp[c, t] += sgn * h
                f = DedispFn.apply(xp, plan)
                vals.append(float((f[:n].double() * w[:n].double()).sum()))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - float(g[c, t])) <= 2e-3 * (1.0 + abs(float(g[c, t])))
