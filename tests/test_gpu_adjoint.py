"""Parity of the CUDA adjoint (re-dispersion) with the oracle transpose, on
both of its kernels (the gather, and the forward pattern tile on the
cotangent rows with the transposed shift table).

Checks: full-plane parity with the FP64 oracle adjoint on multi-range,
binned plans; the dot-product test <A X, W> = <X, A^T W> and central finite
differences of L = sum(Y * W) on the differentiable float32 workload
(1024 channels x 65536 samples x 1024 DMs).
"""
import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from synth import workloads, channel_freqs, filterbank

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("seed", range(4))
def test_adjoint_full_vs_oracle(seed):
    rng = np.random.default_rng(50 + seed)
    n_chan = int(rng.choice([5, 17, 64, 100]))
    freqs = channel_freqs(1400.0, 300.0, n_chan)
    ranges = [(0.0, 20.0, 0.5, 1), (20.0, 40.0, 1.0, int(rng.choice([1, 2, 3]))),
              (40.0, 60.0, 2.0, int(rng.choice([2, 4])))][: int(rng.integers(1, 4))]
    n_samp = int(rng.integers(1200, 3000))
    plan = dd.Plan(freqs, 1400.0, 64e-6, ranges, "f32")
    info = plan.info(n_samp)
    ybar = rng.standard_normal(info["out_elems"]).astype(np.float32)
    parts = [ybar[o:o + a * b].reshape(a, b).astype(np.float64)
             for o, a, b in zip(info["out_offset"], info["n_dm"], info["n_out"])]
    ref = oracle.adjoint(parts, n_chan, n_samp, freqs, 1400.0, 64e-6, ranges)
    ref_abs = oracle.adjoint([np.abs(p) for p in parts], n_chan, n_samp, freqs, 1400.0, 64e-6,
                             ranges)
    got = plan.run_adjoint(torch.from_numpy(ybar).cuda(), n_samp).cpu().numpy()
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= 1e-5 * ref_abs + 1e-30)
    # Samples that no output reads get exactly zero.
    assert np.all(got[ref_abs == 0] == 0)


def test_adjoint_dot_product_and_fd_diff_workload():
    beam = workloads.diff_f32()
    x = filterbank(np.float32, beam.n_chan, beam.n_samp, beam.seed, 0.0, 1.0)
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, "f32")
    info = plan.info(beam.n_samp)
    rng = np.random.default_rng(4001)
    w = rng.standard_normal(info["out_elems"]).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    wt = torch.from_numpy(w).cuda()
    out = plan.empty_output(beam.n_samp)
    plan.run(xt, out=out)
    xbar = plan.run_adjoint(wt, beam.n_samp)
    lhs = float((out[: info["out_elems"]].double() * wt.double()).sum())
    rhs = float((xt.double() * xbar.double()).sum())
    scale = float((out[: info["out_elems"]].double().abs() * wt.double().abs()).sum())
    assert abs(lhs - rhs) <= 1e-6 * scale

    # Central finite differences of L = sum(Y * W) on 64 random entries.  L is
    # linear in X, so (L(X + h e) - L(X - h e)) / 2h equals the gradient up to
    # float32 rounding of the outputs.
    xbar_h = xbar.cpu().numpy().astype(np.float64)
    h = 4.0
    for _ in range(64):
        c, t = int(rng.integers(0, beam.n_chan)), int(rng.integers(0, beam.n_samp))
        vals = []
        for sgn in (1.0, -1.0):
            xp = xt.clone()
            xp[c, t] += sgn * h
            plan.run(xp, out=out)
            vals.append(float((out[: info["out_elems"]].double() * wt.double()).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        tol = 2e-3 * (1.0 + abs(xbar_h[c, t]))
        assert abs(fd - xbar_h[c, t]) <= tol, (c, t, fd, xbar_h[c, t])


def test_adjoint_rejects_integer_plan():
    plan = dd.Plan(channel_freqs(1400.0, 300.0, 8), 1400.0, 64e-6, [(0.0, 5.0, 1.0, 1)], "u8")
    with pytest.raises(dd.DDError) as ei:
        plan.run_adjoint(torch.zeros(1024, device="cuda"), 512)
    assert ei.value.status == 2


@pytest.mark.parametrize("seed", range(6))
def test_adjoint_both_kernels_vs_oracle(seed):
    """Plans with narrow channels (the pattern path: channels as trials with
    the transposed shift table, expanded over bins) and with wide channels
    (the gather path), ragged channel counts and several binned ranges."""
    rng = np.random.default_rng(70 + seed)
    narrow = seed % 2 == 0
    if narrow:  # adjacent channels' delays differ by at most ~1 sample
        n_chan = int(rng.choice([33, 96, 130, 257]))
        freqs = channel_freqs(1500.0, 0.02 * n_chan, n_chan)
        n_dm = int(rng.choice([7, 64, 65, 130]))
    else:  # few wide channels, many DMs: several samples between neighbours
        n_chan = int(rng.choice([9, 17, 33]))
        freqs = channel_freqs(1500.0, 600.0, n_chan)
        n_dm = int(rng.choice([130, 200]))
    k_low = oracle.delay_coeff(freqs[-1], 1500.0) / 64e-6
    step = float(rng.uniform(0.3, 1.5)) / k_low
    ranges = [(0.0, n_dm * step, step, 1)]
    if rng.integers(0, 2):
        ranges.append((n_dm * step, 2 * n_dm * step, 2 * step, int(rng.choice([2, 3, 4]))))
    s_max = max((oracle.extent(freqs, 1500.0, 64e-6, r, 10 ** 9)[0] + 1) * r[3] for r in ranges)
    n_samp = int(s_max + rng.integers(1, 3000))
    plan = dd.Plan(freqs, 1500.0, 64e-6, ranges, "f32")
    info = plan.info(n_samp)
    assert info["adjoint_kernel"] == ("pattern" if narrow else "gather")
    ybar = rng.standard_normal(info["out_elems"]).astype(np.float32)
    parts = [ybar[o:o + a * b].reshape(a, b).astype(np.float64)
             for o, a, b in zip(info["out_offset"], info["n_dm"], info["n_out"])]
    ref = oracle.adjoint(parts, n_chan, n_samp, freqs, 1500.0, 64e-6, ranges)
    ref_abs = oracle.adjoint([np.abs(p) for p in parts], n_chan, n_samp, freqs, 1500.0, 64e-6,
                             ranges)
    got = plan.run_adjoint(torch.from_numpy(ybar).cuda(), n_samp).cpu().numpy()
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= 1e-5 * ref_abs + 1e-30)
    assert np.all(got[ref_abs == 0] == 0)


def test_adjoint_kernel_of_diff_workload():
    beam = workloads.diff_f32()
    plan = dd.Plan(beam.freqs, beam.f_high, beam.t_samp, beam.ranges, "f32", upload=False)
    assert plan.info(beam.n_samp)["adjoint_kernel"] == "pattern"


def test_adjoint_without_scratch_runs_the_gather():
    """dd_run_adjoint (no scratch) on a plan whose adjoint kernel is the
    pattern tile runs the gather; both agree with the oracle transpose."""
    from paper_2311_05341_gb300 import _lib
    rng = np.random.default_rng(91)
    n_chan = 130
    freqs = channel_freqs(1500.0, 2.6, n_chan)
    r = [(0.0, 64 * 0.4, 0.4, 1), (25.6, 51.2, 0.8, 2)]
    n_samp = 6000
    plan = dd.Plan(freqs, 1500.0, 64e-6, r, "f32")
    info = plan.info(n_samp)
    assert info["adjoint_kernel"] == "pattern"
    ybar = rng.standard_normal(info["out_elems"]).astype(np.float32)
    parts = [ybar[o:o + a * b].reshape(a, b).astype(np.float64)
             for o, a, b in zip(info["out_offset"], info["n_dm"], info["n_out"])]
    ref = oracle.adjoint(parts, n_chan, n_samp, freqs, 1500.0, 64e-6, r)
    ref_abs = oracle.adjoint([np.abs(p) for p in parts], n_chan, n_samp, freqs, 1500.0, 64e-6, r)
    yt = torch.from_numpy(ybar).cuda()
    stride = (n_samp + 3) // 4 * 4
    xg = torch.full((n_chan, stride), 7.0, dtype=torch.float32, device="cuda")
    lib = _lib.load()
    assert lib.dd_run_adjoint(plan.handle, yt.data_ptr(), xg.data_ptr(), n_samp, stride,
                              None) == _lib.DD_OK
    got_p = plan.run_adjoint(yt, n_samp).cpu().numpy()
    for got in (xg[:, :n_samp].cpu().numpy(), got_p):
        assert np.all(np.abs(got.astype(np.float64) - ref) <= 1e-5 * ref_abs + 1e-30)
