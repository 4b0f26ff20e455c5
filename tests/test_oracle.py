"""Pins for the CPU oracle against what the paper and the mathematics fix.

None of these re-call the oracle's own formula to produce an expected value:
the expectations come from hand-worked numbers, the paper's own printed
numbers (Table 2, Eq. 4, Eq. 7), a pulsar-astronomy handbook constant, exact
rational arithmetic, closed forms and invariants of the direct transform
(Eq. 3 / Algorithm 1), and an independent Python brute force.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C_DM = Fraction(4148808, 1000)  # MHz^2 s pc^-1 cm^3


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def exact_shift(dm, f, f_ref, b, t_samp):
    """Round-half-up shift in exact rational arithmetic on the FP64 inputs.

    Returns (shift, distance of the exact value from the nearest half-integer).
    """
    dm, f, f_ref, t_samp = (Fraction(v) for v in (dm, f, f_ref, t_samp))
    x = dm * C_DM * (1 / (f * f) - 1 / (f_ref * f_ref)) / (b * t_samp)
    n = math.floor(x + Fraction(1, 2))
    frac = x - math.floor(x)
    return n, abs(frac - Fraction(1, 2))


# --------------------------------------------------------------------------
# Hand-worked example: 3 channels x 12 samples x 4 DMs.
#   f = 400, 350, 300 MHz, f_ref = 400 MHz, t_samp = 5 ms, DMs 0, 0.5, 1, 1.5.
#   Per unit DM, in samples (Eq. 1 / t_samp):
#     ch1: 4148.808 * (1/350^2 - 1/400^2) / 0.005 = 1.58755...
#     ch2: 4148.808 * (1/300^2 - 1/400^2) / 0.005 = 4.03354...
#   Rounded half up: ch1 -> 0, 0.79->1, 1.59->2, 2.38->2
#                    ch2 -> 0, 2.02->2, 4.03->4, 6.05->6
#   S_max = 6, N_out = 12 - 6 = 6.
#   With X[c][t] = 100 c + t:  Y[d][t] = sum_c (100 c + t + s(c,d))
#                                      = 300 + 3 t + sum_c s(c,d).
# --------------------------------------------------------------------------
HAND_FREQS = [400.0, 350.0, 300.0]
HAND_RANGE = (0.0, 2.0, 0.5, 1)
HAND_TABLE = np.array([[0, 0, 0], [0, 1, 2], [0, 2, 4], [0, 2, 6]])


def test_hand_worked_shift_table(oracle_mod):
    t = oracle_mod.shift_table(HAND_FREQS, 400.0, 0.005, HAND_RANGE)
    np.testing.assert_array_equal(t, HAND_TABLE)
    assert oracle_mod.extent(HAND_FREQS, 400.0, 0.005, HAND_RANGE, 12) == (6, 6)


def test_hand_worked_closed_form(oracle_mod):
    x = np.array([[100 * c + t for t in range(12)] for c in range(3)], dtype=np.uint16)
    (y,) = oracle_mod.forward(x, HAND_FREQS, 400.0, 0.005, [HAND_RANGE])
    sums = [0, 3, 6, 8]
    expect = np.array([[300 + 3 * t + sums[d] for t in range(6)] for d in range(4)])
    np.testing.assert_array_equal(y, expect)


def test_hand_worked_arbitrary_input(oracle_mod):
    x = np.array([[(7 * c + t * t) % 256 for t in range(12)] for c in range(3)],
                 dtype=np.uint8)
    (y,) = oracle_mod.forward(x, HAND_FREQS, 400.0, 0.005, [HAND_RANGE])
    for d in range(4):
        for t in range(6):
            assert y[d, t] == sum(int(x[c, t + HAND_TABLE[d, c]]) for c in range(3))


# --------------------------------------------------------------------------
# The paper's own numbers.
# --------------------------------------------------------------------------
def test_table2_trial_counts(oracle_mod):
    """Table 2: fixed-step ranges 0-150/0.1, 150-300/0.2, 300-500/0.25."""
    rows = _golden("tab2_plans.txt")
    assert len(rows) == 3
    for lo, hi, step, count in rows:
        r = (float(lo), float(hi), float(step), 1)
        assert oracle_mod.n_dm(r) == int(count)
        # The last trial stays inside the half-open range.
        last = oracle_mod.dm_value(r, int(count) - 1)
        assert float(lo) <= last < float(hi)


def test_eq4_narrow_band_approximation(oracle_mod):
    """Eq. 4: delay across a narrow channel ~ 8297.4e3 DM df / fc^3 [ms, MHz]."""
    for row in _golden("delay_law.txt"):
        if row[0] != "eq4":
            continue
        fc, df, dm = (float(v) for v in row[1:4])
        k_lo = oracle_mod.delay_coeff(fc - df / 2, 1e4)
        k_hi = oracle_mod.delay_coeff(fc + df / 2, 1e4)
        delay_ms = dm * (k_lo - k_hi) * 1e3
        approx_ms = 8297.4e3 * dm * df / fc ** 3
        # 8297.4 vs 2 * 4148.808 differ by 2.6e-5; (df/fc)^2 terms are tiny.
        assert delay_ms == pytest.approx(approx_ms, rel=5e-5)


def test_eq7_constant(oracle_mod):
    (row,) = [r for r in _golden("delay_law.txt") if r[0] == "eq7"]
    paper_const = float(row[1])
    f, fh = 1300.0, 1700.0
    k = oracle_mod.delay_coeff(f, fh)
    implied = k / (1 / f ** 2 - 1 / fh ** 2)
    assert implied == pytest.approx(paper_const, rel=2e-5)


def test_handbook_delay(oracle_mod):
    """Standard 4.15 ms DM (f/GHz)^-2 delay against infinite frequency."""
    for row in _golden("delay_law.txt"):
        if row[0] != "handbook":
            continue
        f_ghz, dm, ms = float(row[1]), float(row[2]), float(row[3])
        k = oracle_mod.delay_coeff(f_ghz * 1e3, math.inf)
        assert dm * k * 1e3 == pytest.approx(ms, rel=5e-3)


# --------------------------------------------------------------------------
# Shift table against exact rational arithmetic and its invariants.
# --------------------------------------------------------------------------
def _paper_scale_freqs(synth_mod):
    return synth_mod.channel_freqs(1670.0, 320.0, 8192)


def test_shift_table_exact_rational(oracle_mod, synth_mod):
    freqs = _paper_scale_freqs(synth_mod)
    r = (0.0, 409.6, 0.1, 1)
    table = oracle_mod.shift_table(freqs, 1670.0, 64e-6, r)
    assert table.shape == (4096, 8192)
    rng = np.random.default_rng(5)
    ds = np.concatenate([[0, 1, 4095], rng.integers(0, 4096, 40)])
    cs = np.concatenate([[0, 8191], rng.integers(0, 8192, 40)])
    ties = 0
    for d in ds:
        dm = oracle_mod.dm_value(r, int(d))
        assert dm == 0.0 + int(d) * 0.1
        for c in cs:
            n, dist = exact_shift(dm, freqs[c], 1670.0, 1, 64e-6)
            if dist < Fraction(1, 10 ** 9):
                ties += 1
                continue
            assert table[d, c] == n, (d, c)
    assert ties <= 2


def test_shift_table_invariants(oracle_mod, synth_mod):
    freqs = _paper_scale_freqs(synth_mod)
    r = (0.0, 409.6, 0.1, 1)
    t = oracle_mod.shift_table(freqs, 1670.0, 64e-6, r)
    assert np.all(t[0] == 0)                    # DM = 0: no delay anywhere
    assert np.all(np.diff(t, axis=0) >= 0)      # non-decreasing in DM
    assert np.all(np.diff(t, axis=1) >= 0)      # non-decreasing to lower frequency
    # s is proportional to DM up to the rounding: |s(d) - d * s_unit| <= 1
    k_low = oracle_mod.delay_coeff(freqs[-1], 1670.0)
    per_dm = k_low / 64e-6
    d = np.arange(4096)
    assert np.all(np.abs(t[:, -1] - d * 0.1 * per_dm) <= 0.5 + 1e-6)
    s_max, n_out = oracle_mod.extent(freqs, 1670.0, 64e-6, r, 262144)
    assert s_max == t.max() and n_out == 262144 - s_max


def test_tiny_config_extent(oracle_mod, synth_mod):
    freqs = synth_mod.channel_freqs(1500.0, 300.0, 64)
    r = (0.0, 64.0, 0.5, 1)
    assert oracle_mod.n_dm(r) == 128
    s_max, n_out = oracle_mod.extent(freqs, 1500.0, 64e-6, r, 8192)
    n, _ = exact_shift(63.5, freqs[-1], 1500.0, 1, 64e-6)
    assert s_max == n and n_out == 8192 - n


# --------------------------------------------------------------------------
# Direct transform: invariants and an independent brute force.
# --------------------------------------------------------------------------
def _brute(x, table, b, n_out):
    """Independent Eq. 3 with decimation, in Python integers / floats."""
    n_chan = x.shape[0]
    out = np.zeros((table.shape[0], n_out), dtype=np.float64)
    xs = x.astype(np.float64)
    for d in range(table.shape[0]):
        for t in range(n_out):
            acc = 0.0
            for c in range(n_chan):
                s = int(table[d, c])
                acc += xs[c, (t + s) * b:(t + s) * b + b].sum()
            out[d, t] = acc
    return out


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_random_small(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    n_chan = int(rng.integers(1, 9))
    f_ref = float(rng.uniform(300, 1500))
    freqs = np.sort(rng.uniform(0.6 * f_ref, f_ref, n_chan))[::-1]
    t_samp = float(rng.uniform(2e-4, 2e-3))
    ranges = []
    lo = 0.0
    for _ in range(int(rng.integers(1, 4))):
        step = float(rng.choice([0.25, 0.5, 1.0, 2.0]))
        n = int(rng.integers(1, 6))
        ranges.append((lo, lo + n * step, step, int(rng.choice([1, 2, 3]))))
        lo += n * step
    n_samp = 400
    dt = rng.choice([np.uint8, np.uint16, np.float32])
    if dt == np.float32:
        x = rng.standard_normal((n_chan, n_samp)).astype(np.float32)
    else:
        x = rng.integers(0, np.iinfo(dt).max + 1, (n_chan, n_samp)).astype(dt)
    planes = oracle_mod.forward(x, freqs, f_ref, t_samp, ranges)
    for r, y in zip(ranges, planes):
        lo_, hi_, step_, b = r
        n = oracle_mod.n_dm(r)
        table = np.zeros((n, n_chan), dtype=np.int64)
        for d in range(n):
            for c in range(n_chan):
                table[d, c] = exact_shift(Fraction(lo_) + d * Fraction(step_), freqs[c],
                                          f_ref, b, t_samp)[0]
        n_out = n_samp // b - table.max()
        assert y.shape == (n, n_out)
        ref = _brute(x, table, b, n_out)
        if dt == np.float32:
            np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-9)
        else:
            np.testing.assert_array_equal(y, ref)


def test_dm_zero_is_channel_sum(oracle_mod, synth_mod):
    freqs = synth_mod.channel_freqs(1500.0, 300.0, 64)
    x = synth_mod.filterbank(np.uint8, 64, 8192, 1000, 128, 16)
    (y,) = oracle_mod.forward(x, freqs, 1500.0, 64e-6, [(0.0, 64.0, 0.5, 1)])
    np.testing.assert_array_equal(y[0], x.astype(np.int64).sum(axis=0)[:y.shape[1]])


def test_reference_channel_is_a_copy(oracle_mod):
    """A channel at f_ref has no delay at any DM: every row copies it."""
    x = (np.arange(50) % 251).astype(np.uint8)[None, :]
    (y,) = oracle_mod.forward(x, [1000.0], 1000.0, 1e-3, [(0.0, 100.0, 10.0, 1)])
    for d in range(10):
        np.testing.assert_array_equal(y[d], x[0, :50])


def test_decimation_closed_form(oracle_mod):
    """Single reference channel, bin b: Y[0][t] = sum_{j<b} X[b t + j]."""
    x = (np.arange(103) * 37 % 65536).astype(np.uint16)[None, :]
    for b in (1, 2, 3, 4, 8):
        (y,) = oracle_mod.forward(x, [800.0], 800.0, 1e-3, [(0.0, 1.0, 1.0, b)])
        n = 103 // b
        np.testing.assert_array_equal(y[0], x[0, :n * b].astype(np.int64).reshape(n, b).sum(1))


def test_single_channel_pure_shift(oracle_mod):
    x = np.arange(300, dtype=np.float32)[None, :] * 0.5 + 1.0
    f, f_ref, ts = 700.0, 900.0, 1e-3
    r = (0.0, 10.0, 1.0, 1)
    (y,) = oracle_mod.forward(x, [f], f_ref, ts, [r])
    for d in range(10):
        s, _ = exact_shift(Fraction(d), f, f_ref, 1, ts)
        np.testing.assert_array_equal(y[d], x[0, s:s + y.shape[1]])


def test_impulse_response(oracle_mod, synth_mod):
    freqs = synth_mod.channel_freqs(1500.0, 300.0, 16)
    r = (0.0, 32.0, 1.0, 1)
    c0, t0 = 11, 700
    x = np.zeros((16, 1024), np.uint8)
    x[c0, t0] = 1
    (y,) = oracle_mod.forward(x, freqs, 1500.0, 64e-6, [r])
    for d in range(32):
        s, _ = exact_shift(Fraction(d), freqs[c0], 1500.0, 1, 64e-6)
        expect = np.zeros(y.shape[1])
        if 0 <= t0 - s < y.shape[1]:
            expect[t0 - s] = 1
        np.testing.assert_array_equal(y[d], expect)


def test_linearity_exact(oracle_mod, synth_mod):
    freqs = synth_mod.channel_freqs(1400.0, 300.0, 12)
    rng = np.random.default_rng(3)
    x1 = rng.integers(0, 1000, (12, 600)).astype(np.uint16)
    x2 = rng.integers(0, 1000, (12, 600)).astype(np.uint16)
    ranges = [(0.0, 20.0, 1.0, 1), (20.0, 40.0, 2.0, 2)]
    ya = oracle_mod.forward(x1, freqs, 1400.0, 1e-4, ranges)
    yb = oracle_mod.forward(x2, freqs, 1400.0, 1e-4, ranges)
    yc = oracle_mod.forward((3 * x1 + 5 * x2).astype(np.uint16), freqs, 1400.0, 1e-4, ranges)
    for a, b, c in zip(ya, yb, yc):
        np.testing.assert_array_equal(c, 3 * a + 5 * b)


def test_time_shift_equivariance(oracle_mod, synth_mod):
    freqs = synth_mod.channel_freqs(1400.0, 300.0, 8)
    x = synth_mod.filterbank(np.uint8, 8, 900, 7, 128, 16)
    r = (0.0, 30.0, 1.0, 1)
    (y,) = oracle_mod.forward(x, freqs, 1400.0, 1e-4, [r])
    k = 37
    (yk,) = oracle_mod.forward(np.ascontiguousarray(x[:, k:]), freqs, 1400.0, 1e-4, [r])
    np.testing.assert_array_equal(yk, y[:, k:k + yk.shape[1]])


def test_rows_and_window_match_full_plane(oracle_mod, synth_mod):
    freqs = synth_mod.channel_freqs(1400.0, 300.0, 8)
    x = synth_mod.filterbank(np.float32, 8, 500, 9, 0, 1)
    r = (1.0, 21.0, 0.5, 2)
    (y,) = oracle_mod.forward(x, freqs, 1400.0, 1e-4, [r])
    part = oracle_mod.forward_rows(x, freqs, 1400.0, 1e-4, r, [3, 0, 39], 5, 60)
    np.testing.assert_array_equal(part, y[[3, 0, 39], 5:60])


def test_pulse_recovery_tiny(oracle_mod, synth_mod):
    """An injected DM = 30 pulse is found at its DM with a high peak S/N.

    The paper's output comparison (Sec. 5.3) checks that the injected pulse's
    DM is recovered; the S/N threshold is this build's choice.
    """
    freqs = synth_mod.channel_freqs(1500.0, 300.0, 64)
    r = (0.0, 64.0, 0.5, 1)
    table = oracle_mod.shift_table(freqs, 1500.0, 64e-6, r)
    d_true, t0, w = 60, 3000, 4
    x = synth_mod.filterbank(np.uint8, 64, 8192, 1000, 128, 16,
                             pulses=[(t0 + table[d_true], w, 40.0)])
    (y,) = oracle_mod.forward(x, freqs, 1500.0, 64e-6, [r])
    box = np.stack([np.convolve(row, np.ones(w), mode="valid") for row in y])
    noise = box[:, : t0 - 200]
    med = np.median(noise)
    sigma = 1.4826 * np.median(np.abs(noise - med))
    snr = (box - med) / sigma
    d_best, t_best = np.unravel_index(np.argmax(snr), snr.shape)
    assert d_best == d_true and t_best == t0
    assert snr[d_best, t_best] >= 15.0
    # Boxcar widths: the injected width gives the best S/N at the true DM.
    best = []
    for ww in (1, 2, 4, 8, 16):
        b = np.convolve(y[d_true], np.ones(ww), mode="valid")
        nz = b[: t0 - 200]
        m = np.median(nz)
        best.append(((b.max() - m) / (1.4826 * np.median(np.abs(nz - m))), ww))
    assert max(best)[1] == w


# --------------------------------------------------------------------------
# Adjoint: the transpose of the forward map.
# --------------------------------------------------------------------------
def _tiny_plan(synth_mod):
    freqs = synth_mod.channel_freqs(1400.0, 300.0, 5)
    ranges = [(0.0, 6.0, 1.0, 1), (6.0, 14.0, 2.0, 2), (14.0, 20.0, 3.0, 3)]
    return freqs, 1400.0, 2e-3, ranges


def test_adjoint_explicit_matrix(oracle_mod, synth_mod):
    freqs, f_ref, ts, ranges = _tiny_plan(synth_mod)
    n_chan, n_samp = 5, 60
    cols = []
    for i in range(n_chan * n_samp):
        e = np.zeros(n_chan * n_samp, np.float32)
        e[i] = 1.0
        planes = oracle_mod.forward(e.reshape(n_chan, n_samp), freqs, f_ref, ts, ranges)
        cols.append(np.concatenate([p.ravel() for p in planes]))
    a = np.stack(cols, axis=1)  # [n_out_total][n_in]
    assert set(np.unique(a)) <= {0.0, 1.0}
    shapes = [p.shape for p in planes]
    rng = np.random.default_rng(1)
    ybar = rng.standard_normal(a.shape[0])
    parts, off = [], 0
    for s in shapes:
        parts.append(ybar[off:off + s[0] * s[1]].reshape(s))
        off += s[0] * s[1]
    xbar = oracle_mod.adjoint(parts, n_chan, n_samp, freqs, f_ref, ts, ranges)
    np.testing.assert_allclose(xbar.ravel(), a.T @ ybar, rtol=1e-13, atol=1e-12)


def test_adjoint_dot_product(oracle_mod, synth_mod):
    freqs = synth_mod.channel_freqs(1400.0, 300.0, 32)
    ranges = [(0.0, 40.0, 0.5, 1), (40.0, 80.0, 1.0, 2)]
    x = synth_mod.filterbank(np.float32, 32, 3000, 11, 0, 1)
    planes = oracle_mod.forward(x, freqs, 1400.0, 1e-4, ranges)
    rng = np.random.default_rng(2)
    ys = [rng.standard_normal(p.shape) for p in planes]
    lhs = sum(float(np.sum(p * y)) for p, y in zip(planes, ys))
    xbar = oracle_mod.adjoint(ys, 32, 3000, freqs, 1400.0, 1e-4, ranges)
    rhs = float(np.sum(x.astype(np.float64) * xbar))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_adjoint_finite_differences(oracle_mod, synth_mod):
    """Central differences of L = sum(Y * W) match the adjoint applied to W."""
    freqs, f_ref, ts, ranges = _tiny_plan(synth_mod)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((5, 60)).astype(np.float32)
    planes = oracle_mod.forward(x, freqs, f_ref, ts, ranges)
    ws = [rng.standard_normal(p.shape) for p in planes]
    grad = oracle_mod.adjoint(ws, 5, 60, freqs, f_ref, ts, ranges)

    def loss(xx):
        return sum(float(np.sum(p * w)) for p, w in
                   zip(oracle_mod.forward(xx, freqs, f_ref, ts, ranges), ws))

    h = 0.25  # exact in float32 for these magnitudes; L is linear
    for _ in range(20):
        c, t = int(rng.integers(0, 5)), int(rng.integers(0, 60))
        xp, xm = x.copy(), x.copy()
        xp[c, t] += h
        xm[c, t] -= h
        fd = (loss(xp) - loss(xm)) / (float(xp[c, t]) - float(xm[c, t]))
        assert fd == pytest.approx(grad[c, t], rel=1e-9, abs=1e-9)


def test_generator_reference_vectors(synth_mod):
    """splitmix64 seeded with 0: first output 0xE220A8397B1DCDAF (published)."""
    assert synth_mod.splitmix64(0, 1) == 0xE220A8397B1DCDAF
    zs = np.array([synth_mod.normal(123, i) for i in range(20000)])
    assert abs(zs.mean()) < 0.03 and abs(zs.std() - 1) < 0.03


def test_adjoint_channels_are_rows_of_full_adjoint(oracle_mod, synth_mod):
    freqs, f_ref, ts, ranges = _tiny_plan(synth_mod)
    rng = np.random.default_rng(8)
    planes = oracle_mod.forward(rng.standard_normal((5, 60)).astype(np.float32), freqs, f_ref, ts,
                                ranges)
    ys = [rng.standard_normal(p.shape) for p in planes]
    full = oracle_mod.adjoint(ys, 5, 60, freqs, f_ref, ts, ranges)
    part = oracle_mod.adjoint_channels(ys, 5, 60, freqs, f_ref, ts, ranges, [4, 0, 2])
    np.testing.assert_array_equal(part, full[[4, 0, 2]])


def test_transpose_pins(oracle_mod):
    """The front-end transpose: a hand-written 2 x 3 case, the involution, and
    a channel row equal to the strided column of the time-major array."""
    x = np.array([[1, 2, 3], [4, 5, 6]], dtype=np.uint8)  # 2 times x 3 channels
    np.testing.assert_array_equal(oracle_mod.transpose(x), [[1, 4], [2, 5], [3, 6]])
    rng = np.random.default_rng(5)
    y = rng.standard_normal((37, 11)).astype(np.float32)
    np.testing.assert_array_equal(oracle_mod.transpose(oracle_mod.transpose(y)), y)
    z = rng.integers(0, 65536, (50, 9)).astype(np.uint16)
    assert list(oracle_mod.transpose(z)[4]) == [int(z[t, 4]) for t in range(50)]


def test_packed4_nibble_order(oracle_mod):
    """4-bit input: byte 0x21 holds samples 1 (low nibble, earlier) then 2.
    With one trial DM of 0 the output is the channel sum of the samples."""
    data = np.array([[0x21, 0x43, 0x65], [0x10, 0x32, 0x54]], dtype=np.uint8)
    x = oracle_mod.Packed4(data, 6)
    freqs = np.array([1400.0, 1300.0])
    out = oracle_mod.forward(x, freqs, 1400.0, 1e-3, [(0.0, 0.5, 1.0, 1)])[0]
    np.testing.assert_array_equal(out, [[1 + 0, 2 + 1, 3 + 2, 4 + 3, 5 + 4, 6 + 5]])


def test_packed4_equals_unpacked_u8(oracle_mod, synth_mod):
    """The 4-bit path reads the same samples as the (pinned) 8-bit path on the
    unpacked values, with time binning and an odd sample count."""
    rng = np.random.default_rng(44)
    vals = rng.integers(0, 16, (23, 3002)).astype(np.uint8)
    packed = synth_mod.pack4(vals)
    freqs = synth_mod.channel_freqs(1500.0, 300.0, 23)
    ranges = [(0.0, 20.0, 0.5, 1), (20.0, 40.0, 1.0, 2), (40.0, 60.0, 2.0, 3)]
    n = 3001
    a = oracle_mod.forward(oracle_mod.Packed4(packed, n), freqs, 1500.0, 64e-6, ranges)
    b = oracle_mod.forward(np.ascontiguousarray(vals[:, :n]), freqs, 1500.0, 64e-6, ranges)
    for pa, pb in zip(a, b):
        np.testing.assert_array_equal(pa, pb)


def test_adjoint_is_a_forward_transform_of_padded_rows(oracle_mod, synth_mod):
    """The identity the CUDA adjoint is built on, checked in FP64 against the
    oracle transpose: per range, with P = s_max and the cotangent rows padded
    with P zeros on both sides, xbar_r[c][u] = sum_d Z[d][u + P - s(c, d)] --
    Eq. 3 on "channels" d at shifts P - s(c, d) for the channels taken in
    reverse order (shifts that grow with the reversed index) -- and the raw
    samples take the decimated sample floor(t / b)."""
    freqs = synth_mod.channel_freqs(1400.0, 300.0, 24)
    ranges = [(0.0, 30.0, 0.5, 1), (30.0, 60.0, 1.0, 2)]
    t_samp, n_samp = 1e-4, 1500
    rng = np.random.default_rng(12)
    want_planes = oracle_mod.forward(np.zeros((24, n_samp), np.float32), freqs, 1400.0, t_samp,
                                     ranges)
    ys = [rng.standard_normal(p.shape) for p in want_planes]
    want = oracle_mod.adjoint(ys, 24, n_samp, freqs, 1400.0, t_samp, ranges)
    got = np.zeros((24, n_samp))
    for r, y in zip(ranges, ys):
        s = oracle_mod.shift_table(freqs, 1400.0, t_samp, r).astype(np.int64)  # [d][c]
        n_dm, n_out = y.shape
        b = r[3]
        u_len = (n_samp - 1) // b + 1
        pad = int(s.max())
        z = np.zeros((n_dm, u_len + pad))
        z[:, pad:pad + n_out] = y
        # Reversed channel order: trial c' = n_chan - 1 - c, shifts pad - s.
        shifts_t = pad - s[:, ::-1]  # [d][c']
        assert np.all(shifts_t >= 0)
        # Increments along c' are the adjacent channels' delay differences (>= 0).
        assert np.all(np.diff(shifts_t, axis=1) >= 0)
        zc = np.zeros((24, u_len))
        for cp in range(24):
            for d in range(n_dm):
                zc[cp] += z[d, shifts_t[d, cp]:shifts_t[d, cp] + u_len]
        got += zc[::-1][:, np.arange(n_samp) // b]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
