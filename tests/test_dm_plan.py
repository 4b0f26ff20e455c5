"""DM plans from a smearing tolerance (dd_plan_dm_ranges).

Checked by brute force against the paper's own expressions rather than the
planner's: the intra-channel smear of Eq. 4, the across-band delay of Eq. 1 as
computed by the oracle, and the nearest trial of each sampled DM."""
import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from paper_2311_05341_gb300 import _lib
from synth import channel_freqs


def _check_plan(freqs, t_samp, dm_max, tol, width, max_bin, max_ranges):
    ranges = dd.dm_ranges(freqs, t_samp, dm_max, tol, width, max_bin, max_ranges)
    assert 1 <= len(ranges) <= max_ranges
    assert ranges[0][0] == 0.0 and ranges[-1][1] >= dm_max
    f_lo, f_hi = float(freqs.min()), float(freqs.max())
    df = (f_hi - f_lo) / (len(freqs) - 1)
    f_c = 0.5 * (f_lo + f_hi)
    # Across-band delay per unit DM from the oracle's Eq. 1.
    k_band = oracle.delay_coeff(f_lo, f_hi)
    prev_bin = 1
    for i, (lo, hi, step, b) in enumerate(ranges):
        if i:
            assert lo == pytest.approx(ranges[i - 1][1], rel=1e-12)
        assert step > 0 and hi > lo
        assert b >= prev_bin and b <= max_bin and (b & (b - 1)) == 0
        prev_bin = b
        n = int(round((hi - lo) / step))
        assert lo + n * step == pytest.approx(hi, rel=1e-9)
        # Sampled DMs of the range: the nearest trial broadens a pulse by at
        # most a factor tol.
        for dm in np.linspace(lo, min(hi, dm_max), 257)[:-1]:
            trials = lo + step * np.arange(n)
            if i + 1 < len(ranges):  # the next range's first trial
                trials = np.append(trials, ranges[i + 1][0])
            delta = float(np.min(np.abs(trials - dm)))
            t_chan = 8297.4e3 * dm * df / f_c ** 3 * 1e-3  # Eq. 4, ms -> s
            w = np.sqrt((b * t_samp) ** 2 + t_chan ** 2 + width ** 2)
            smear = delta * k_band
            assert np.sqrt(w ** 2 + smear ** 2) <= tol * w * (1 + 1e-9)
    return ranges


@pytest.mark.parametrize("f_top,bw,t_samp,dm_max", [(1550.0, 300.0, 64e-6, 3000.0),
                                                    (900.0, 200.0, 128e-6, 2000.0),
                                                    (500.0, 200.0, 256e-6, 1500.0)])
def test_plans_meet_the_tolerance(f_top, bw, t_samp, dm_max):
    freqs = channel_freqs(f_top, bw, 4096)
    ranges = _check_plan(freqs, t_samp, dm_max, 1.25, 0.0, 16, 16)
    assert len(ranges) >= 3  # the step grows and binning starts at high DM
    assert ranges[-1][3] > 1


def test_single_range_and_width():
    freqs = channel_freqs(1400.0, 300.0, 1024)
    (lo, hi, step, b), = _check_plan(freqs, 64e-6, 500.0, 1.25, 0.0, 1, 1)
    assert b == 1 and hi >= 500.0
    # A wider intrinsic pulse allows a coarser first step.
    wide = _check_plan(freqs, 64e-6, 500.0, 1.25, 1e-3, 16, 16)
    assert wide[0][2] > step


def test_plan_feeds_the_planner():
    freqs = channel_freqs(1550.0, 300.0, 256)
    ranges = dd.dm_ranges(freqs, 64e-6, 1000.0)
    plan = dd.Plan(freqs, 1550.0, 64e-6, ranges, "u8", upload=False)
    info = plan.info(1 << 20)
    assert info["n_ranges"] == len(ranges)
    assert all(n > 0 for n in info["n_out"])


@pytest.mark.parametrize("kw", [dict(tol=1.0), dict(dm_max=0.0), dict(t_samp=0.0),
                                dict(max_bin=0), dict(max_ranges=0)])
def test_bad_arguments(kw):
    args = dict(freqs=channel_freqs(1400.0, 300.0, 64), t_samp=64e-6, dm_max=100.0)
    args.update(kw)
    with pytest.raises(dd.DDError) as ei:
        dd.dm_ranges(**args)
    assert ei.value.status == _lib.DD_ERR_INVALID_ARG
