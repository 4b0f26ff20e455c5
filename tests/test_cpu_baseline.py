"""The tiled CPU baseline (bench.py's labelled second CPU number) against the
oracle: identical integer results, float within the usual bound."""
import numpy as np
import pytest

import cpu_baseline
import oracle
from synth import channel_freqs, filterbank


@pytest.mark.parametrize("dtype,n_chan,n_samp", [(np.uint8, 37, 5001), (np.uint16, 64, 4099),
                                                 (np.float32, 19, 3000), (np.uint8, 1, 2500)])
def test_tiled_cpu_equals_oracle(dtype, n_chan, n_samp):
    freqs = channel_freqs(1400.0, 300.0, n_chan)
    r = (0.0, 20.0, 0.3, 1)
    shifts = oracle.shift_table(freqs, 1400.0, 64e-6, r).astype(np.int32)
    s_max, n_out = oracle.extent(freqs, 1400.0, 64e-6, r, n_samp)
    mean, sd = (0.0, 1.0) if dtype == np.float32 else (100.0, 30.0)
    x = filterbank(dtype, n_chan, n_samp, 77, mean, sd)
    got = cpu_baseline.forward(x, shifts, n_out)
    ref = oracle.forward(x, freqs, 1400.0, 64e-6, [r])[0]
    if dtype == np.float32:
        ab = oracle.forward(x, freqs, 1400.0, 64e-6, [r], take_abs=True)[0]
        assert np.all(np.abs(got - ref) <= 1e-5 * ab + 1e-30)
    else:
        np.testing.assert_array_equal(got, ref)
