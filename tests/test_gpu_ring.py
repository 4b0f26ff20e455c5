"""The packed ring of dd_run_scratch: ranges with a packed copy run in time
segments from two packed slots (packing overlapped with the kernels on the
plan's side streams), against the oracle (bit-exact for integer input,
1e-5 x sum_c |X| for float32) and against the other ways of running the same
tables (full copy, unpacking the input)."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from paper_2311_05341_gb300 import _lib
from synth import channel_freqs, filterbank, filterbank4

from gpu_util import assert_float_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


_NOISE = {"u8": (np.uint8, 200, 80), "u16": (np.uint16, 40000, 12000),
          "f32": (np.float32, 0.0, 1.0)}


def _input(dtype, n_chan, n_samp, seed):
    """The oracle's input and the device rows (16-byte row stride; 4-bit: two
    samples per byte, the earlier in the low nibble)."""
    if dtype == "u4":
        data = filterbank4(n_chan, n_samp, seed, 8.0, 4.0, row_bytes=(n_samp + 31) // 32 * 16)
        return oracle.Packed4(data, n_samp), torch.from_numpy(data).cuda()
    npdt, mean, sd = _NOISE[dtype]
    x = filterbank(npdt, n_chan, n_samp, seed, mean, sd)
    per = 16 // x.itemsize
    stride = (n_samp + per - 1) // per * per
    xd = torch.zeros((n_chan, stride), dtype=getattr(torch, str(x.dtype)), device="cuda")
    xd[:, :n_samp] = torch.from_numpy(x).cuda()
    return x, xd


def _check(dtype, got, ref, ref_abs, what):
    if dtype == "f32":
        assert_float_parity(got, ref, ref_abs, what)
    else:
        np.testing.assert_array_equal(got, ref, err_msg=what)


@pytest.mark.parametrize("dtype,seed", [("u8", 0), ("u8", 1), ("u8", 2), ("u4", 3), ("u16", 4),
                                        ("u16", 5)])
def test_ring_matches_oracle_and_full_copy(dtype, seed):
    """Several segment counts (2 up to more segments than time tiles), the
    full copy and the unpacking kernel: every output against the oracle."""
    rng = np.random.default_rng(6100 + seed)
    n_chan = int(rng.choice([61, 256, 300]))
    f_high = 1500.0
    freqs = channel_freqs(f_high, 300.0, n_chan)
    k_low = oracle.delay_coeff(freqs[-1], f_high) / 64e-6
    step = float(rng.uniform(0.4, 1.6)) / k_low
    n_dm = int(rng.choice([64, 100, 130]))
    ranges = [(0.0, n_dm * step, step, 1)]
    s_max = oracle.extent(freqs, f_high, 64e-6, ranges[0], 10 ** 9)[0]
    n_samp = int(s_max + rng.choice([9000, 20001, 30017]))
    x, xd = _input(dtype, n_chan, n_samp, 6200 + seed)
    ref = oracle.forward(x, freqs, f_high, 64e-6, ranges)[0]
    plan = dd.Plan(freqs, f_high, 64e-6, ranges, dtype)
    info = plan.info(n_samp)
    assert info["packed_copy"] == [True] and info["tile_dms"] == [_lib.DD_TILE_PATTERN]
    full = plan.packed_scratch_bytes(n_samp, 1)
    for segments in (0, 1, 2, 3, 7, 16, 64, 256):
        if segments > 1:
            ring = plan.packed_scratch_bytes(n_samp, segments)
            assert 0 < ring
        got = plan.run(xd, n_samp=n_samp, segments=segments)[0].cpu().numpy()
        _check(dtype, got, ref, None, f"segments {segments}")
    assert full == n_chan * ((n_samp + 3) // 4 * 4) * 4


def test_ring_multi_range_plan():
    """A bin-1 range in the ring beside binned ranges that read the input
    (uint8 at bins 2 and 4: no packed copy) on the caller's stream."""
    freqs = channel_freqs(1400.0, 300.0, 200)
    ranges = [(0.0, 8.0, 0.05, 1), (8.0, 20.0, 0.1, 2), (20.0, 40.0, 0.25, 4)]
    n_samp = 48000
    x, xd = _input("u8", 200, n_samp, 6300)
    ref = oracle.forward(x, freqs, 1400.0, 64e-6, ranges)
    plan = dd.Plan(freqs, 1400.0, 64e-6, ranges, "u8")
    assert plan.info(n_samp)["packed_copy"] == [True, False, False]
    for segments in (0, 5, 16):
        got = plan.run(xd, n_samp=n_samp, segments=segments)
        for r, (g, o) in enumerate(zip(got, ref)):
            np.testing.assert_array_equal(g.cpu().numpy(), o, err_msg=f"{segments}, range {r}")


def test_ring_explicit_packed_float_pairs():
    """DD_TILE_PACKED float32 (64-bit words of two floats) from the ring."""
    freqs = channel_freqs(1500.0, 300.0, 130)
    ranges = [(0.0, 20.0, 0.2, 1)]
    n_samp = 40000
    x, xd = _input("f32", 130, n_samp, 6400)
    ref = oracle.forward(x, freqs, 1500.0, 64e-6, ranges)[0]
    ab = oracle.forward(x, freqs, 1500.0, 64e-6, ranges, take_abs=True)[0]
    plan = dd.Plan(freqs, 1500.0, 64e-6, ranges, "f32")
    assert plan.info(n_samp)["packed_copy"] == [False]  # the automatic float tile has none
    plan.set_tile(0, "packed")
    assert plan.info(n_samp)["packed_copy"] == [True]
    for segments in (1, 4, 16):
        got = plan.run(xd, n_samp=n_samp, segments=segments)[0].cpu().numpy()
        assert_float_parity(got, ref, ab, f"segments {segments}")


def test_ring_on_a_side_stream_back_to_back():
    """Calls on a non-default stream, back to back with different inputs into
    different outputs: each call's ring work stays ordered on its stream."""
    freqs = channel_freqs(1500.0, 300.0, 128)
    ranges = [(0.0, 12.8, 0.1, 1)]
    n_samp = 60000
    plan = dd.Plan(freqs, 1500.0, 64e-6, ranges, "u8")
    xs = [_input("u8", 128, n_samp, 6500 + i) for i in range(3)]
    st = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(st):
        for _, xd in xs:
            outs.append(plan.run(xd, n_samp=n_samp, stream=st, segments=8)[0])
    st.synchronize()
    for (x, _), o in zip(xs, outs):
        np.testing.assert_array_equal(o.cpu().numpy(),
                                      oracle.forward(x, freqs, 1500.0, 64e-6, ranges)[0])


def test_ring_scratch_query_and_refusals():
    freqs = channel_freqs(1500.0, 300.0, 64)
    lib = _lib.load()
    # Binned packed copies have no ring.
    plan = dd.Plan(freqs, 1500.0, 64e-6, [(0.0, 6.4, 0.1, 2)], "u8")
    plan.set_tile(0, "packed")
    n = ctypes.c_size_t(0)
    assert lib.dd_plan_packed_scratch_bytes(plan.handle, 20000, 8, ctypes.byref(n)) == \
        _lib.DD_ERR_UNSUPPORTED
    assert lib.dd_plan_packed_scratch_bytes(plan.handle, 20000, 1, ctypes.byref(n)) == _lib.DD_OK
    assert n.value == plan.input_scratch_bytes(20000) > 0
    for bad in (0, 257):
        assert lib.dd_plan_packed_scratch_bytes(plan.handle, 20000, bad, ctypes.byref(n)) == \
            _lib.DD_ERR_INVALID_ARG
    # The binned explicit copy still runs with too little scratch for the ring
    # refused: it needs its full copy.
    x, xd = _input("u8", 64, 20000, 6600)
    out = plan.empty_output(20000)
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    st = lib.dd_run_scratch(plan.handle, xd.data_ptr(), xd.stride(0), 20000, out.data_ptr(),
                            small.data_ptr(), small.numel(), None)
    assert st == _lib.DD_ERR_BUDGET


def test_two_copies_fall_back_to_full_copy_and_unpacking():
    """An explicit packed range at another pair distance (H = 19) beside an
    automatic range (H = 23) needs two copies, so no ring: scratch for the
    explicit copy alone runs that range packed and the automatic one unpacking
    the input; scratch for both copies runs both packed.  Every output against
    the oracle."""
    freqs = channel_freqs(1500.0, 300.0, 160)
    ranges = [(0.0, 6.4, 0.05, 1), (6.4, 12.8, 0.05, 1)]
    n_samp = 30000
    x, xd = _input("u8", 160, n_samp, 6700)
    ref = oracle.forward(x, freqs, 1500.0, 64e-6, ranges)
    plan = dd.Plan(freqs, 1500.0, 64e-6, ranges, "u8")
    shapes = dd.tile_shapes()
    h19 = [i for i, s in enumerate(shapes) if s["words_per_lane"] == 19 and s["channel_pairs"]
           and not s["float_pairs"]][0]
    plan.set_tile_shape(1, "packed", h19)
    assert plan.info(n_samp)["packed_copy"] == [True, True]
    with pytest.raises(dd.DDError):
        plan.packed_scratch_bytes(n_samp, 8)
    lib = _lib.load()
    out = plan.empty_output(n_samp)
    for nbytes in (plan.input_scratch_bytes(n_samp), plan.packed_scratch_bytes(n_samp, 1)):
        sc = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        _lib.check(lib.dd_run_scratch(plan.handle, xd.data_ptr(), xd.stride(0), n_samp,
                                      out.data_ptr(), sc.data_ptr(), nbytes, None))
        torch.cuda.synchronize()
        for r, (g, o) in enumerate(zip(plan.split(out, n_samp), ref)):
            np.testing.assert_array_equal(g.cpu().numpy(), o, err_msg=f"{nbytes} B, range {r}")
