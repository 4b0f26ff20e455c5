"""The persistent batch (one launch over many uneven beams, CUDA graph).

Each beam's output in the batch must equal its output alone (bit for bit: the
same tile arithmetic runs in both), the alone output must match the oracle,
and a replayed graph must follow new input contents.
"""
import numpy as np
import pytest

import oracle
from paper_2311_05341_gb300 import batch as ddb
from synth import channel_freqs, filterbank

from gpu_util import assert_float_parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _beams():
    """Uneven beams: channel counts, dtypes, sampling times and DM plans differ."""
    out = []
    f = channel_freqs(1520.0, 310.0, 256)
    out.append(ddb.BeamSpec(f, 1520.0, 64e-6, [(0.0, 25.6, 0.1, 1)], "u8", 9000))
    f = channel_freqs(1400.0, 300.0, 300)
    out.append(ddb.BeamSpec(f, 1400.0, 64e-6, [(0.0, 6.4, 0.05, 1), (6.4, 12.8, 0.1, 1)], "u8",
                            7001))
    f = channel_freqs(1670.0, 320.0, 512)
    out.append(ddb.BeamSpec(f, 1670.0, 54.6e-6, [(0.0, 19.2, 0.2, 1)], "u16", 6000))
    f = channel_freqs(400.0, 100.0, 96)
    out.append(ddb.BeamSpec(f, 400.0, 327.68e-6, [(0.0, 6.4, 0.2, 1)], "f32", 5000))
    f = channel_freqs(1500.0, 300.0, 130)
    out.append(ddb.BeamSpec(f, 1500.0, 128e-6, [(0.0, 12.0, 0.2, 1)], "f32", 4001))
    return out


_NOISE = {"u8": (np.uint8, 128, 40), "u16": (np.uint16, 32768, 9000),
          "f32": (np.float32, 0.0, 1.0)}


def _fill(runner, seed0):
    hosts = []
    for i, (b, x) in enumerate(zip(runner.beams, runner.inputs)):
        npdt, mean, sd = _NOISE[b.dtype]
        h = filterbank(npdt, len(b.freqs), b.n_samp, seed0 + i, mean, sd)
        x[:, : b.n_samp].copy_(torch.from_numpy(h).to(x.device))
        hosts.append(h)
    torch.cuda.synchronize()
    return hosts


def _check_oracle(b, host, planes):
    ref = oracle.forward(host, b.freqs, b.f_ref, b.t_samp, b.ranges)
    for r, (g, o) in enumerate(zip(planes, ref)):
        g = g.cpu().numpy()
        if b.dtype == "f32":
            ab = oracle.forward(host, b.freqs, b.f_ref, b.t_samp, b.ranges, take_abs=True)[r]
            assert_float_parity(g, o, ab, f"range {r}")
        else:
            np.testing.assert_array_equal(g, o)


@pytest.mark.parametrize("autotune", [True, False])
def test_batch_equals_alone_and_oracle(autotune):
    runner = ddb.BatchRunner(_beams(), autotune=autotune, graph=True)
    assert runner.n_jobs == 6
    if autotune:
        # (tile, shape) per range: the pattern or packed tile in a table shape,
        # or an offset tile.
        assert all(t[0] in ("pattern", "packed", 4, 2, 1) for shp in runner.shapes
                   for t in shp)
    else:
        assert all(dr in ddb.BATCH_SHAPES for shp in runner.shapes for dr in shp)
    if not autotune:
        # The first feasible tile: the pattern tile, except for the steep
        # 96-channel float beam (offset tile): both persistent families run.
        assert [shp[0] for shp in runner.shapes] == ["pattern", "pattern", "pattern", 1,
                                                     "pattern"]
        # At least the u8, u16 and f32 pattern variants plus the offset family.
        assert runner.n_launches >= 4
    hosts = _fill(runner, 600)
    runner.run()
    torch.cuda.synchronize()
    runner.status()
    batched = [o.clone() for o in runner.outputs]
    runner.run_per_beam()
    torch.cuda.synchronize()
    for i, (bo, o) in enumerate(zip(batched, runner.outputs)):
        assert torch.equal(bo, o), f"beam {i} differs between batch and alone"
    for i, b in enumerate(runner.beams):
        _check_oracle(b, hosts[i], runner.planes(i))


def test_graph_replay_follows_new_inputs():
    runner = ddb.BatchRunner(_beams()[:3], autotune=False, graph=True)
    _fill(runner, 700)
    runner.run()
    hosts = _fill(runner, 800)
    for o in runner.outputs:
        o.fill_(-1)
    runner.run()
    runner.run()
    torch.cuda.synchronize()
    for i, b in enumerate(runner.beams):
        _check_oracle(b, hosts[i], runner.planes(i))


def test_batch_with_4bit_beams():
    """Packed 4-bit beams in a batch with an 8-bit one: batch == alone == oracle."""
    from synth import filterbank4
    beams = [ddb.BeamSpec(channel_freqs(1520.0, 310.0, 200), 1520.0, 64e-6,
                          [(0.0, 25.6, 0.1, 1)], "u4", 9000),
             ddb.BeamSpec(channel_freqs(1400.0, 300.0, 96), 1400.0, 64e-6,
                          [(0.0, 12.8, 0.1, 1), (12.8, 25.6, 0.2, 2)], "u4", 7001),
             ddb.BeamSpec(channel_freqs(1670.0, 320.0, 128), 1670.0, 64e-6,
                          [(0.0, 12.8, 0.1, 1)], "u8", 6000)]
    runner = ddb.BatchRunner(beams, autotune=False, graph=True)
    hosts = []
    for i, (b, x) in enumerate(zip(runner.beams, runner.inputs)):
        if b.dtype == "u4":
            h = filterbank4(len(b.freqs), b.n_samp, 900 + i, 8, 4, row_bytes=x.shape[1])
            x.copy_(torch.from_numpy(h).to(x.device))
            hosts.append(oracle.Packed4(h, b.n_samp))
        else:
            h = filterbank(np.uint8, len(b.freqs), b.n_samp, 900 + i, 128, 40)
            x[:, : b.n_samp].copy_(torch.from_numpy(h).to(x.device))
            hosts.append(h)
    torch.cuda.synchronize()
    runner.run()
    torch.cuda.synchronize()
    runner.status()
    batched = [o.clone() for o in runner.outputs]
    runner.run_per_beam()
    torch.cuda.synchronize()
    for i, (bo, o) in enumerate(zip(batched, runner.outputs)):
        assert torch.equal(bo, o), f"beam {i} differs between batch and alone"
    for i, b in enumerate(runner.beams):
        _check_oracle(b, hosts[i], runner.planes(i))


def test_batch_packed_and_shape_tiles():
    """Beams on the packed tile (uint8, uint16 and float pairs, each packed by
    the batch run) and on explicit pattern shapes of the tuning table, in one
    batch: batch == alone == oracle."""
    from paper_2311_05341_gb300 import tile_shapes
    shapes = tile_shapes()
    tune = [i for i, s in enumerate(shapes) if not s["automatic"] and s["channel_pairs"]]
    f2 = [i for i, s in enumerate(shapes) if s["float_pairs"]]
    beams = [ddb.BeamSpec(channel_freqs(1520.0, 310.0, 256), 1520.0, 64e-6,
                          [(0.0, 25.6, 0.1, 1)], "u8", 9000),
             ddb.BeamSpec(channel_freqs(1670.0, 320.0, 300), 1670.0, 54.6e-6,
                          [(0.0, 19.2, 0.2, 1)], "u16", 7001),
             ddb.BeamSpec(channel_freqs(400.0, 100.0, 96), 400.0, 327.68e-6,
                          [(0.0, 3.2, 0.05, 1)], "f32", 5000),
             ddb.BeamSpec(channel_freqs(1400.0, 300.0, 130), 1400.0, 64e-6,
                          [(0.0, 6.4, 0.05, 1), (6.4, 12.8, 0.1, 2)], "u8", 6000)]
    tiles = [[("packed", -1)], [("packed", tune[0])], [("packed", f2[-1])],
             [("pattern", tune[1]), ("pattern", -1)]]
    runner = ddb.BatchRunner(beams, autotune=False, graph=True, tiles=tiles)
    assert runner.n_launches >= 3 + 3  # three packing launches and the persistent ones
    hosts = _fill(runner, 990)
    runner.run()
    torch.cuda.synchronize()
    runner.status()
    batched = [o.clone() for o in runner.outputs]
    runner.run_per_beam()
    torch.cuda.synchronize()
    for i, (bo, o) in enumerate(zip(batched, runner.outputs)):
        assert torch.equal(bo, o), f"beam {i} differs between batch and alone"
    for i, b in enumerate(runner.beams):
        _check_oracle(b, hosts[i], runner.planes(i))
