"""Oracle parity at the stated shapes of the batched and streaming workloads.

The batched workload (24 uint8 beams of 1024 channels x 131072 samples, 8
uint16 beams of 4096 channels x 65536 samples at 54.6 us, 4 float32 beams of
336 channels x 32768 samples at 327.68 us) runs through the persistent batch
launch exactly as the benchmark builds it (autotuned tiles, CUDA graph); every
16th DM row of every beam, plus the rows of its injected pulse, is compared at
full length with the oracle's direct transform (Eq. 3, Algorithm 1): bit-exact
for the integer beams, |err| <= 1e-5 sum_c |X| for the float beams.

The streaming workload (4096-channel uint8 beams, 65536-sample chunks, the
four-range decimated plan to DM 2000 at bin 8) runs two beams of three chunks
each through the streaming server, interleaved so that their work overlaps on
the device; every kept output of every 16th DM row of every range is compared
with the oracle's transform of the concatenated stream.
"""
import numpy as np
import pytest

import oracle
from paper_2311_05341_gb300 import batch as ddb
from paper_2311_05341_gb300 import stream as dds
from synth import workloads

from gpu_util import assert_float_parity, oracle_input

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rows(n, every=16, extra=()):
    return sorted(set(range(0, n, every)) | {n - 1} | {int(e) for e in extra})


def _compare_rows(beam, x, plane, r, rows, what):
    got = plane[torch.tensor(rows, device=plane.device)].cpu().numpy()
    ref = oracle.forward_rows(x, beam.freqs, beam.f_high, beam.t_samp, beam.ranges[r], rows)
    assert got.shape == ref.shape, what
    if beam.dtype == "f32":
        ab = oracle.forward_rows(x, beam.freqs, beam.f_high, beam.t_samp, beam.ranges[r], rows,
                                 take_abs=True)
        assert_float_parity(got, ref, ab, what)
    else:
        np.testing.assert_array_equal(got, ref, err_msg=what)


def test_batched_workload_against_oracle():
    beams = workloads.batched()
    specs = [ddb.BeamSpec(b.freqs, b.f_high, b.t_samp, b.ranges, b.dtype, b.n_samp)
             for b in beams]
    runner = ddb.BatchRunner(specs, autotune=True, graph=True)
    assert runner.n_jobs == 36
    for b, xd in zip(beams, runner.inputs):
        x, _, _, _ = oracle_input(b)
        xd[:, : b.n_samp].copy_(torch.from_numpy(x).to(xd.device))
    torch.cuda.synchronize()
    runner.run()
    torch.cuda.synchronize()
    runner.status()
    batched = [o.clone() for o in runner.outputs]
    # The plain per-beam path gives the same outputs, element for element.
    runner.run_per_beam()
    torch.cuda.synchronize()
    for i, (bo, o) in enumerate(zip(batched, runner.outputs)):
        assert torch.equal(bo, o), f"beam {i} ({beams[i].name}) differs from its own dd_run"
    for i, b in enumerate(beams):
        x, _, n_dm, n_out = oracle_input(b)  # regenerated: same seed, same samples
        plane = runner.plans[i].split(batched[i], b.n_samp)[0]
        assert tuple(plane.shape) == (n_dm[0], n_out[0])
        pulses = [p[1] for p in workloads.resolve_pulses(b, n_dm, n_out)]
        _compare_rows(b, x, plane, 0, _rows(n_dm[0], extra=pulses), b.name)


def test_stream_workload_against_oracle():
    chunk, n_chunks = 65536, 3
    n_samp = chunk * n_chunks
    beams = [workloads.stream_beam(i, n_samp) for i in range(2)]
    data = {}
    for i, b in enumerate(beams):
        x, _, _, _ = oracle_input(b)
        data[i] = x
    spec = dds.StreamSpec(beams[0].freqs, beams[0].f_high, beams[0].t_samp, beams[0].ranges,
                          "u8")
    srv = dds.StreamServer(chunk, 64 << 30, keep_outputs=True)
    for i in data:
        assert srv.request(i, spec)
    for k in range(n_chunks):  # interleaved: the beams' work overlaps on the device
        for i, x in data.items():
            c = torch.from_numpy(np.ascontiguousarray(x[:, k * chunk:(k + 1) * chunk]))
            srv.submit(i, c.pin_memory())
        srv.pump()
    srv.drain()
    assert srv.stats()["chunks"] == n_chunks * len(data)
    plan = srv._plan(spec)
    ov = dds.overlap_for(plan, spec.ranges)
    for i, b in enumerate(beams):
        kept = srv.outputs(srv.beams[i])
        for r, rr in enumerate(b.ranges):
            n = (n_samp - ov) // rr[3]
            assert kept[r].shape == (oracle.n_dm(rr), n)
            rows = _rows(kept[r].shape[0])
            ref = oracle.forward_rows(data[i], b.freqs, b.f_high, b.t_samp, rr, rows, 0, n)
            np.testing.assert_array_equal(kept[r][rows], ref, err_msg=f"beam {i} range {r}")
