"""Streaming server: chunked == one-shot, alone == in the mix, HBM admission.

A beam's stream is cut into chunks; the server keeps the max-delay overlap on
the device and emits chunk / bin new outputs per range per chunk.  Those must
equal the same samples of one dd_run over the concatenated stream (bit for
bit, uint8), whether the beam runs alone or mixed with other beams whose work
overlaps on the device, and beams beyond the HBM budget wait for admission.
"""
import numpy as np
import pytest

import oracle
import paper_2311_05341_gb300 as dd
from paper_2311_05341_gb300 import stream as dds
from synth import channel_freqs, filterbank

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CHUNK = 8192
N_CHUNKS = 5
RANGES = [(0.0, 15.0, 0.1, 1), (15.0, 30.0, 0.2, 2), (30.0, 60.0, 0.5, 4), (60.0, 100.0, 1.0, 8)]


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _spec(n_chan=256):
    return dds.StreamSpec(channel_freqs(1670.0, 320.0, n_chan), 1670.0, 64e-6, RANGES, "u8")


def _stream_data(seed, n_chan=256):
    return filterbank(np.uint8, n_chan, CHUNK * N_CHUNKS, seed, 128, 40)


def _chunks(x):
    return [torch.from_numpy(np.ascontiguousarray(x[:, k * CHUNK:(k + 1) * CHUNK])).pin_memory()
            for k in range(N_CHUNKS)]


def _one_shot(spec, x):
    plan = dd.Plan(spec.freqs, spec.f_ref, spec.t_samp, spec.ranges, "u8")
    planes = plan.run(torch.from_numpy(x).cuda())
    return [p.cpu().numpy() for p in planes], plan


def _run_server(streams, budget, order):
    """streams: {beam_id: (spec, chunks)}; order: list of beam ids, one chunk each."""
    srv = dds.StreamServer(CHUNK, budget, keep_outputs=True)
    for bid, (spec, _) in streams.items():
        srv.request(bid, spec)
    sent = {bid: 0 for bid in streams}
    done = {}
    for bid in order:
        srv.submit(bid, streams[bid][1][sent[bid]])
        sent[bid] += 1
        srv.pump()
        if sent[bid] == N_CHUNKS:
            # Stream ended: wait for its chunks, then leave and admit waiters.
            while any(j.beam == bid for j in list(srv.queue) + srv.inflight):
                srv.pump(block=True)
            done[bid] = srv.outputs(srv.release(bid))
    srv.drain()
    return done, srv


def test_chunked_equals_one_shot_and_oracle():
    spec = _spec()
    x = _stream_data(500)
    ref, plan = _one_shot(spec, x)
    done, srv = _run_server({0: (spec, _chunks(x))}, 1 << 34, [0] * N_CHUNKS)
    got = done[0]
    ov = dds.overlap_for(plan, RANGES)
    for r, (g, o) in enumerate(zip(got, ref)):
        b = RANGES[r][3]
        n = (N_CHUNKS * CHUNK - ov) // b
        assert g.shape[1] == n and o.shape[1] >= n
        np.testing.assert_array_equal(g, o[:, :n], err_msg=f"range {r}")
    # And against the oracle directly on a few rows of each range.
    for r, rr in enumerate(RANGES):
        rows = [0, got[r].shape[0] // 2, got[r].shape[0] - 1]
        n = got[r].shape[1]
        o = oracle.forward_rows(x, spec.freqs, spec.f_ref, spec.t_samp, rr, rows, 0, n)
        np.testing.assert_array_equal(got[r][rows], o)
    assert srv.stats()["chunks"] == N_CHUNKS


def test_alone_equals_mixed_with_admission():
    specs = {0: _spec(256), 1: _spec(256), 2: _spec(128)}
    data = {b: _stream_data(600 + b, len(specs[b].freqs)) for b in specs}
    streams = {b: (specs[b], _chunks(data[b])) for b in specs}
    alone, _ = _run_server({0: streams[0]}, 1 << 34, [0] * N_CHUNKS)
    probe = dds.StreamServer(CHUNK, 1 << 34)
    need = [probe.beam_bytes(specs[b]) for b in specs]
    slots = max(probe.slots_bytes(specs[b]) for b in specs)  # shared packed-copy scratch
    budget = slots + need[0] + need[1] + need[2] // 2  # the third beam must wait
    srv = dds.StreamServer(CHUNK, budget, keep_outputs=True)
    assert srv.request(0, specs[0]) and srv.request(1, specs[1])
    assert not srv.request(2, specs[2]) and not srv.is_admitted(2)
    # Interleave 0 and 1 (their work overlaps on the device), then 2 after 0 leaves.
    order = [0, 1] * N_CHUNKS + [2] * N_CHUNKS
    mixed, srv2 = _run_server(streams, budget, order)
    for r in range(len(RANGES)):
        np.testing.assert_array_equal(mixed[0][r], alone[0][r])
    # Beam 2's result also equals its own one-shot transform.
    ref, plan = _one_shot(specs[2], data[2])
    for r, (g, o) in enumerate(zip(mixed[2], ref)):
        np.testing.assert_array_equal(g, o[:, : g.shape[1]])
    st = srv2.stats()
    assert st["chunks"] == 3 * N_CHUNKS and st["rejected"] == 0


def test_chunked_4bit_equals_one_shot():
    """Packed 4-bit chunks (two samples per byte) through the server equal one
    dd_run over the concatenated packed stream and the oracle's 4-bit path."""
    from synth import filterbank4
    spec = dds.StreamSpec(channel_freqs(1670.0, 320.0, 192), 1670.0, 64e-6, RANGES, "u4")
    x = filterbank4(192, CHUNK * N_CHUNKS, 700, 8, 4)  # [192][CHUNK * N_CHUNKS / 2] bytes
    half = CHUNK // 2
    chunks = [torch.from_numpy(np.ascontiguousarray(x[:, k * half:(k + 1) * half])).pin_memory()
              for k in range(N_CHUNKS)]
    done, srv = _run_server({0: (spec, chunks)}, 1 << 34, [0] * N_CHUNKS)
    plan = dd.Plan(spec.freqs, spec.f_ref, spec.t_samp, spec.ranges, "u4")
    ref = [p.cpu().numpy() for p in plan.run(torch.from_numpy(x).cuda(),
                                              n_samp=CHUNK * N_CHUNKS)]
    got = done[0]
    for r, (g, o) in enumerate(zip(got, ref)):
        np.testing.assert_array_equal(g, o[:, : g.shape[1]], err_msg=f"range {r}")
    rows = [0, got[0].shape[0] - 1]
    o = oracle.forward_rows(oracle.Packed4(x, CHUNK * N_CHUNKS), spec.freqs, spec.f_ref,
                            spec.t_samp, RANGES[0], rows, 0, got[0].shape[1])
    np.testing.assert_array_equal(got[0][rows], o)


def test_snapshot_restore_equals_uninterrupted():
    """A beam checkpointed between chunks and resumed on a new server gives the
    same outputs as the uninterrupted stream (and the one-shot transform)."""
    spec = _spec(192)
    x = _stream_data(650, 192)
    chunks = _chunks(x)
    whole, _ = _run_server({0: (spec, chunks)}, 1 << 34, [0] * N_CHUNKS)
    first = dds.StreamServer(CHUNK, 1 << 34, keep_outputs=True)
    assert first.request(0, spec)
    for k in range(2):
        first.submit(0, chunks[k])
    first.drain()
    state = first.snapshot(0)
    part1 = first.outputs(first.release(0))
    second = dds.StreamServer(CHUNK, 1 << 34, keep_outputs=True)
    assert second.restore(0, state)
    for k in range(2, N_CHUNKS):
        second.submit(0, chunks[k])
    second.drain()
    part2 = second.outputs(second.beams[0])
    for r in range(len(RANGES)):
        resumed = np.concatenate([part1[r], part2[r]], axis=1)
        np.testing.assert_array_equal(resumed, whole[0][r], err_msg=f"range {r}")
    ref, _ = _one_shot(spec, x)
    for r, (g, o) in enumerate(zip(whole[0], ref)):
        np.testing.assert_array_equal(g, o[:, : g.shape[1]], err_msg=f"range {r}")


def test_window_outputs_equal_full_run():
    """dd_run_window's first n_keep outputs of every range equal dd_run's (the
    packed tile and the plain tiles alike)."""
    spec = _spec(256)
    x = _stream_data(660)
    n = x.shape[1]
    for packed in (False, True):
        plan = dd.Plan(spec.freqs, spec.f_ref, spec.t_samp, spec.ranges, "u8")
        if packed:
            plan.set_tile(0, "packed")
        xd = torch.from_numpy(x).cuda()
        full = [p.cpu().numpy() for p in plan.run(xd)]
        keep = [max(1, f.shape[1] // 3 + 5 * r) for r, f in enumerate(full)]
        win = [p.cpu().numpy() for p in plan.run_window(xd, keep)]
        for r, (f, w) in enumerate(zip(full, win)):
            assert w.shape == (f.shape[0], keep[r])
            np.testing.assert_array_equal(w, f[:, : keep[r]], err_msg=f"range {r}")
        with pytest.raises(dd.DDError):
            plan.run_window(xd, [f.shape[1] + 1 for f in full])
    assert n > 0
