"""Multi-GPU is replicas only: N independent processes, no data-path
collective.  The one exchange is the timing reduction in bench.py (max over
ranks); it is checked here with two gloo ranks on the CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    # Rank r processed 1000 units in 2 + r seconds.
    value, seconds = bench.replica_throughput(1000.0, 2.0 + rank, "cpu")
    q.put((rank, value, seconds))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # Both ranks see the job time of the slower rank and 2 x 1000 units over it.
    for rank, value, seconds in got:
        assert seconds == 3.0
        assert value == pytest.approx(2000.0 / 3.0)


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(500.0, 2.0, "cpu") == (250.0, 2.0)
