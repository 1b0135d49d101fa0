"""Multi-rank bench aggregation on CPU: N gloo ranks as N independent
replicas; the whole-job time is the slowest rank's and the throughput counts
every rank's views (no data-path collective, only the timing reduction)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_all, value = bench.aggregate(100.0 + 25.0 * rank, world, "cpu")
    q.put((rank, ms_all, value))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replicas_take_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sys.path.insert(0, ROOT)
    import bench
    slow = 100.0 + 25.0 * (world - 1)
    for rank, ms_all, value in res:
        assert ms_all == slow
        assert value == pytest.approx(world * bench.N_VIEWS / (slow / 1000.0))


def test_single_rank_is_local_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(50.0, 1, "cpu") == (50.0, bench.N_VIEWS / 0.05)
