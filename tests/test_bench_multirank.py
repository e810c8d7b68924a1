"""The multi-rank (replica) aggregation of bench.py on two gloo ranks on CPU: the whole-job
rate is every rank's units over the slowest rank's time."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one: 200 ms
    rate, slow = bench.whole_job_rate(local_ms, 1e6)
    q.put((rank, rate, slow))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, slow in out:
        assert slow == 200.0
        assert rate == pytest.approx(2 * 1e6 / 0.2)


def test_single_process_rate_without_process_group():
    sys.path.insert(0, ROOT)
    import bench
    rate, slow = bench.whole_job_rate(50.0, 1e6)
    assert slow == 50.0 and rate == pytest.approx(2e7)
