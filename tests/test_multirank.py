"""The benchmark's multi-rank aggregation on CPU (gloo, world size 2): the
job time is the slowest rank's, the value is all ranks' units over it."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_seconds = [2.0, 3.5][rank]
    slowest = bench.max_over_ranks(local_seconds, world, "cpu")
    value = bench.job_throughput(299 * 5, world, slowest)
    dist.barrier()
    q.put((rank, slowest, value))
    dist.destroy_process_group()


def test_two_ranks_max_time_and_weak_scaling_value():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in out:
        assert slowest == 3.5
        assert value == pytest.approx(299 * 5 * 2 / 3.5)


def test_single_rank_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, 1, "cpu") == 1.25
    assert bench.job_throughput(10, 1, 2.0) == 5.0
