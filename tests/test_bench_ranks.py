"""The multi-rank host logic of bench.py on CPU (gloo, two ranks): the job's
time is the slowest rank's, and the job's value counts every rank's units
(replicas of the single-graph colouring; no data-path collective)."""
import os
import socket

import pytest


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    m = bench.max_over_ranks(ms, world)
    v = bench.job_value(1000, 4, world, m)
    out.put((rank, m, v))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 15.0  # the slowest rank's time, seen by both
        assert abs(v - 1000 * 4 * 2 / 0.015) < 1e-6 * v


def test_single_rank_is_the_identity():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_value(10, 2, 1, 1000.0) == 20.0
