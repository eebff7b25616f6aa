"""The multi-rank host logic of bench.py (replicas, max over ranks) with two gloo ranks on the CPU."""

from __future__ import annotations

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
    m = bench.max_over_ranks(ms, world, "cpu")
    v = bench.whole_job_value(1_000_000, 4, m, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, m, v))


def test_two_ranks_take_the_slowest_time():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's 15 ms; two replicas of 1 Mpix x 4 steps in 15 ms
    assert [o[1] for o in out] == [15.0, 15.0]
    assert all(abs(o[2] - 2 * 4.0 / 15e-3) < 1e-9 for o in out)


def test_one_rank_is_its_own_time():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert abs(bench.whole_job_value(429_670_400, 10, 92.0, 1) - 429.6704 * 10 / 0.092) < 1e-6
