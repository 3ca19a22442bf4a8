"""The benchmark's multi-rank path on the CPU (gloo, world size 2): each rank
is an independent replica; the slowest rank's time sets the job's time and
the job's rate counts every rank's queries."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 + 5.0 * rank                 # rank 1 is the slower replica
    total = bench.max_over_ranks(torch, dist, local_ms, world, "cpu")
    out[rank] = (total, bench.job_rate(world, 1000, total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_count_all_queries():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    total, rate = res[0]
    assert total == 15.0
    assert abs(rate - 2 * 1000 / 0.015) < 1e-6


def test_one_process_is_its_own_job():
    import bench
    assert bench.max_over_ranks(torch, None, 12.5, 1, "cpu") == 12.5
    assert bench.job_rate(1, 500, 2.0) == 250000.0
