"""The N > 1 path of bench.py on CPU: ranks as gloo processes (world size 2). Replicas share no
data; the job's time is the slowest rank's and the job's throughput is N x the per-rank units
over that time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        out[rank] = bench.max_over_ranks(ms, dist)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 15.0
    assert bench.job_rate(30_192_037, world, out[0]) == pytest.approx(2 * 30_192_037 / 0.015)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(100, 1, 2.0) == pytest.approx(50_000.0)
