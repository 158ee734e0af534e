"""The multi-GPU path of the benchmark is replicas only (one solve does not shard): each
rank solves its own replica, no data-path collective, and the job time is the maximum
over ranks.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sec = [3.0, 5.0][rank]  # rank 1 is the slowest
        m = bench.max_over_ranks(sec, world, device="cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.replica_seed(rank))
        rate = bench.job_rate(4, m, world)
        out.put((rank, m, seeds, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, seeds, rate in res:
        assert m == 5.0                  # the slowest rank's time
        assert seeds == [0, 1]           # distinct replicas
        assert rate == pytest.approx(2 * 4 / 5.0)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_rate(3, 1.5, 1) == 2.0
