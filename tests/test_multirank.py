"""Host logic of the multi-GPU benchmark with two gloo ranks on the CPU.

Each rank runs an independent replica: distinct seeds, no collective on the data path.  The
job's time is the max over ranks, and the whole-job rate counts every rank's sites."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 7.5 * rank  # a per-rank time
        got = bench.max_over_ranks(ms, world, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(42, rank) + bench.batch_seed_offset(rank))
        rate = bench.whole_job_rate(1000, 4, world, got)
        out.put((rank, got, seeds, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_distinct_seeds():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, seeds, rate in res:
        assert got == pytest.approx(17.5)  # the slower rank's time, seen by every rank
        assert len(set(seeds)) == world   # independent replicas
        assert rate == pytest.approx(1000 * 4 * world / 17.5e-3)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.rank_seed(7, 0) == 7 and bench.batch_seed_offset(0) == 0
