"""The bench's multi-rank host logic on two CPU ranks (gloo): each rank draws its
own probes, the job time is the slowest rank's, the value counts every rank's
estimates.  The ranks run the same helpers the timed run uses, with no GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 1000.0 * (rank + 1) + 0.25  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(local_ms, world, "cpu")
        dist.barrier()
        out.put((rank, bench.rank_probe_seed(rank), ms_max, bench.job_value(world, 3, ms_max)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_bookkeeping():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=10) for _ in range(world))
    seeds = [g[1] for g in got]
    assert len(set(seeds)) == world  # independent probes per rank
    for _, _, ms_max, value in got:
        assert ms_max == pytest.approx(2000.25)  # max over ranks, seen by every rank
        assert value == pytest.approx(world * 3 / 2.00025)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_value(1, 2, 500.0) == pytest.approx(4.0)
