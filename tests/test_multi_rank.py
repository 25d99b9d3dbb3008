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


# ---- one estimate split over ranks (probe blocks per rank, one all-gather of the brackets)

def _problem_for_shards():
    import numpy as np
    from oracle import estimator, kernels, precond
    from oracle.splitmix import rademacher_block
    from paper_2405_03474_gb300 import inputs
    n, S, t = 300, 8, 12
    X = inputs.points(n, 2, "uniform", seed=40)
    M = kernels.kernel_matrix(X, kernels.MATERN52, 0.25, 1.0, 1e-2)
    F = precond.factors(*precond.build(M, rademacher_block(2, n, 12), 1, 1e-2))
    B = precond.operator_B(M, F)
    Z = rademacher_block(41, n, S)  # the probe stream: column j is probe j
    return estimator, F, B, Z, t, np


def _shard_rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2405_03474_gb300 import sharded
        estimator, F, B, Z, t, np = _problem_for_shards()
        col0, count = sharded.shard_of(Z.shape[1], rank, world)
        Zr = Z[:, col0:col0 + count]
        # this rank's brackets, from the oracle (the CPU stands in for the device's solves)
        _, per_probe, _ = estimator.estimate_converged(B, F["logdet_P"], Zr, 3)
        slq, _ = estimator.estimate_slq(B, F["logdet_P"], Zr, t)
        local = {"per_probe": per_probe, "logdet_P": F["logdet_P"], "slq_logdet": slq, "iters": 10 + rank,
                 "converged": True, "final_rel_resid": 1e-3 * (rank + 1),
                 "max_resid": [0.1 * (rank + 1), 0.05, 0.01 * (2 - rank), 0.0, 0.0]}
        res = sharded.combine_sharded(local)
        out.put((rank, res["logdet"], res["trace_est"], res["std_err"], res["slq_logdet"], res["iters"],
                 res["final_rel_resid"], list(res["max_resid"]), list(res["per_probe"])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_one_estimate_matches_single_process():
    import numpy as np
    from paper_2405_03474_gb300 import api
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=10) for _ in range(world))
    estimator, F, B, Z, t, _ = _problem_for_shards()
    # one process over all probes: the oracle's Algorithm 1 output and SLQ
    est, per_probe, _ = estimator.estimate_converged(B, F["logdet_P"], Z, 3)
    slq, _ = estimator.estimate_slq(B, F["logdet_P"], Z, t)
    one = api.ld_combine(per_probe, F["logdet_P"])  # the library's own single-call combination
    std = np.std(per_probe, ddof=1) / np.sqrt(len(per_probe))
    for rank, logdet, trace, std_err, slq_r, iters, final_rel, max_resid, brackets in got:
        np.testing.assert_array_equal(brackets, per_probe)  # gathered in probe order
        assert logdet == one["logdet"] and std_err == one["std_err"]
        assert logdet == pytest.approx(est, rel=1e-14)
        assert trace == pytest.approx(est - F["logdet_P"], rel=1e-14)
        assert std_err == pytest.approx(std, rel=1e-13)
        assert slq_r == pytest.approx(slq, rel=1e-14)
        assert iters == 11 and final_rel == pytest.approx(2e-3)
        np.testing.assert_allclose(max_resid, [0.2, 0.05, 0.02, 0.0, 0.0])


def test_shard_columns_cover_the_probe_stream_once():
    from paper_2405_03474_gb300 import sharded
    for S, world in ((16, 1), (16, 2), (16, 4), (48, 8)):
        cols = []
        for r in range(world):
            c0, cnt = sharded.shard_of(S, r, world)
            cols += list(range(c0, c0 + cnt))
        assert cols == list(range(S))
    with pytest.raises(ValueError):
        sharded.shard_of(10, 0, 4)
