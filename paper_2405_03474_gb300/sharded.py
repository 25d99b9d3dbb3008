"""One estimate split over the ranks of a torch.distributed group.

Algorithm 1's per-probe work (steps 2-3: the Krylov solves of each probe) is
independent from probe to probe; only its output, log det P plus the Hutchinson
mean over the probes, joins them.  So the probe blocks of one estimate shard over
ranks with no exchange on the data path: rank r runs the S / R probes in stream
columns [r S / R, (r + 1) S / R) (device-drawn probes, option ``probe_col0``)
against the same preconditioner, and one all-gather of the per-probe brackets
(S fp64 values) plus a few per-rank scalars gives every rank the estimate that
one process running all S probes gives.  The brackets are joined by the
library's ``ld_combine`` in probe order.

Argument marshalling and the collective only; every step of the estimate runs
in the library.
"""
import numpy as np
import torch
import torch.distributed as dist

from . import api

# per-rank scalars gathered beside the brackets
_N_STATS = 5 + 5  # logdet_P, slq_logdet, iters, converged, final_rel_resid, max_resid[5]


def shard_of(num_probes, rank, world):
    """(first stream column, count) of the probes rank `rank` of `world` runs."""
    if num_probes % world:
        raise ValueError("num_probes (%d) must be a multiple of the world size (%d)" % (num_probes, world))
    per = num_probes // world
    return rank * per, per


def _gather(t, world, group):
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    return torch.stack(parts).cpu().numpy()


def combine_sharded(local, group=None, device=None):
    """Join the per-rank results of one sharded estimate.

    ``local`` is the dict ``api.logdet_estimate`` returned on this rank (its
    ``per_probe`` are this rank's brackets in probe order).  Every rank must hold
    the same number of probes.  Returns the estimate of all probes: log det,
    trace, std-err from the library's ``ld_combine`` of the gathered brackets;
    log det P and SLQ as the mean over ranks (equal when the ranks share P);
    iterations, final residual and residual check as the max over ranks;
    converged if every rank converged."""
    world = dist.get_world_size(group)
    if device is None:
        device = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    br = torch.as_tensor(np.asarray(local["per_probe"], dtype=np.float64), device=device)
    stats = np.zeros(_N_STATS)
    stats[0] = local["logdet_P"]
    stats[1] = local["slq_logdet"]
    stats[2] = local["iters"]
    stats[3] = 1.0 if local["converged"] else 0.0
    stats[4] = local["final_rel_resid"]
    stats[5:10] = np.asarray(local["max_resid"], dtype=np.float64)[:5]
    all_br = _gather(br, world, group).reshape(-1)
    st = _gather(torch.as_tensor(stats, device=device), world, group)
    out = api.ld_combine(all_br, float(np.mean(st[:, 0])))
    out.update({
        "slq_logdet": float(np.mean(st[:, 1])),
        "iters": int(st[:, 2].max()),
        "converged": bool(st[:, 3].min() > 0.5),
        "final_rel_resid": float(st[:, 4].max()),
        "max_resid": list(st[:, 5:10].max(axis=0)),
        "per_probe": all_br,
        "ranks": world,
    })
    return out


def logdet_estimate_sharded(X, kernel, precond=None, num_probes=16, group=None, **opts):
    """One estimate of log det M whose probes are split over the ranks of `group`.

    Each rank passes its own copy of the points and the same preconditioner (built
    from the same seed, or imported from the same factors); the probes are drawn on
    the device from the SplitMix64 stream (``seed``, ``probe_kind``), rank r taking
    its columns by ``probe_col0``.  Returns ``combine_sharded``'s dict on every
    rank."""
    if "probes" in opts or "probe_col0" in opts:
        raise ValueError("sharded estimates draw their probes on the device by stream column")
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    col0, count = shard_of(num_probes, rank, world)
    ppb = opts.pop("probes_per_block", None) or count
    if count % ppb:
        raise ValueError("each rank's %d probes must be a multiple of probes_per_block (%d)" % (count, ppb))
    local = api.logdet_estimate(X, kernel, precond=precond, num_probes=count, probes_per_block=ppb,
                                probe_col0=col0, **opts)
    return combine_sharded(local, group)
