"""Accuracy experiments of Section 3 with this library's estimator.

``d_sweep``: the sweep over the point dimension d at fixed n (the paper's
Figure on errors against d, n = 20,000): points N(0, I_d), amplitude and
lengthscale 1, s = 35 Rademacher probes, t = 20 Lanczos steps, a rank-25
randomized-SVD preconditioner with 5 iterations (Section 3's parameters).  For
each d it reports |estimate - log det M| for r_1, r_3, r_5 and for stochastic
Lanczos quadrature computed from the same tridiagonals.  The reference log det M
is a float64 Cholesky of the stored matrix on the GPU (``torch.linalg.cholesky``),
used only as ground truth here.  The paper does not state the noise variance; it
is an argument (default 1e-2, our reading).  The probes of point set k use the
SplitMix64 seed 1 + 1000 k, independent of the sketch's seed 2 (probes equal to
the sketch's columns would lie in the preconditioner's subspace and bias the
trace estimate).

Run: ``python -m paper_2405_03474_gb300.experiments --n 20000 --dims 1 2 3 5 8 12 16 20 --seeds 4``
"""
import argparse
import itertools
import json

import torch

from . import api, inputs


def exact_logdet(X, kernel):
    M = api.ld_dense_materialize(X, kernel, "fp64")
    L = torch.linalg.cholesky(M)
    val = 2.0 * torch.log(torch.diagonal(L)).sum().item()
    del M, L
    return val


def d_sweep(n=20000, dims=(1, 2, 3, 5, 8, 12, 16, 20), kinds=(api.RBF, api.MATERN52), noise=1e-2,
            probes=35, t=20, rank=25, power_iters=5, precision="fp64", seeds=(0,)):
    """One row per (kernel, d, point seed); ``summarise`` averages them over seeds."""
    rows = []
    for kind, d, seed in itertools.product(kinds, dims, seeds):
        X = torch.as_tensor(inputs.points(n, d, "normal", seed=seed)).cuda()
        kern = api.Kernel(kind, 1.0, 1.0, noise)
        exact = exact_logdet(X, kern)
        P = api.Precond.build(X, kern, rank, power_iters=power_iters, seed=inputs.SEED_SKETCH,
                              precision="fp64" if precision == "fp64" else "fp32")
        row = {"kernel": "rbf" if kind == api.RBF else "matern52", "d": d, "n": n, "seed": seed,
               "exact": exact}
        for order in (1, 3, 5):
            r = api.logdet_estimate(X, kern, precond=P, order=order, num_probes=probes, fixed_iters=t,
                                    max_iters=t, precision=precision, seed=inputs.SEED_PROBES + 1000 * seed)
            row["err_r%d" % order] = abs(r["logdet"] - exact)
            if order == 3:
                row["err_slq"] = abs(r["slq_logdet"] - exact)
        P.free()
        rows.append(row)
        print(json.dumps(row), flush=True)
    return rows


def summarise(rows):
    """Mean absolute errors per (kernel, d) over the seeds."""
    out = {}
    for r in rows:
        key = (r["kernel"], r["d"])
        acc = out.setdefault(key, {"kernel": r["kernel"], "d": r["d"], "count": 0})
        acc["count"] += 1
        for k in ("err_r1", "err_r3", "err_r5", "err_slq"):
            acc[k] = acc.get(k, 0.0) + r[k]
    for acc in out.values():
        for k in ("err_r1", "err_r3", "err_r5", "err_slq"):
            acc[k] /= acc["count"]
    return list(out.values())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--dims", type=int, nargs="+", default=[1, 2, 3, 5, 8, 12, 16, 20])
    ap.add_argument("--noise", type=float, default=1e-2)
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--seeds", type=int, default=1, help="point sets per (kernel, d)")
    args = ap.parse_args()
    rows = d_sweep(n=args.n, dims=tuple(args.dims), noise=args.noise, precision=args.precision,
                   seeds=tuple(range(args.seeds)))
    for acc in summarise(rows):
        print(json.dumps({"mean_over_seeds": acc}), flush=True)


if __name__ == "__main__":
    main()
