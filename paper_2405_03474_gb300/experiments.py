"""Accuracy experiments of Section 3 with this library's estimator.

``d_sweep``: the sweep over the point dimension d at fixed n (the paper's
Figure on errors against d, n = 20,000): points N(0, I_d), amplitude and
lengthscale 1, s = 35 Rademacher probes, t = 20 Lanczos steps, a rank-25
randomized-SVD preconditioner with 5 iterations (Section 3's parameters).  For
each d it reports |estimate - log det M| for r_1, r_3, r_5 and for stochastic
Lanczos quadrature computed from the same tridiagonals.  The reference log det M
is a float64 Cholesky of the stored matrix on the GPU (``torch.linalg.cholesky``),
used only as ground truth here.  The paper does not state the noise variance; it
is an argument (default 1e-2, our reading).

Run: ``python -m paper_2405_03474_gb300.experiments --n 20000 --dims 1 2 3 5 8 12 16 20``
"""
import argparse
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
            probes=35, t=20, rank=25, power_iters=5, precision="fp64", seed=0):
    rows = []
    for kind in kinds:
        for d in dims:
            X = torch.as_tensor(inputs.points(n, d, "normal", seed=seed)).cuda()
            kern = api.Kernel(kind, 1.0, 1.0, noise)
            exact = exact_logdet(X, kern)
            P = api.Precond.build(X, kern, rank, power_iters=power_iters, seed=inputs.SEED_SKETCH,
                                  precision="fp64" if precision == "fp64" else "fp32")
            row = {"kernel": "rbf" if kind == api.RBF else "matern52", "d": d, "n": n, "exact": exact}
            for order in (1, 3, 5):
                r = api.logdet_estimate(X, kern, precond=P, order=order, num_probes=probes, fixed_iters=t,
                                        max_iters=t, precision=precision, seed=inputs.SEED_PROBES)
                row["err_r%d" % order] = abs(r["logdet"] - exact)
                if order == 3:
                    row["err_slq"] = abs(r["slq_logdet"] - exact)
            P.free()
            rows.append(row)
            print(json.dumps(row), flush=True)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--dims", type=int, nargs="+", default=[1, 2, 3, 5, 8, 12, 16, 20])
    ap.add_argument("--noise", type=float, default=1e-2)
    ap.add_argument("--precision", default="fp64")
    args = ap.parse_args()
    d_sweep(n=args.n, dims=tuple(args.dims), noise=args.noise, precision=args.precision)


if __name__ == "__main__":
    main()
