"""Writes estimate_matern_n32768_d4.txt: Algorithm 1 (Section 2) run by the CPU FP64
oracle, matrix-free, on n = 2^15 Matern-5/2 points in [0,1]^4 (lengthscale 0.1,
variance 1, noise 1e-2: the large matrix-free workload's kernel at a size the oracle
finishes in minutes).

The estimate is taken literally: t = 20 Lanczos steps per probe with full
reorthogonalisation (``estimator.estimate_lanczos_block``), a Thomas solve per
shift of r_3 (Table 1), the Hutchinson mean over 16 Rademacher probes, plus
log det P of a rank-128 randomized truncated-SVD preconditioner (one subspace
iteration, Rademacher sketch from SplitMix64 seed 2).  The kernel matrix is never
formed: every product is ``kernels.kz_matfree``.  The SLQ values of the same
tridiagonals (Section 3's comparison method) are stored beside the estimate.

Only ``oracle/`` and the seeded input generators are called.  Usage:

    python tests/golden/make_estimate_matern_n32768_d4.py

(about 3 minutes on 8 host cores).  The GPU test rebuilds the same
preconditioner with ``problem()`` below and checks its log det P against the
stored value before comparing the estimates.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import estimator, kernels, precond  # noqa: E402
from oracle.splitmix import rademacher_block  # noqa: E402
from paper_2405_03474_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "estimate_matern_n32768_d4.txt")
CONFIG = dict(n=1 << 15, d=4, dist="uniform", kind=kernels.MATERN52, lengthscale=0.1, variance=1.0,
              noise=1e-2, order=3, rank=128, power_iters=1, probes=16, t=20, seed_points=0,
              seed_probes=1, seed_sketch=2)


def problem(cfg=CONFIG):
    """Points, probes and the oracle's preconditioner of the stored case.

    Returns X (n-by-d), Z (n-by-s float64 signs), A, D (P = D + A A^T), the split
    factor F and the matrix-free product V -> (K + noise I) V."""
    n, d = cfg["n"], cfg["d"]
    X = inputs.points(n, d, cfg["dist"], seed=cfg["seed_points"])
    Z = inputs.rademacher(n, cfg["probes"], seed=cfg["seed_probes"]).astype(np.float64)

    def matmul(V):
        return kernels.kz_matfree(X, V, cfg["kind"], cfg["lengthscale"], cfg["variance"], cfg["noise"])

    Omega = rademacher_block(cfg["seed_sketch"], n, cfg["rank"])
    A = precond.rsvd(matmul, Omega, cfg["power_iters"])
    # diag(M) = k(0) + noise for every point
    diagM = np.full(n, float(kernels.kernel_of_r2(0.0, cfg["kind"], cfg["lengthscale"], cfg["variance"]))
                    + cfg["noise"])
    D = precond.diag_residual(diagM, A, cfg["noise"])
    F = precond.factors(A, D)
    return X, Z, A, D, F, matmul


def read(path=OUT):
    """The stored values as a dict (floats; 'bracket' and 'slq_form' as arrays)."""
    vals, br, sl = {}, {}, {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, val = line.split(None, 1)
        if key.startswith("bracket_"):
            br[int(key[8:])] = float(val)
        elif key.startswith("slq_form_"):
            sl[int(key[9:])] = float(val)
        else:
            vals[key] = float(val)
    vals["bracket"] = np.array([br[i] for i in sorted(br)])
    vals["slq_form"] = np.array([sl[i] for i in sorted(sl)])
    return vals


def main():
    cfg = CONFIG
    t0 = time.time()
    X, Z, A, D, F, matmul = problem(cfg)
    t1 = time.time()
    est, per_probe, q, tri = estimator.estimate_lanczos_block(precond.operator_B_apply(matmul, F),
                                                               F["logdet_P"], Z, cfg["order"], cfg["t"])
    slq = np.array([estimator.slq_form(a, bt, float(Z[:, i] @ Z[:, i])) for i, (a, bt) in enumerate(tri)])
    t2 = time.time()
    with open(OUT, "w") as f:
        f.write("# Algorithm 1 (Section 2) by the CPU FP64 oracle, matrix-free, literal form: t Lanczos steps\n")
        f.write("# per probe (full reorthogonalisation), Thomas per shift of r_3 (Table 1), Hutchinson mean.\n")
        f.write("# Written by: python tests/golden/make_estimate_matern_n32768_d4.py  (oracle/ only;\n")
        f.write("# preconditioner %.0f s, estimate %.0f s on %d host cores)\n" % (t1 - t0, t2 - t1, os.cpu_count()))
        for key in ("n", "d", "kind", "lengthscale", "variance", "noise", "order", "rank", "power_iters",
                    "probes", "t", "seed_points", "seed_probes", "seed_sketch"):
            f.write("%s %r\n" % (key, cfg[key]))
        f.write("logdet_P %r\n" % F["logdet_P"])
        f.write("estimate %r\n" % est)
        f.write("slq %r\n" % float(F["logdet_P"] + np.mean(slq)))
        for i, v in enumerate(per_probe):
            f.write("bracket_%d %r\n" % (i, float(v)))
        for i, v in enumerate(slq):
            f.write("slq_form_%d %r\n" % (i, float(v)))
    print("wrote %s: logdet_P %.15g estimate %.15g (%.0f s + %.0f s)" % (OUT, F["logdet_P"], est, t1 - t0, t2 - t1))


if __name__ == "__main__":
    main()
