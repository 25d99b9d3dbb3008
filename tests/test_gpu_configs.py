"""The small workloads run as stated, against the oracle and the exact log det."""
import numpy as np
import pytest

from gpu_util import cuda
from oracle import estimator, kernels, precond
from oracle.splitmix import rademacher_block
from paper_2405_03474_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def test_matern_n2048_d2_fp64_dense_against_oracle_and_cholesky():
    # n = 2048 points uniform in [0,1]^2, Matern-5/2, lengthscale 0.2, variance 1, noise 1e-2,
    # FP64 dense; r_3 with a rank-64 randomized-SVD preconditioner (5 subspace iterations,
    # Section 3's count) and 32 Rademacher probes; compared with the exact Cholesky log det.
    w = inputs.WORKLOADS["matern_n2048_d2"]
    n, d, s, r, q = w["n"], w["d"], w["probes"], w["rank"], w["power_iters"]
    X = inputs.points(n, d, w["dist"], seed=inputs.SEED_POINTS)
    k = api.Kernel(w["kind"], w["lengthscale"], w["variance"], w["noise"])
    M = kernels.kernel_matrix(X, w["kind"], w["lengthscale"], w["variance"], w["noise"])
    Ao, Do = precond.build(M, rademacher_block(inputs.SEED_SKETCH, n, r), q, w["noise"])
    F = precond.factors(Ao, Do)
    B = precond.operator_B(M, F)
    # the device's own FP64 build from the same sketch gives the same P
    Pg = api.Precond.build(cuda(X), k, r, power_iters=q, seed=inputs.SEED_SKETCH, precision="fp64")
    assert Pg.logdet_P == pytest.approx(F["logdet_P"], rel=1e-10)
    Z = inputs.rademacher(n, s, seed=inputs.SEED_PROBES)
    P = api.Precond.import_(Ao, Do, "fp64")
    res = api.logdet_estimate(cuda(X), k, precond=P, probes=cuda(Z), order=w["order"], num_probes=s,
                              precision="fp64", dense=True, rel_tol=1e-13, max_iters=3000, residual_check=True)
    est, per_probe, _ = estimator.estimate_converged(B, F["logdet_P"], Z.astype(np.float64), w["order"])
    assert res["logdet"] == pytest.approx(est, rel=1e-10)
    np.testing.assert_allclose(res["per_probe"], per_probe, rtol=1e-9)
    assert max(res["max_resid"][:w["order"]]) < 1e-11
    # against the exact value: the estimator's expectation is log det P + tr r_3(B), which
    # misses log det M by the exact r_3 bias; the rest is Hutchinson noise
    exact = estimator.logdet_exact(M)
    bias = estimator.rk_bias(B, w["order"])
    print("matern_n2048_d2: estimate %.6f +- %.6f, exact (Cholesky) %.6f, r_3 bias %.3g, rel err %.2e"
          % (res["logdet"], res["std_err"], exact, bias, abs(res["logdet"] - exact) / abs(exact)))
    assert abs(res["logdet"] + bias - exact) < 5 * res["std_err"] + 1e-9 * abs(exact)
