"""Stored dense M = K + noise I (the rbf_n65536_d3 workload keeps M in HBM) against the oracle."""
import numpy as np
import pytest

from gpu_util import cuda, host, relerr, torch
from oracle import estimator, kernels, precond
from oracle.splitmix import rademacher_block
from paper_2405_03474_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [api.RBF, api.MATERN52])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-14), ("fp32", 1e-6)])
def test_materialize_and_product_match_oracle(kind, prec, tol):
    n, d, c = 1000, 3, 24
    X = inputs.points(n, d, "normal", seed=1)
    k = api.Kernel(kind, 0.5, 1.3, 1e-3)
    M = api.ld_dense_materialize(cuda(X), k, prec)
    Mo = kernels.kernel_matrix(X, kind, 0.5, 1.3, 1e-3)
    assert np.abs(host(M) - Mo).max() < tol * 10
    V = inputs.gaussian(n, c, seed=2)
    dt = torch.float64 if prec == "fp64" else torch.float32
    W = api.ld_dense_kz(M, cuda(V, dt), prec)
    assert relerr(host(W), Mo @ V) < tol * 10


@pytest.mark.parametrize("order", [1, 3, 5])
def test_dense_estimate_equals_matrix_free_and_oracle(order):
    n, s = 2000, 8
    X = inputs.points(n, 3, "normal", seed=0)
    k = api.Kernel(api.RBF, 0.5, 1.0, 1e-2)
    M = kernels.kernel_matrix(X, kernels.RBF, 0.5, 1.0, 1e-2)
    A, D = precond.build(M, rademacher_block(2, n, 32), 2, 1e-2)
    F = precond.factors(A, D)
    Z = inputs.rademacher(n, s, seed=1)
    P = api.Precond.import_(A, D, "fp64")
    common = dict(precond=P, probes=cuda(Z), order=order, num_probes=s, precision="fp64", rel_tol=1e-12,
                  max_iters=3000)
    rd = api.logdet_estimate(cuda(X), k, dense=True, **common)
    rf = api.logdet_estimate(cuda(X), k, dense=False, **common)
    assert rd["logdet"] == pytest.approx(rf["logdet"], rel=1e-12)
    est, _, _ = estimator.estimate_converged(precond.operator_B(M, F), F["logdet_P"], Z.astype(np.float64), order)
    assert rd["logdet"] == pytest.approx(est, rel=1e-10)


def test_dense_fp32_estimate_within_1e4():
    n, s = 4096, 16
    X = inputs.points(n, 3, "normal", seed=0)
    k = api.Kernel(api.RBF, 0.5, 1.0, 1e-3)
    M = kernels.kernel_matrix(X, kernels.RBF, 0.5, 1.0, 1e-3)
    A, D = precond.build(M, rademacher_block(2, n, 64), 2, 1e-3)
    F = precond.factors(A, D)
    Z = inputs.rademacher(n, s, seed=1)
    P = api.Precond.import_(A, D, "fp32")
    r = api.logdet_estimate(cuda(X), k, precond=P, probes=cuda(Z), order=3, num_probes=s, precision="fp32",
                            rel_tol=1e-6, max_iters=3000, dense=True)
    est, _, _ = estimator.estimate_converged(precond.operator_B(M, F), F["logdet_P"], Z.astype(np.float64), 3)
    assert r["logdet"] == pytest.approx(est, rel=1e-4)
