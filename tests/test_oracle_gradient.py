"""Pins for oracle/gradient.py: central finite differences of the oracle's own
log det functions (exact and estimator with P and probes frozen)."""
import numpy as np
import pytest

from oracle import estimator, gradient, kernels, precond
from oracle.splitmix import rademacher_block
from paper_2405_03474_gb300 import inputs


@pytest.mark.parametrize("kind", [kernels.RBF, kernels.MATERN52])
def test_exact_gradient_matches_fd(kind):
    X = inputs.points(150, 2, "uniform", seed=2)
    th = np.array([0.3, 1.2, 0.05])

    def f(t):
        return estimator.logdet_exact(kernels.kernel_matrix(X, kind, t[0], t[1], t[2]))

    g = gradient.exact_grad(X, kind, *th)
    for a in range(3):
        h = 1e-5 * th[a]
        e = np.zeros(3)
        e[a] = h
        fd = (f(th + e) - f(th - e)) / (2 * h)
        assert g[a] == pytest.approx(fd, rel=1e-6)


@pytest.mark.parametrize("kind", [kernels.RBF, kernels.MATERN52])
def test_estimator_gradient_matches_fd_with_frozen_P(kind):
    n = 160
    X = inputs.points(n, 2, "uniform", seed=3)
    th = np.array([0.25, 0.9, 0.02])
    M0 = kernels.kernel_matrix(X, kind, *th)
    A, D = precond.build(M0, rademacher_block(2, n, 10), 2, th[2])
    F = precond.factors(A, D)
    Z = rademacher_block(1, n, 5)

    def f(t):
        M = kernels.kernel_matrix(X, kind, *t)
        return estimator.estimate_converged(precond.operator_B(M, F), F["logdet_P"], Z, 3)[0]

    g = gradient.estimator_grad(X, kind, *th, A, D, Z, 3)
    for a in range(3):
        h = 1e-5 * th[a]
        e = np.zeros(3)
        e[a] = h
        fd = (f(th + e) - f(th - e)) / (2 * h)
        assert g[a] == pytest.approx(fd, rel=1e-6)


def test_estimator_gradient_approximates_exact_gradient():
    # With many probes and a good preconditioner the estimator's gradient is close
    # to tr(M^-1 dM) (statistical, loose).
    n = 200
    X = inputs.points(n, 2, "uniform", seed=4)
    th = (0.2, 1.0, 0.05)
    M = kernels.kernel_matrix(X, kernels.RBF, *th)
    A, D = precond.build(M, rademacher_block(2, n, 30), 3, th[2])
    Z = rademacher_block(1, n, 64)
    g = gradient.estimator_grad(X, kernels.RBF, *th, A, D, Z, 5)
    ge = gradient.exact_grad(X, kernels.RBF, *th)
    np.testing.assert_allclose(g, ge, rtol=0.05)
