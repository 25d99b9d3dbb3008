"""Pins for oracle/precond.py: determinant lemma, the split factor, rSVD recovery."""
import numpy as np
import pytest

from oracle import kernels, precond
from oracle.splitmix import rademacher_block
from paper_2405_03474_gb300 import inputs


def _random_lowrank(n, r, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, r)) * np.linspace(2.0, 0.1, r)[None, :]
    D = rng.uniform(0.2, 1.5, n)
    return A, D


def test_logdet_P_matches_dense_slogdet():
    A, D = _random_lowrank(200, 12, 0)
    F = precond.factors(A, D)
    sign, ref = np.linalg.slogdet(np.diag(D) + A @ A.T)
    assert sign > 0
    assert F["logdet_P"] == pytest.approx(ref, rel=1e-12)


def test_split_factor_inverts_P():
    # L^-1 P L^-T = I, Q is orthonormal, and R = I + Q (C - I) Q^T has R R^T = I + G G^T.
    A, D = _random_lowrank(150, 9, 1)
    F = precond.factors(A, D)
    P = np.diag(D) + A @ A.T
    Li = precond.dense_Linv(F)
    np.testing.assert_allclose(Li @ P @ Li.T, np.eye(150), atol=1e-11)
    Q = F["Q"]
    np.testing.assert_allclose(Q.T @ Q, np.eye(9), atol=1e-13)
    C = np.linalg.inv(F["Cinv"])
    assert np.allclose(np.triu(C, 1), 0.0)
    R = np.eye(150) + Q @ (C - np.eye(9)) @ Q.T
    G = A / np.sqrt(D)[:, None]
    np.testing.assert_allclose(R @ R.T, np.eye(150) + G @ G.T, atol=1e-11)
    V = np.random.default_rng(2).standard_normal((150, 4))
    np.testing.assert_allclose(precond.apply_LinvT(F, V), Li.T @ V, atol=1e-12)


def test_operator_B_is_similar_to_M_Pinv():
    X = inputs.points(120, 2, "uniform", seed=3)
    M = kernels.kernel_matrix(X, kernels.MATERN52, 0.3, 1.0, 1e-2)
    A, D = _random_lowrank(120, 6, 4)
    F = precond.factors(A, D)
    B = precond.operator_B(M, F)
    P = np.diag(D) + A @ A.T
    ev_B = np.sort(np.linalg.eigvalsh(B))
    ev_MP = np.sort(np.linalg.eigvals(M @ np.linalg.inv(P)).real)
    np.testing.assert_allclose(ev_B, ev_MP, rtol=1e-9)


def test_rsvd_recovers_exact_low_rank_plus_diagonal():
    # M = U diag(lam) U^T with rank r: the rank-r sketch recovers M exactly.
    n, r = 300, 10
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((n, r)))
    lam = np.linspace(50.0, 1.0, r)
    M = (U * lam) @ U.T
    Om = rademacher_block(11, n, r)
    A = precond.rsvd(lambda V: M @ V, Om, 2)
    np.testing.assert_allclose(A @ A.T, M, atol=1e-10)


def test_rsvd_top_eigenvalues_on_kernel_matrix():
    # with a spectral gap and power iterations, A A^T holds the top-r eigenvalues of M
    X = inputs.points(400, 2, "uniform", seed=6)
    M = kernels.kernel_matrix(X, kernels.RBF, 0.5, 1.0, 1e-3)
    r = 8
    A, D = precond.build(M, rademacher_block(2, 400, r), 5, 1e-3)
    got = np.sort(np.linalg.eigvalsh(A.T @ A))[::-1]
    ref = np.sort(np.linalg.eigvalsh(M))[::-1][:r]
    np.testing.assert_allclose(got, ref, rtol=1e-6)
    # D is the diagonal of the residual, clamped at the noise level
    np.testing.assert_allclose(D, np.maximum(np.diag(M) - np.sum(A * A, axis=1), 1e-3), rtol=1e-12, atol=1e-14)
    assert np.all(D >= 1e-3)


def test_identity_and_diagonal_preconditioners():
    A, D = precond.identity(5)
    F = precond.factors(A, D)
    assert F["logdet_P"] == 0.0
    np.testing.assert_allclose(precond.dense_Linv(F), np.eye(5))
    d = np.array([1.0, 2.0, 4.0])
    A, D = precond.diagonal(d)
    assert precond.factors(A, D)["logdet_P"] == pytest.approx(np.log(8.0))


def test_plus_scaling_variant():
    # P = a I + A A^T keeps the rSVD factor and replaces the diagonal by a constant
    n, r, a = 200, 12, 0.05
    X = inputs.points(n, 2, "uniform", seed=8)
    M = kernels.kernel_matrix(X, kernels.RBF, 0.4, 1.0, a)
    Om = rademacher_block(2, n, r)
    A1, _ = precond.build(M, Om, 2, a)
    A2, D2 = precond.build_scaled(M, Om, 2, a)
    np.testing.assert_allclose(A1 @ A1.T, A2 @ A2.T, atol=1e-12)
    np.testing.assert_array_equal(D2, np.full(n, a))
    F = precond.factors(A2, D2)
    assert F["logdet_P"] == pytest.approx(np.linalg.slogdet(a * np.eye(n) + A2 @ A2.T)[1], rel=1e-12)


def test_rank_one_build_is_the_appendix_rank_one_preconditioner():
    # The Appendix's rank-one preconditioner P = D + lambda v v^T with D = diag(M - lambda v v^T)
    # is this build at rank 1: subspace iteration converges to the top eigenpair (lambda, v).
    n = 250
    X = inputs.points(n, 2, "uniform", seed=12)
    M = kernels.kernel_matrix(X, kernels.MATERN52, 0.5, 1.0, 1e-2)
    A, D = precond.build(M, rademacher_block(2, n, 1), 30, 1e-2)
    lam, U = np.linalg.eigh(M)
    v = U[:, -1]
    np.testing.assert_allclose(A[:, 0] @ A[:, 0], lam[-1], rtol=1e-10)
    np.testing.assert_allclose(np.abs(A[:, 0]) / np.sqrt(lam[-1]), np.abs(v), atol=1e-8)
    np.testing.assert_allclose(D, np.maximum(np.diag(M - lam[-1] * np.outer(v, v)), 1e-2), rtol=1e-8)


def test_matrix_free_B_equals_dense_B():
    n = 120
    X = inputs.points(n, 3, "uniform", seed=21)
    M = kernels.kernel_matrix(X, kernels.RBF, 0.25, 1.0, 1e-2)
    F = precond.factors(*precond.build(M, rademacher_block(2, n, 9), 1, 1e-2))
    V = inputs.gaussian(n, 4, seed=22)
    got = precond.operator_B_apply(lambda W: M @ W, F)(V)
    np.testing.assert_allclose(got, precond.operator_B(M, F) @ V, rtol=1e-11, atol=1e-11)
