"""Pins for oracle/estimator.py: Hutchinson exactness, M = P, exhaustive probes,
Lanczos = direct solves, Cholesky log det, bias formula."""
import itertools

import numpy as np
import pytest

from oracle import coeffs, estimator, kernels, precond
from oracle.splitmix import rademacher_block
from paper_2405_03474_gb300 import inputs


def test_logdet_exact_against_lu_and_diagonal():
    X = inputs.points(250, 3, "normal", seed=1)
    M = kernels.kernel_matrix(X, kernels.RBF, 0.7, 1.0, 1e-2)
    sign, ref = np.linalg.slogdet(M)  # LU, an independent factorisation
    assert sign > 0
    assert estimator.logdet_exact(M) == pytest.approx(ref, rel=1e-12)
    d = np.array([0.5, 2.0, 3.0, 7.0])
    assert estimator.logdet_exact(np.diag(d)) == pytest.approx(np.sum(np.log(d)), rel=1e-15)
    # 2x2 closed form
    M2 = np.array([[2.0, 0.5], [0.5, 1.0]])
    assert estimator.logdet_exact(M2) == pytest.approx(np.log(2.0 - 0.25), rel=1e-15)


@pytest.mark.parametrize("k", coeffs.ORDERS)
def test_hutchinson_exact_on_diagonal(k):
    # M diagonal, P = I: z^T r(M) z = sum_i z_i^2 r(m_ii) = sum_i r(m_ii) for every sign z.
    d = np.random.default_rng(3).uniform(0.1, 5.0, 64)
    M = np.diag(d)
    Z = rademacher_block(5, 64, 6)
    est, per_probe, _ = estimator.estimate_converged(M, 0.0, Z, k)
    ref = float(np.sum(coeffs.rk_eval_pf(k, d)))
    np.testing.assert_allclose(per_probe, ref, rtol=1e-13)
    assert est == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("k", coeffs.ORDERS)
def test_M_equal_P_gives_logdet_P(k):
    # B = I, r(1) = 0: the estimate is log det P for every probe.
    rng = np.random.default_rng(4)
    n, r = 90, 5
    A = rng.standard_normal((n, r))
    D = rng.uniform(0.5, 2.0, n)
    M = np.diag(D) + A @ A.T
    F = precond.factors(A, D)
    B = precond.operator_B(M, F)
    np.testing.assert_allclose(B, np.eye(n), atol=1e-12)
    est, per_probe, _ = estimator.estimate_converged(B, F["logdet_P"], rademacher_block(1, n, 4), k)
    np.testing.assert_allclose(per_probe, 0.0, atol=1e-10)
    assert est == pytest.approx(np.linalg.slogdet(M)[1], rel=1e-12)


@pytest.mark.parametrize("k", coeffs.ORDERS)
def test_exhaustive_probes_give_trace_of_rk(k):
    # Averaging z^T r(B) z over all 2^n sign vectors gives tr r(B) = sum r(lam_i(B)).
    n = 8
    X = inputs.points(n, 2, "uniform", seed=7)
    M = kernels.kernel_matrix(X, kernels.MATERN52, 0.4, 1.0, 0.05)
    A, D = precond.build(M, rademacher_block(2, n, 2), 1, 0.05)
    F = precond.factors(A, D)
    B = precond.operator_B(M, F)
    Z = np.array(list(itertools.product([-1.0, 1.0], repeat=n))).T
    est, _, _ = estimator.estimate_converged(B, F["logdet_P"], Z, k)
    assert est == pytest.approx(F["logdet_P"] + estimator.trace_rk(B, k), rel=1e-12)
    # and log det M minus that equals the exact r_k bias
    assert estimator.logdet_exact(M) - est == pytest.approx(estimator.rk_bias(B, k), abs=1e-10)


def test_thomas_matches_dense_solve():
    rng = np.random.default_rng(8)
    m = 12
    diag = rng.uniform(3, 4, m)
    off = rng.uniform(-1, 1, m - 1)
    rhs = rng.standard_normal(m)
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    np.testing.assert_allclose(estimator.thomas(off, diag, off, rhs), np.linalg.solve(T, rhs), rtol=1e-12)


def test_lanczos_reproduces_B_and_full_t_equals_direct():
    n = 60
    X = inputs.points(n, 2, "uniform", seed=9)
    M = kernels.kernel_matrix(X, kernels.RBF, 0.3, 1.0, 1e-1)
    F = precond.factors(*precond.identity(n))
    B = precond.operator_B(M, F)
    v = rademacher_block(3, n, 1)[:, 0]
    a, bt, Q = estimator.lanczos(B, v, 10)
    T = np.diag(a) + np.diag(bt, 1) + np.diag(bt, -1)
    np.testing.assert_allclose(Q @ Q.T, np.eye(len(a)), atol=1e-12)
    np.testing.assert_allclose(Q @ B @ Q.T, T, atol=1e-10)
    Z = rademacher_block(4, n, 3)
    for k in coeffs.ORDERS:
        e1, p1, _ = estimator.estimate_lanczos(B, 0.0, Z, k, n)
        e2, p2, _ = estimator.estimate_converged(B, 0.0, Z, k)
        np.testing.assert_allclose(p1, p2, rtol=1e-9)


def test_lanczos_quadrature_converges_with_t():
    n = 200
    X = inputs.points(n, 2, "uniform", seed=10)
    M = kernels.kernel_matrix(X, kernels.MATERN52, 0.2, 1.0, 1e-2)
    A, D = precond.build(M, rademacher_block(2, n, 16), 3, 1e-2)
    F = precond.factors(A, D)
    B = precond.operator_B(M, F)
    Z = rademacher_block(1, n, 4)
    ref, _, _ = estimator.estimate_converged(B, F["logdet_P"], Z, 3)
    errs = [abs(estimator.estimate_lanczos(B, F["logdet_P"], Z, 3, t)[0] - ref) for t in (2, 5, 10, 40)]
    assert errs[-1] < 1e-8 * abs(ref)
    assert errs[0] > errs[2]


def test_r3_more_accurate_than_r1_on_kernel_matrices():
    # Section 3: r_3 has lower error than r_1 (here: the exact r_k bias, no probe noise).
    for kind in (kernels.RBF, kernels.MATERN52):
        X = inputs.points(300, 5, "normal", seed=11)
        M = kernels.kernel_matrix(X, kind, 1.0, 1.0, 1e-2)
        A, D = precond.build(M, rademacher_block(2, 300, 25), 5, 1e-2)
        B = precond.operator_B(M, precond.factors(A, D))
        b1, b3, b5 = (abs(estimator.rk_bias(B, k)) for k in (1, 3, 5))
        assert b3 < b1 and b5 < b1


def test_slq_with_full_lanczos_is_exact_quadratic_form():
    # With t = n the Gauss quadrature of z^T log(B) z is exact: compare with eigh(B).
    n = 40
    X = inputs.points(n, 2, "uniform", seed=12)
    M = kernels.kernel_matrix(X, kernels.MATERN52, 0.3, 1.0, 5e-2)
    F = precond.factors(*precond.build(M, rademacher_block(2, n, 8), 2, 5e-2))
    B = precond.operator_B(M, F)
    lam, U = np.linalg.eigh(B)
    Z = rademacher_block(3, n, 5)
    _, per = estimator.estimate_slq(B, F["logdet_P"], Z, n)
    ref = np.einsum("ij,i,ij->j", U.T @ Z, np.log(lam), U.T @ Z)
    np.testing.assert_allclose(per, ref, rtol=1e-9)
    # and with all 2^n sign vectors (n small) it gives log det M exactly
    n2 = 8
    X2 = inputs.points(n2, 2, "uniform", seed=13)
    M2 = kernels.kernel_matrix(X2, kernels.RBF, 0.5, 1.0, 0.1)
    F2 = precond.factors(*precond.identity(n2))
    Zall = np.array(list(itertools.product([-1.0, 1.0], repeat=n2))).T
    est, _ = estimator.estimate_slq(precond.operator_B(M2, F2), 0.0, Zall, n2)
    assert est == pytest.approx(estimator.logdet_exact(M2), rel=1e-10)


def test_multishift_cg_equals_direct_shifted_solves():
    # One CG run on the seed system gives every shifted solution (Section 2, after
    # Jegerlehner); at the r_3 / r_5 pole spacings and after enough steps the iterates
    # equal (B + delta I)^-1 z from a dense solve.
    n = 80
    X = inputs.points(n, 2, "uniform", seed=14)
    M = kernels.kernel_matrix(X, kernels.MATERN52, 0.3, 1.0, 5e-2)
    F = precond.factors(*precond.build(M, rademacher_block(2, n, 12), 2, 5e-2))
    B = precond.operator_B(M, F)
    z = rademacher_block(6, n, 1)[:, 0]
    for k in (3, 5):
        _, _, sigma = coeffs.rk_coeffs(k)
        seed = B + sigma[0] * np.eye(n)
        deltas = sigma - sigma[0]
        xs = estimator.multishift_cg(seed, z, deltas, 3 * n)
        for j, dj in enumerate(deltas):
            ref = np.linalg.solve(seed + dj * np.eye(n), z)
            np.testing.assert_allclose(xs[j], ref, rtol=1e-9, atol=1e-11 * np.abs(ref).max())
        # and the quadratic forms are those of the converged estimator
        q = z @ xs.T
        np.testing.assert_allclose(q, estimator.shifted_quadforms(B, z[:, None], sigma)[0], rtol=1e-9)


def test_tridiagonal_from_cg_coefficients_equals_lanczos():
    # CG and Lanczos build the same Krylov space: T from the CG scalars equals the
    # Lanczos T of the same start vector (before the basis loses orthogonality).
    n, t = 120, 15
    X = inputs.points(n, 3, "uniform", seed=15)
    M = kernels.kernel_matrix(X, kernels.RBF, 0.35, 1.0, 2e-2)
    F = precond.factors(*precond.build(M, rademacher_block(2, n, 10), 2, 2e-2))
    B = precond.operator_B(M, F) + 0.5 * np.eye(n)
    z = rademacher_block(8, n, 1)[:, 0]
    a, bt, _ = estimator.lanczos(B, z, t)
    d, off = estimator.cg_tridiagonal(B, z, t)
    np.testing.assert_allclose(d, a, rtol=1e-10)
    np.testing.assert_allclose(off, bt, rtol=1e-9)


@pytest.mark.parametrize("k", coeffs.ORDERS)
def test_lanczos_exact_once_krylov_space_is_exhausted(k):
    # B with m distinct eigenvalues: the Krylov space of any z has dimension <= m, so
    # Algorithm 1 with t = m is Gauss quadrature with m nodes on an m-point measure,
    # exact for the rational r_k: the literal estimate equals the converged one.
    rng = np.random.default_rng(16)
    n, lam = 60, np.array([0.3, 0.9, 1.7, 4.0, 11.0])
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    B = (U * np.repeat(lam, n // len(lam))) @ U.T
    B = 0.5 * (B + B.T)
    Z = rademacher_block(9, n, 4)
    e_lit, p_lit, _ = estimator.estimate_lanczos(B, 0.0, Z, k, len(lam))
    e_con, p_con, _ = estimator.estimate_converged(B, 0.0, Z, k)
    np.testing.assert_allclose(p_lit, p_con, rtol=1e-10)
    # with one step fewer the quadrature is not exact
    _, p_short, _ = estimator.estimate_lanczos(B, 0.0, Z, k, len(lam) - 1)
    assert np.max(np.abs(p_short - p_con)) > 1e-8 * np.max(np.abs(p_con))


def test_block_lanczos_equals_lanczos_per_column():
    # the s recurrences run in lockstep (one block product per step) are each the
    # single-vector Lanczos of their own probe
    n, t = 150, 12
    X = inputs.points(n, 3, "uniform", seed=17)
    M = kernels.kernel_matrix(X, kernels.MATERN52, 0.3, 1.0, 1e-2)
    F = precond.factors(*precond.build(M, rademacher_block(2, n, 10), 2, 1e-2))
    B = precond.operator_B(M, F)
    Z = rademacher_block(11, n, 5)
    tri = estimator.lanczos_block(lambda W: B @ W, Z, t)
    for c in range(Z.shape[1]):
        a, bt, _ = estimator.lanczos(B, Z[:, c], t)
        np.testing.assert_allclose(tri[c][0], a, rtol=1e-12)
        np.testing.assert_allclose(tri[c][1], bt, rtol=1e-11)


@pytest.mark.parametrize("k", coeffs.ORDERS)
def test_block_lanczos_with_full_t_equals_direct_solves(k):
    # t = n: the Krylov space is the whole space, so Algorithm 1 equals the converged
    # estimator (dense shifted solves), here with B given only as a product
    n = 48
    X = inputs.points(n, 2, "uniform", seed=18)
    M = kernels.kernel_matrix(X, kernels.RBF, 0.3, 1.0, 1e-1)
    F = precond.factors(*precond.build(M, rademacher_block(2, n, 6), 1, 1e-1))
    B = precond.operator_B(M, F)
    Z = rademacher_block(12, n, 4)
    e1, p1, _, _ = estimator.estimate_lanczos_block(lambda W: B @ W, F["logdet_P"], Z, k, n)
    e2, p2, _ = estimator.estimate_converged(B, F["logdet_P"], Z, k)
    np.testing.assert_allclose(p1, p2, rtol=1e-9)
    assert e1 == pytest.approx(e2, rel=1e-11)


def test_matrix_free_algorithm1_equals_dense_algorithm1():
    # the same literal Algorithm 1 on B = L^-1 M L^-T applied matrix-free (kz_matfree)
    # and on the dense B, with the SLQ forms of the same tridiagonals
    n, t, ell, nu = 400, 10, 0.2, 1e-2
    X = inputs.points(n, 4, "uniform", seed=19)
    M = kernels.kernel_matrix(X, kernels.MATERN52, ell, 1.0, nu)
    F = precond.factors(*precond.build(M, rademacher_block(2, n, 16), 1, nu))
    B = precond.operator_B(M, F)
    Z = rademacher_block(13, n, 6)
    apply = precond.operator_B_apply(lambda V: kernels.kz_matfree(X, V, kernels.MATERN52, ell, 1.0, nu), F)
    e_mf, p_mf, _, tri = estimator.estimate_lanczos_block(apply, F["logdet_P"], Z, 3, t)
    e_d, p_d, _ = estimator.estimate_lanczos(B, F["logdet_P"], Z, 3, t)
    np.testing.assert_allclose(p_mf, p_d, rtol=1e-10)
    slq_mf = [estimator.slq_form(a, bt, float(Z[:, i] @ Z[:, i])) for i, (a, bt) in enumerate(tri)]
    _, slq_d = estimator.estimate_slq(B, F["logdet_P"], Z, t)
    np.testing.assert_allclose(slq_mf, slq_d, rtol=1e-10)


def test_multishift_iterates_at_fixed_t_are_cg_iterates_of_each_shifted_system():
    # After t steps (long before convergence) the multi-shift iterate of shift delta is
    # the t-th plain CG iterate of (seed + delta I) x = z from x_0 = 0 (the Krylov space
    # of z is shift-invariant), here from scipy's CG; its residual is what the residual
    # check reports.
    from scipy.sparse.linalg import cg
    n, t = 200, 5
    X = inputs.points(n, 2, "uniform", seed=20)
    M = kernels.kernel_matrix(X, kernels.MATERN52, 0.2, 1.0, 1e-2)
    F = precond.factors(*precond.build(M, rademacher_block(2, n, 8), 1, 1e-2))
    B = precond.operator_B(M, F)
    z = rademacher_block(14, n, 1)[:, 0]
    _, _, sigma = coeffs.rk_coeffs(3)
    seed = B + sigma[0] * np.eye(n)
    xs = estimator.multishift_cg(seed, z, sigma - sigma[0], t)
    for j, sj in enumerate(sigma):
        ref, _ = cg(B + sj * np.eye(n), z, x0=np.zeros(n), rtol=0.0, atol=0.0, maxiter=t)
        np.testing.assert_allclose(xs[j], ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
        # not yet solved: the residual is far above rounding
        assert np.linalg.norm(z - (B + sj * np.eye(n)) @ xs[j]) > 1e-4 * np.linalg.norm(z)
