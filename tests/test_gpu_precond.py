"""Parity of the preconditioner (import, factor, apply, build) against the oracle."""
import numpy as np
import pytest

from gpu_util import assert_elementwise, cuda, host, torch
from oracle import kernels, precond
from oracle.splitmix import rademacher_block
from paper_2405_03474_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _apply_scales(F, V):
    """Elementwise magnitude bounds of L^-1 V and L^-T V: the same products as
    precond.apply_Linv / apply_LinvT with every factor replaced by its absolute value."""
    Q, Ci, ds = np.abs(F["Q"]), np.abs(F["Cinv"] - np.eye(F["Cinv"].shape[0])), F["dinv_sqrt"]
    W = ds[:, None] * np.abs(V)
    s_inv = W + Q @ (Ci @ (Q.T @ W))
    s_invT = ds[:, None] * (np.abs(V) + Q @ (Ci.T @ (Q.T @ np.abs(V))))
    return s_inv, s_invT


def _lowrank(n, r, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, r)) * np.linspace(3.0, 0.2, r)[None, :]
    D = rng.uniform(0.3, 1.2, n)
    return A, D


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_import_factor_and_apply(prec, tol):
    n, r, c = 900, 24, 6
    A, D = _lowrank(n, r, 0)
    F = precond.factors(A, D)
    P = api.Precond.import_(A, D, prec)
    # an fp32 handle stores G in fp32: log det(I + G^T G) moves by ~ r * 2^-24 * |log det|
    assert P.logdet_P == pytest.approx(F["logdet_P"], rel=1e-12 if prec == "fp64" else r * 2.0 ** -24)
    V = inputs.gaussian(n, c, seed=1)
    dt = torch.float64 if prec == "fp64" else torch.float32
    Vt = cuda(V, dt)
    s_inv, s_invT = _apply_scales(F, V)
    assert_elementwise(host(P.apply(Vt, transpose=False)), precond.apply_Linv(F, V), s_inv, tol, "L^-1 V")
    assert_elementwise(host(P.apply(Vt, transpose=True)), precond.apply_LinvT(F, V), s_invT, tol, "L^-T V")
    A2, D2, ld2 = P.export()
    np.testing.assert_allclose(D2, D, rtol=1e-15)
    np.testing.assert_allclose(A2 @ A2.T, A @ A.T, rtol=0, atol=(1e-10 if prec == "fp64" else 1e-4) * np.abs(A @ A.T).max())


def test_identity_rank_zero():
    n = 300
    P = api.Precond.import_(np.zeros((n, 0)), np.ones(n), "fp64")
    assert P.logdet_P == 0.0
    V = cuda(inputs.gaussian(n, 3, seed=2))
    np.testing.assert_array_equal(host(P.apply(V)), host(V))


@pytest.mark.parametrize("kind,dist,ell", [(api.MATERN52, "uniform", 0.2), (api.RBF, "normal", 0.7)])
def test_build_fp64_matches_oracle_rsvd(kind, dist, ell):
    # Same Rademacher sketch on both sides (SplitMix64, seed 2): P = D + A A^T agrees.
    n, d, r, q, nu = 1200, 2, 32, 2, 1e-2
    X = inputs.points(n, d, dist, seed=0)
    k = api.Kernel(kind, ell, 1.0, nu)
    P = api.Precond.build(cuda(X), k, r, power_iters=q, seed=2, precision="fp64")
    A, D, ldP = P.export()
    M = kernels.kernel_matrix(X, kind, ell, 1.0, nu)
    Ao, Do = precond.build(M, rademacher_block(2, n, r), q, nu)
    np.testing.assert_allclose(D, Do, rtol=1e-9, atol=1e-12)
    AA, AAo = A @ A.T, Ao @ Ao.T
    assert np.abs(AA - AAo).max() < 1e-9 * np.abs(AAo).max()
    assert ldP == pytest.approx(precond.factors(Ao, Do)["logdet_P"], rel=1e-10)
    # the handle's own factor is consistent with what it exports
    assert ldP == pytest.approx(precond.factors(A, D)["logdet_P"], rel=1e-12)


def test_build_fp32_is_close_to_oracle():
    n, d, r, q, nu = 2000, 3, 48, 2, 1e-2
    X = inputs.points(n, d, "uniform", seed=1)
    k = api.Kernel(api.MATERN52, 0.3, 1.0, nu)
    P = api.Precond.build(cuda(X), k, r, power_iters=q, seed=2, precision="fp32")
    A, D, ldP = P.export()
    M = kernels.kernel_matrix(X, api.MATERN52, 0.3, 1.0, nu)
    Ao, Do = precond.build(M, rademacher_block(2, n, r), q, nu)
    assert ldP == pytest.approx(precond.factors(Ao, Do)["logdet_P"], rel=1e-4)
    assert ldP == pytest.approx(precond.factors(A, D)["logdet_P"], rel=1e-6)


def test_diagonal_and_plus_scaling_variants_match_oracle():
    n, d, r, q, nu = 1000, 2, 24, 2, 2e-2
    X = inputs.points(n, d, "uniform", seed=4)
    k = api.Kernel(api.MATERN52, 0.25, 1.0, nu)
    M = kernels.kernel_matrix(X, api.MATERN52, 0.25, 1.0, nu)
    # rank 0: P = diag(M) (Appendix "Diagonal")
    P0 = api.Precond.build(cuda(X), k, 0, precision="fp64")
    _, D0, ld0 = P0.export()
    np.testing.assert_allclose(D0, np.diag(M), rtol=1e-15)
    assert ld0 == pytest.approx(np.sum(np.log(np.diag(M))), rel=1e-14)
    # plus scaling: P = a I + A A^T with the same sketch
    Ps = api.Precond.build_scaled(cuda(X), k, r, nu, power_iters=q, seed=2, precision="fp64")
    A, D, ldP = Ps.export()
    Ao, Do = precond.build_scaled(M, rademacher_block(2, n, r), q, nu)
    np.testing.assert_array_equal(D, Do)
    assert np.abs(A @ A.T - Ao @ Ao.T).max() < 1e-9 * np.abs(Ao @ Ao.T).max()
    assert ldP == pytest.approx(precond.factors(Ao, Do)["logdet_P"], rel=1e-10)


def test_build_with_fp16_sketch_matches_its_export_and_the_oracle():
    # the bench builds P with the fp16 tensor-core sketch: the handle's log det P is that of
    # the factors it exports (oracle determinant lemma), and close to the oracle's own build
    # from the same Rademacher sketch (the fp16 products move the subspace slightly)
    n, d, r, q, nu = 4000, 4, 64, 2, 1e-2
    X = inputs.points(n, d, "uniform", seed=2)
    k = api.Kernel(api.MATERN52, 0.2, 1.0, nu)
    P = api.Precond.build(cuda(X), k, r, power_iters=q, seed=2, precision="f16_tc")
    A, D, ldP = P.export()
    F = precond.factors(A, D)
    assert ldP == pytest.approx(F["logdet_P"], rel=1e-6)
    M = kernels.kernel_matrix(X, api.MATERN52, 0.2, 1.0, nu)
    Ao, Do = precond.build(M, rademacher_block(2, n, r), q, nu)
    assert ldP == pytest.approx(precond.factors(Ao, Do)["logdet_P"], rel=2e-3)
    # its applies are those of the exported factors
    V = inputs.gaussian(n, 5, seed=3)
    s_inv, s_invT = _apply_scales(F, V)
    assert_elementwise(host(P.apply(cuda(V, torch.float32))), precond.apply_Linv(F, V), s_inv, 2e-5, "L^-1 V")
    assert_elementwise(host(P.apply(cuda(V, torch.float32), transpose=True)), precond.apply_LinvT(F, V), s_invT,
                       2e-5, "L^-T V")
