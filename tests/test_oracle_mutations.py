"""The oracle's pins have teeth: each plausible mistake planted in the oracle
(a dropped term, a wrong sign, index or constant, a transposed operand) makes
one of its pin tests fail.

The mistake is planted in memory only: the oracle module's source is read,
one exact passage is replaced, the result is executed as a fresh module and its
functions are patched over the real module's for the duration of one test.
Every case first runs the pin on the oracle as it is (it must pass), then on
the mutant (it must fail with an assertion or a linear-algebra error).
"""
import importlib
import inspect
import types

import numpy as np
import pytest


def _plant(monkeypatch, modname, old, new):
    mod = importlib.import_module(modname)
    src = inspect.getsource(mod)
    assert src.count(old) == 1, "the passage to replace must occur exactly once"
    mutant = types.ModuleType(modname)
    mutant.__file__ = mod.__file__
    mutant.__package__ = mod.__package__
    exec(compile(src.replace(old, new), mod.__file__, "exec"), mutant.__dict__)
    for name, obj in vars(mutant).items():
        if isinstance(obj, types.FunctionType) and obj.__module__ == modname:
            monkeypatch.setattr(mod, name, obj)


def P(modname, old, new, pin, *args, id):
    tmod, tname = pin.split("::")
    return pytest.param(modname, old, new, tmod, tname, args, id=id)


MUTANTS = [
    # coefficients of r_k (Eq. 1, Table 1)
    P("oracle.coeffs", "[7, 27, -27, -7]", "[7, 26, -27, -7]",
      "test_oracle_coeffs::test_partial_fractions_match_table1", 3, id="eq1-numerator-coefficient"),
    P("oracle.coeffs", "_horner(numf, -s) / _horner(dden, -s)", "_horner(numf, s) / _horner(dden, -s)",
      "test_oracle_coeffs::test_partial_fractions_match_table1", 5, id="residue-at-wrong-pole"),
    P("oracle.coeffs", "out = out + cj / (z + sj)", "out = out + cj / (z - sj)",
      "test_oracle_coeffs::test_partial_fractions_equal_closed_form", 3, id="partial-fraction-sign"),
    # the estimator (Algorithm 1, Hutchinson)
    P("oracle.estimator", "per_probe = b * znorm2 + q @ c", "per_probe = q @ c",
      "test_oracle_estimator::test_hutchinson_exact_on_diagonal", 3, id="dropped-b-term"),
    P("oracle.estimator", "logdet_P + np.mean(per_probe)", "logdet_P + np.sum(per_probe)",
      "test_oracle_estimator::test_hutchinson_exact_on_diagonal", 1, id="hutchinson-normalisation"),
    P("oracle.estimator", "L = np.linalg.cholesky(B + sj * np.eye(n))", "L = np.linalg.cholesky(B - sj * np.eye(n))",
      "test_oracle_estimator::test_hutchinson_exact_on_diagonal", 3, id="shift-sign"),
    P("oracle.estimator", "den = diag[i] - lower[i - 1] * cp[i - 1]", "den = diag[i] - lower[i - 1] * cp[i]",
      "test_oracle_estimator::test_thomas_matches_dense_solve", id="thomas-index"),
    P("oracle.estimator", "out[j] = vn * w[0]", "out[j] = w[0]",
      "test_oracle_estimator::test_lanczos_reproduces_B_and_full_t_equals_direct", id="lanczos-dropped-norm"),
    P("oracle.estimator", "alpha[k] = q @ w", "alpha[k] = w @ w",
      "test_oracle_estimator::test_lanczos_reproduces_B_and_full_t_equals_direct", id="lanczos-diagonal"),
    P("oracle.estimator", "np.sum(V[0] ** 2 * np.log(theta))", "np.sum(V[:, 0] ** 2 * np.log(theta))",
      "test_oracle_estimator::test_slq_with_full_lanczos_is_exact_quadratic_form", id="slq-transposed-eigvec"),
    P("oracle.estimator", "return 2.0 * float(np.sum(np.log(np.diag(L))))", "return float(np.sum(np.log(np.diag(L))))",
      "test_oracle_estimator::test_logdet_exact_against_lu_and_diagonal", id="cholesky-logdet-factor"),
    P("oracle.estimator", "diag[1:] += b[:-1] / a[:-1]", "diag[1:] += b[1:] / a[1:]",
      "test_oracle_estimator::test_tridiagonal_from_cg_coefficients_equals_lanczos", id="cg-tridiagonal-index"),
    P("oracle.estimator", "np.sqrt(b[:-1]) / a[:-1]", "b[:-1] / a[:-1]",
      "test_oracle_estimator::test_tridiagonal_from_cg_coefficients_equals_lanczos", id="cg-offdiagonal-sqrt"),
    P("oracle.estimator", "zeta_prev * a_prev * (1.0 + deltas * a))", "zeta_prev * a_prev * (1.0 - deltas * a))",
      "test_oracle_estimator::test_multishift_cg_equals_direct_shifted_solves", id="multishift-zeta-sign"),
    P("oracle.estimator", "(b * (zeta_next / zeta) ** 2)", "(b * (zeta_next / zeta))",
      "test_oracle_estimator::test_multishift_cg_equals_direct_shifted_solves", id="multishift-beta-square"),
    P("oracle.estimator", "alpha[c, k] = cur[:, c] @ w", "alpha[c, k] = w @ w",
      "test_oracle_estimator::test_block_lanczos_equals_lanczos_per_column", id="block-lanczos-diagonal"),
    P("oracle.estimator", "cur[:, c] = w / beta[c, k]", "cur[:, c] = w",
      "test_oracle_estimator::test_block_lanczos_with_full_t_equals_direct_solves", 3, id="block-lanczos-normalisation"),
    # kernels (Section 3, Rasmussen & Williams forms)
    P("oracle.kernels", "(1.0 + u + u * u / 3.0)", "(1.0 + u + u * u / 2.0)",
      "test_oracle_kernels::test_matern52_equals_general_matern_bessel_form", id="matern-polynomial"),
    P("oracle.kernels", "np.exp(-r2 / (2.0 * lengthscale * lengthscale))", "np.exp(-r2 / (lengthscale * lengthscale))",
      "test_oracle_kernels::test_rbf_is_gaussian_density_ratio", id="rbf-half-factor"),
    P("oracle.kernels", "(u * u / (3.0 * lengthscale))", "(u * u / (3.0 * lengthscale ** 2))",
      "test_oracle_kernels::test_lengthscale_derivative_matches_central_difference", 1, id="matern-derivative"),
    P("oracle.kernels", "M[np.diag_indices(n)] += noise", "M[np.diag_indices(n)] += 0.0",
      "test_oracle_kernels::test_kernel_matrix_is_spd_and_rows_match", 0, id="dropped-noise"),
    P("oracle.kernels", "out += noise * V[rows]", "out += 0.0 * V[rows]",
      "test_oracle_kernels::test_kernel_matrix_is_spd_and_rows_match", 1, id="matrix-free-dropped-noise"),
    P("oracle.kernels", "rows = np.arange(i0, min(n, i0 + rows_per_task))", "rows = np.arange(i0, min(n, i0 + rows_per_task - 1))",
      "test_oracle_kernels::test_matrix_free_product_equals_dense_product", 1, id="matrix-free-row-range"),
    # preconditioner (Section 2, Appendix)
    P("oracle.precond", 'W = V + F["Q"] @ (F["Cinv"].T @ T - T)', 'W = V + F["Q"] @ (F["Cinv"] @ T - T)',
      "test_oracle_precond::test_split_factor_inverts_P", id="LinvT-transposed-core"),
    P("oracle.precond", 'W = F["dinv_sqrt"][:, None] * V', "W = V",
      "test_oracle_precond::test_split_factor_inverts_P", id="Linv-dropped-diagonal"),
    P("oracle.precond", "logdet_core = 2.0 * np.sum(np.log(np.diag(C)))", "logdet_core = np.sum(np.log(np.diag(C)))",
      "test_oracle_precond::test_logdet_P_matches_dense_slogdet", id="determinant-lemma-factor"),
    P("oracle.precond", 'D = diagM - np.einsum("ik,ik->i", A, A)', "D = diagM",
      "test_oracle_precond::test_rsvd_top_eigenvalues_on_kernel_matrix", id="residual-diagonal"),
    P("oracle.precond", "C = Q.T @ matmul(Q)", "C = Q.T @ Q",
      "test_oracle_precond::test_rsvd_recovers_exact_low_rank_plus_diagonal", id="rsvd-core"),
    P("oracle.precond", "apply_Linv(F, matmul(apply_LinvT(F, V)))", "apply_LinvT(F, matmul(apply_Linv(F, V)))",
      "test_oracle_precond::test_matrix_free_B_equals_dense_B", id="matrix-free-B-order"),
    # gradients (Section 3)
    P("oracle.gradient", "g[a] += -c[j] * np.sum(Y * (dM @ Y)) / s", "g[a] += c[j] * np.sum(Y * (dM @ Y)) / s",
      "test_oracle_gradient::test_estimator_gradient_matches_fd_with_frozen_P", 0, id="adjoint-sign"),
    P("oracle.gradient", "Y = precond.apply_LinvT(F, Xs)", "Y = Xs",
      "test_oracle_gradient::test_estimator_gradient_matches_fd_with_frozen_P", 1, id="adjoint-dropped-LinvT"),
    P("oracle.gradient", "return dl, K / variance, np.eye(n)", "return dl, K, np.eye(n)",
      "test_oracle_gradient::test_exact_gradient_matches_fd", 0, id="variance-derivative"),
    # surrogate MLP
    P("oracle.mlp", "return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))", "return 0.5 * x * (1.0 + erf(x / 2.0))",
      "test_oracle_mlp::test_param_count_and_gelu", id="gelu-constant"),
    P("oracle.mlp", "dz = (2.0 / N) * (pred - y)[:, None]", "dz = (1.0 / N) * (pred - y)[:, None]",
      "test_oracle_mlp::test_parameter_gradient_matches_fd", id="mse-gradient-factor"),
    P("oracle.mlp", "mhat = m / (1.0 - beta1 ** step)", "mhat = m",
      "test_oracle_mlp::test_first_adam_step_is_lr_times_sign", id="adam-bias-correction"),
    # counter-based generator
    P("oracle.splitmix", "(k + np.uint64(1)) * GAMMA", "k * GAMMA",
      "test_oracle_splitmix::test_published_seed0_sequence", id="splitmix-counter-offset"),
    P("oracle.splitmix", "k = cols[None, :] * np.uint64(n) + rows[:, None]\n    bits",
      "k = rows[:, None] * np.uint64(s) + cols[None, :]\n    bits",
      "test_oracle_splitmix::test_rademacher_block_layout_and_balance", id="rademacher-transposed-counter"),
    P("oracle.splitmix", "np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)",
      "np.sqrt(-2.0 * np.log(u2)) * np.cos(2.0 * np.pi * u1)",
      "test_oracle_splitmix::test_gaussian_block_is_standard_normal", id="box-muller-swapped-uniforms"),
    P("oracle.splitmix", "Q = Q * np.sign(np.diag(R))", "Q = Q",
      "test_oracle_splitmix::test_orthogonal_block_structure", id="orthogonal-sign-fix"),
]


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # some mutants divide by zero
@pytest.mark.parametrize("modname,old,new,tmod,tname,args", MUTANTS)
def test_pin_catches_planted_mistake(monkeypatch, modname, old, new, tmod, tname, args):
    pin = getattr(importlib.import_module(tmod), tname)
    pin(*args)  # passes on the oracle as it is
    _plant(monkeypatch, modname, old, new)
    with pytest.raises((AssertionError, np.linalg.LinAlgError)):
        pin(*args)
