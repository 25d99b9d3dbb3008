"""Pins for oracle/kernels.py: textbook forms, special values, the general Matern."""
import math

import numpy as np
import pytest
from scipy.special import gamma, kv

from oracle import kernels
from paper_2405_03474_gb300 import inputs


def test_special_values():
    v, l = 1.7, 0.3
    assert kernels.kernel_of_r2(0.0, kernels.RBF, l, v) == pytest.approx(v)
    assert kernels.kernel_of_r2(0.0, kernels.MATERN52, l, v) == pytest.approx(v)
    # RBF at r = l: v e^{-1/2};  Matern at u = sqrt(5) r / l = 1: v (7/3) e^{-1}
    assert kernels.kernel_of_r2(l * l, kernels.RBF, l, v) == pytest.approx(v * math.exp(-0.5), rel=1e-15)
    r = l / math.sqrt(5.0)
    assert kernels.kernel_of_r2(r * r, kernels.MATERN52, l, v) == pytest.approx(v * 7 / 3 / math.e, rel=1e-14)


def test_matern52_equals_general_matern_bessel_form():
    # General Matern: v 2^(1-p)/Gamma(p) (sqrt(2p) r/l)^p K_p(sqrt(2p) r/l), p = 5/2.
    l, v, p = 0.4, 1.3, 2.5
    r = np.linspace(0.01, 3.0, 200)
    a = math.sqrt(2 * p) * r / l
    ref = v * 2 ** (1 - p) / gamma(p) * a ** p * kv(p, a)
    got = kernels.kernel_of_r2(r * r, kernels.MATERN52, l, v)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_rbf_is_gaussian_density_ratio():
    # exp(-r^2/(2 l^2)) is the N(0, l^2) density at r divided by its value at 0.
    from scipy.stats import norm
    l = 0.7
    r = np.linspace(0, 4, 50)
    ref = norm.pdf(r, scale=l) / norm.pdf(0, scale=l)
    np.testing.assert_allclose(kernels.kernel_of_r2(r * r, kernels.RBF, l, 1.0), ref, rtol=1e-13)


@pytest.mark.parametrize("kind", [kernels.RBF, kernels.MATERN52])
def test_lengthscale_derivative_matches_central_difference(kind):
    r2 = np.linspace(0.0, 2.0, 101)
    l, v, h = 0.37, 1.2, 1e-6
    fd = (kernels.kernel_of_r2(r2, kind, l + h, v) - kernels.kernel_of_r2(r2, kind, l - h, v)) / (2 * h)
    np.testing.assert_allclose(kernels.dkernel_dl_of_r2(r2, kind, l, v), fd, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("kind", [kernels.RBF, kernels.MATERN52])
def test_kernel_matrix_is_spd_and_rows_match(kind):
    X = inputs.points(300, 3, "uniform", seed=5)
    M = kernels.kernel_matrix(X, kind, 0.2, 1.0, 1e-3)
    np.testing.assert_allclose(M, M.T, atol=0)
    np.linalg.cholesky(M)
    # brute force over pairs for a few entries
    for i, j in [(0, 0), (3, 17), (299, 5)]:
        r2 = sum((X[i, t] - X[j, t]) ** 2 for t in range(3))
        ref = float(kernels.kernel_of_r2(r2, kind, 0.2, 1.0)) + (1e-3 if i == j else 0.0)
        assert M[i, j] == pytest.approx(ref, rel=1e-14)
    V = inputs.gaussian(300, 5, seed=9)
    rows = np.array([0, 7, 128, 299])
    np.testing.assert_allclose(kernels.kz_rows(X, V, rows, kind, 0.2, 1.0, 1e-3), (M @ V)[rows],
                               rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kind", [kernels.RBF, kernels.MATERN52])
def test_matrix_free_product_equals_dense_product(kind):
    # every row of (K + noise I) V without forming K, over ragged row ranges on 3 threads
    X = inputs.points(250, 4, "uniform", seed=6)
    V = inputs.gaussian(250, 7, seed=10)
    M = kernels.kernel_matrix(X, kind, 0.15, 1.3, 2e-2)
    got = kernels.kz_matfree(X, V, kind, 0.15, 1.3, 2e-2, rows_per_task=7, threads=3)
    np.testing.assert_allclose(got, M @ V, rtol=1e-12, atol=1e-12)
