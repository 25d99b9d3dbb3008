"""Gradients of log det M with respect to (lengthscale, variance, noise).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 3 mentions a conjugate-gradient based gradient of log det (Wang et al.
2019).  Two oracles:

* ``exact_grad``: d log det M / d theta = tr(M^-1 dM/dtheta), via Cholesky.
* ``estimator_grad``: the derivative of the converged estimator with the
  preconditioner P and the probes held fixed (P "frozen", the stop-gradient
  reading).  With B = L^-1 M L^-T and x_ij = (B + sigma_j I)^-1 z_i, the
  identity d(A^-1) = -A^-1 dA A^-1 gives

      d/dtheta [z^T (B + sigma I)^-1 z] = -y^T (dM/dtheta) y,   y = L^-T x,

  so d est / d theta = (1/s) sum_i sum_j (-c_j) y_ij^T (dM/dtheta) y_ij.
  Freezing P is exact for log det M itself because log det M =
  log det P + log det(M P^-1) holds for every fixed P.
"""
import numpy as np

from . import coeffs, kernels, precond


def dM_matrices(X, kind, lengthscale, variance):
    """(dM/dl, dM/dv, dM/dnu) as dense matrices."""
    n = X.shape[0]
    K = kernels.kernel_matrix(X, kind, lengthscale, variance, 0.0)
    dl = kernels.dkernel_dl_matrix(X, kind, lengthscale, variance)
    return dl, K / variance, np.eye(n)


def exact_grad(X, kind, lengthscale, variance, noise):
    """tr(M^-1 dM/dtheta) for theta = (lengthscale, variance, noise)."""
    M = kernels.kernel_matrix(X, kind, lengthscale, variance, noise)
    L = np.linalg.cholesky(M)
    out = []
    for dM in dM_matrices(X, kind, lengthscale, variance):
        Y = np.linalg.solve(L, dM)
        Minv_dM = np.linalg.solve(L.T, Y)
        out.append(float(np.trace(Minv_dM)))
    return np.array(out)


def estimator_grad(X, kind, lengthscale, variance, noise, A, D, Z, k):
    """Gradient of the converged estimator with P = D + A A^T frozen."""
    _, c, sigma = coeffs.rk_coeffs(k)
    M = kernels.kernel_matrix(X, kind, lengthscale, variance, noise)
    F = precond.factors(A, D)
    B = precond.operator_B(M, F)
    Z = np.asarray(Z, dtype=np.float64)
    s = Z.shape[1]
    n = B.shape[0]
    dMs = dM_matrices(X, kind, lengthscale, variance)
    g = np.zeros(3)
    for j, sj in enumerate(sigma):
        Xs = np.linalg.solve(B + sj * np.eye(n), Z)
        Y = precond.apply_LinvT(F, Xs)
        for a, dM in enumerate(dMs):
            g[a] += -c[j] * np.sum(Y * (dM @ Y)) / s
    return g
