"""Gaussian-process covariance functions and kernel-matrix products.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 3 measures the method on covariance matrices of the Matern-5/2 and RBF
kernels (forms from Rasmussen & Williams, which the paper cites).  With
r = ||x - y||, lengthscale l, variance (amplitude squared) v and noise
variance nu added to the diagonal:

    RBF:        k(r) = v * exp(-r^2 / (2 l^2))
    Matern-5/2: k(r) = v * (1 + u + u^2/3) * exp(-u),   u = sqrt(5) r / l
    M = K + nu I.

Lengthscale derivatives (differentiating the forms above):

    RBF:        dk/dl = k * r^2 / l^3
    Matern-5/2: dk/dl = v * (u^2 / (3 l)) * (1 + u) * exp(-u)

and dk/dv = k / v, dM/dnu = I.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

RBF = 0
MATERN52 = 1


def kernel_of_r2(r2, kind, lengthscale, variance):
    """k as a function of the squared distance r2 (float64 array)."""
    r2 = np.asarray(r2, dtype=np.float64)
    if kind == RBF:
        return variance * np.exp(-r2 / (2.0 * lengthscale * lengthscale))
    if kind == MATERN52:
        u = np.sqrt(5.0 * r2) / lengthscale
        return variance * (1.0 + u + u * u / 3.0) * np.exp(-u)
    raise ValueError("unknown kernel kind %r" % (kind,))


def dkernel_dl_of_r2(r2, kind, lengthscale, variance):
    """dk/d(lengthscale) as a function of r2."""
    r2 = np.asarray(r2, dtype=np.float64)
    if kind == RBF:
        k = kernel_of_r2(r2, kind, lengthscale, variance)
        return k * r2 / lengthscale ** 3
    if kind == MATERN52:
        u = np.sqrt(5.0 * r2) / lengthscale
        return variance * (u * u / (3.0 * lengthscale)) * (1.0 + u) * np.exp(-u)
    raise ValueError("unknown kernel kind %r" % (kind,))


def sqdist(XA, XB):
    """Squared Euclidean distances by explicit coordinate differences."""
    XA = np.asarray(XA, dtype=np.float64)
    XB = np.asarray(XB, dtype=np.float64)
    diff = XA[:, None, :] - XB[None, :, :]
    return np.einsum("ijk,ijk->ij", diff, diff)


def kernel_matrix(X, kind, lengthscale, variance, noise=0.0):
    """Dense M = K(X, X) + noise * I (n-by-n float64)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    M = np.empty((n, n))
    step = max(1, 2 ** 22 // max(1, n * X.shape[1]))
    for i0 in range(0, n, step):
        M[i0:i0 + step] = kernel_of_r2(sqdist(X[i0:i0 + step], X), kind, lengthscale, variance)
    M[np.diag_indices(n)] += noise
    return M


def dkernel_dl_matrix(X, kind, lengthscale, variance):
    """Dense dK/d(lengthscale) (n-by-n float64)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    out = np.empty((n, n))
    step = max(1, 2 ** 22 // max(1, n * X.shape[1]))
    for i0 in range(0, n, step):
        out[i0:i0 + step] = dkernel_dl_of_r2(sqdist(X[i0:i0 + step], X), kind, lengthscale, variance)
    return out


def kz_rows(X, V, rows, kind, lengthscale, variance, noise=0.0):
    """Rows ``rows`` of (K + noise I) V without forming K (matrix-free).

    X is n-by-d, V is n-by-s; returns len(rows)-by-s.  Each output row is the
    plain sum over all n points j of k(x_row, x_j) V[j, :], plus noise V[row, :].
    """
    X = np.asarray(X, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    rows = np.asarray(rows)
    n = X.shape[0]
    out = np.zeros((len(rows), V.shape[1]))
    chunk = max(1, 2 ** 24 // max(1, len(rows) * X.shape[1]))
    for j0 in range(0, n, chunk):
        Kb = kernel_of_r2(sqdist(X[rows], X[j0:j0 + chunk]), kind, lengthscale, variance)
        out += Kb @ V[j0:j0 + chunk]
    out += noise * V[rows]
    return out


def kz_matfree(X, V, kind, lengthscale, variance, noise=0.0, rows_per_task=128, threads=None):
    """All rows of (K + noise I) V without forming K: ``kz_rows`` over consecutive
    row ranges, the ranges spread over a thread pool (numpy releases the GIL in
    its elementwise loops and BLAS calls, so the host cores share the work).
    Each output row is computed exactly as ``kz_rows`` computes it."""
    X = np.asarray(X, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    n = X.shape[0]
    out = np.empty((n, V.shape[1]))
    starts = list(range(0, n, rows_per_task))

    def task(i0):
        rows = np.arange(i0, min(n, i0 + rows_per_task))
        out[rows] = kz_rows(X, V, rows, kind, lengthscale, variance, noise)

    with ThreadPoolExecutor(threads or os.cpu_count() or 1) as ex:
        list(ex.map(task, starts))
    return out
