"""Randomized truncated-SVD preconditioner P = D + A A^T and its factor L.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 2 asks for a preconditioner P with cheap P v, P^-1 v and det P, and
uses a randomized truncated SVD (Halko, Martinsson & Tropp: range finder
Algorithm 4.1 with subspace iteration Algorithm 4.4, then the direct
eigendecomposition Algorithm 5.3); Section 3 uses 25 eigenvalues and 5
iterations; the Appendix names the form P = D + A A^T ("Truncated Randomized
SVD").  Readings taken where the paper is silent:

* sketch Omega is n-by-r Rademacher (no oversampling); ``q`` subspace
  iterations each apply M once to an orthonormalised block, so the range is
  that of M^(q+1) Omega; orth() is Householder QR with diag(R) > 0;
* C = Q^T M Q (symmetrised), C = V Lambda V^T, Lambda clamped at 0,
  A = Q V Lambda^(1/2);
* D = diag(M) - rowsumsq(A), clamped below at max(nu, 1e-12 * diag(M)).

The split factor used by the estimator (P = L L^T; the paper runs Lanczos on
M P^-1 and leaves the factor open) is built from the thin QR of G = D^-1/2 A:

    G = Q_G R_G   (Householder, diag(R_G) > 0),
    C C^T = I + R_G R_G^T   (Cholesky, C lower triangular),
    R = I + Q_G (C - I) Q_G^T,  so  R R^T = I + G G^T,
    L = D^1/2 R,   L^-1 = (I + Q_G (C^-1 - I) Q_G^T) D^-1/2,

and by the matrix determinant lemma log det P = sum log D + 2 sum log C_kk.
"""
import numpy as np


def orth(Y):
    """Orthonormal basis of range(Y): Householder QR with positive diag(R)."""
    Q, R = np.linalg.qr(Y)
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    return Q * sgn[None, :]


def rsvd(matmul, Omega, q):
    """Randomized truncated eigendecomposition of a symmetric PSD operator.

    ``matmul(V)`` returns M V for an n-by-r block.  Returns A (n-by-r) with
    A A^T = Q C_+ Q^T, the rank-r approximation of M.
    """
    Y = matmul(Omega)
    for _ in range(q):
        Y = matmul(orth(Y))
    Q = orth(Y)
    C = Q.T @ matmul(Q)
    C = 0.5 * (C + C.T)
    lam, V = np.linalg.eigh(C)
    lam = np.maximum(lam, 0.0)
    return Q @ (V * np.sqrt(lam)[None, :])


def diag_residual(diagM, A, noise):
    """D = diag(M) - rowsumsq(A), clamped below at max(noise, 1e-12 diag(M))."""
    diagM = np.asarray(diagM, dtype=np.float64)
    D = diagM - np.einsum("ik,ik->i", A, A)
    floor = np.maximum(noise, 1e-12 * diagM)
    return np.maximum(D, floor)


def build(M, Omega, q, noise):
    """P = D + A A^T from a dense M (rank = Omega.shape[1])."""
    A = rsvd(lambda V: M @ V, Omega, q)
    D = diag_residual(np.diag(M), A, noise)
    return A, D


def build_scaled(M, Omega, q, a):
    """Appendix "Truncated Randomized SVD plus scaling": P = a I + A A^T."""
    A = rsvd(lambda V: M @ V, Omega, q)
    return A, np.full(M.shape[0], float(a))


def factors(A, D):
    """Split factor of P = D + A A^T (see module docstring).

    Returns dict with Q (n-by-r), Cinv (r-by-r lower), dinv_sqrt (n), logdet_P.
    """
    A = np.asarray(A, dtype=np.float64)
    D = np.asarray(D, dtype=np.float64)
    n, r = A.shape
    dinv_sqrt = 1.0 / np.sqrt(D)
    G = A * dinv_sqrt[:, None]
    if r > 0:
        Q, RG = np.linalg.qr(G)
        sgn = np.sign(np.diag(RG))
        sgn[sgn == 0] = 1.0
        Q = Q * sgn[None, :]
        RG = RG * sgn[:, None]
        C = np.linalg.cholesky(np.eye(r) + RG @ RG.T)
        Cinv = np.linalg.inv(C)
        logdet_core = 2.0 * np.sum(np.log(np.diag(C)))
    else:
        Q = np.zeros((n, 0))
        Cinv = np.zeros((0, 0))
        logdet_core = 0.0
    return {
        "Q": Q,
        "Cinv": Cinv,
        "dinv_sqrt": dinv_sqrt,
        "logdet_P": float(np.sum(np.log(D)) + logdet_core),
    }


def apply_Linv(F, V):
    """L^-1 V = (I + Q (C^-1 - I) Q^T) D^-1/2 V."""
    W = F["dinv_sqrt"][:, None] * V
    T = F["Q"].T @ W
    return W + F["Q"] @ (F["Cinv"] @ T - T)


def apply_LinvT(F, V):
    """L^-T V = D^-1/2 (I + Q (C^-T - I) Q^T) V."""
    T = F["Q"].T @ V
    W = V + F["Q"] @ (F["Cinv"].T @ T - T)
    return F["dinv_sqrt"][:, None] * W


def dense_Linv(F):
    n = F["dinv_sqrt"].shape[0]
    return apply_Linv(F, np.eye(n))


def operator_B(M, F):
    """B = L^-1 M L^-T, symmetric and similar to M P^-1 (Section 2)."""
    Li = dense_Linv(F)
    B = Li @ M @ Li.T
    return 0.5 * (B + B.T)


def operator_B_apply(matmul, F):
    """B = L^-1 M L^-T as a block product, for an M given only as ``matmul(V)`` = M V
    (the matrix-free form of ``operator_B``)."""
    return lambda V: apply_Linv(F, matmul(apply_LinvT(F, V)))


def identity(n):
    """P = I (Appendix "Identity"): A is n-by-0 and D = 1."""
    return np.zeros((n, 0)), np.ones(n)


def diagonal(diagM):
    """P = diag(M) (Appendix "Diagonal")."""
    diagM = np.asarray(diagM, dtype=np.float64)
    return np.zeros((diagM.shape[0], 0)), diagM.copy()
