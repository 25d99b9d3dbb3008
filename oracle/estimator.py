"""Algorithm 1 (the r_k log-determinant estimator) and exact log det.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 2 writes log det M = log det P + tr log(M P^-1) and replaces log by the
partial-fraction form of r_k (Table 1), then estimates the trace with
Hutchinson's estimator over s probe vectors (Section 1; the "(1/n) sum over n"
printed there is read as (1/s) sum over the s probes, as in Algorithm 1's
output).  Algorithm 1 obtains each shifted quadratic form from t Lanczos
steps and a tridiagonal (Thomas) solve per shift.

Readings (where the paper is silent or garbled):

* Lanczos runs on the symmetric B = L^-1 M L^-T (``precond.operator_B``),
  which is similar to M P^-1 and so has the same trace of r_k;
* one Krylov space per probe; Algorithm 1's "(T - alpha_i)" and "Q^t w_j" are
  read as (T - alpha_j) with alpha_j = -sigma_j and Q^t w_{i,j};
* ``estimate_lanczos`` is Algorithm 1 taken literally (t steps, full
  reorthogonalisation, Thomas); ``estimate_converged`` is its t -> infinity
  limit, z^T (B + sigma_j I)^-1 z by a Cholesky solve.
"""
import numpy as np

from . import coeffs


def logdet_exact(M):
    """log det M = 2 sum log diag(chol(M)) (Section 3's ground truth)."""
    L = np.linalg.cholesky(np.asarray(M, dtype=np.float64))
    return 2.0 * float(np.sum(np.log(np.diag(L))))


def shifted_quadforms(B, Z, sigma):
    """q[i, j] = z_i^T (B + sigma_j I)^-1 z_i by Cholesky solves (n-by-s Z)."""
    n = B.shape[0]
    q = np.empty((Z.shape[1], len(sigma)))
    for j, sj in enumerate(sigma):
        L = np.linalg.cholesky(B + sj * np.eye(n))
        Y = np.linalg.solve(L, Z)  # L^-1 Z
        q[:, j] = np.einsum("ij,ij->j", Y, Y)
    return q


def combine(logdet_P, Z, q, k):
    """Algorithm 1 output: log det P + (1/s) sum_i [b |z_i|^2 + sum_j c_j q_ij].

    Returns (estimate, per-probe values of the bracket).
    """
    b, c, _ = coeffs.rk_coeffs(k)
    znorm2 = np.einsum("ij,ij->j", Z, Z)
    per_probe = b * znorm2 + q @ c
    return float(logdet_P + np.mean(per_probe)), per_probe


def estimate_converged(B, logdet_P, Z, k):
    """Estimator with exact shifted solves (Algorithm 1 with t -> infinity)."""
    _, _, sigma = coeffs.rk_coeffs(k)
    q = shifted_quadforms(B, np.asarray(Z, dtype=np.float64), sigma)
    est, per_probe = combine(logdet_P, Z, q, k)
    return est, per_probe, q


def lanczos(B, v, t):
    """t steps of Lanczos on symmetric B from v/|v| with full reorthogonalisation.

    Returns the tridiagonal T as (diag, offdiag) and the t-by-n basis Q (rows).
    Stops early on an invariant subspace (beta = 0).
    """
    n = B.shape[0]
    Q = np.zeros((t, n))
    alpha = np.zeros(t)
    beta = np.zeros(t)
    q = v / np.linalg.norm(v)
    m = t
    for k in range(t):
        Q[k] = q
        w = B @ q
        alpha[k] = q @ w
        w = w - Q[:k + 1].T @ (Q[:k + 1] @ w)
        w = w - Q[:k + 1].T @ (Q[:k + 1] @ w)
        beta[k] = np.linalg.norm(w)
        if k + 1 == t:
            break
        if beta[k] <= 1e-14 * max(1.0, abs(alpha[k])):
            m = k + 1
            break
        q = w / beta[k]
    return alpha[:m], beta[:m - 1], Q[:m]


def thomas(lower, diag, upper, rhs):
    """Thomas algorithm for a tridiagonal system (Section 2 cites Thomas 1949)."""
    m = len(diag)
    cp = np.zeros(m)
    dp = np.zeros(m)
    cp[0] = upper[0] / diag[0] if m > 1 else 0.0
    dp[0] = rhs[0] / diag[0]
    for i in range(1, m):
        den = diag[i] - lower[i - 1] * cp[i - 1]
        cp[i] = upper[i] / den if i < m - 1 else 0.0
        dp[i] = (rhs[i] - lower[i - 1] * dp[i - 1]) / den
    x = np.zeros(m)
    x[-1] = dp[-1]
    for i in range(m - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def step3_quadforms(a, bt, vn, sigma):
    """Algorithm 1 step 3 for one probe v with |v| = vn and Lanczos tridiagonal
    T = (diag a, offdiag bt): per shift, (T - alpha_j) w = |v| e_1 by Thomas
    (alpha_j = -sigma_j), and the quadratic form v^T Q^T w = |v| e_1^T w."""
    m = len(a)
    e1 = np.zeros(m)
    e1[0] = vn
    out = np.empty(len(sigma))
    for j, sj in enumerate(sigma):
        w = thomas(bt, a + sj, bt, e1)
        out[j] = vn * w[0]
    return out


def estimate_lanczos(B, logdet_P, Z, k, t):
    """Algorithm 1 taken literally: Lanczos (t steps) then Thomas per shift."""
    _, _, sigma = coeffs.rk_coeffs(k)
    Z = np.asarray(Z, dtype=np.float64)
    s = Z.shape[1]
    q = np.empty((s, len(sigma)))
    for i in range(s):
        v = Z[:, i]
        a, bt, _ = lanczos(B, v, t)
        q[i] = step3_quadforms(a, bt, np.linalg.norm(v), sigma)
    est, per_probe = combine(logdet_P, Z, q, k)
    return est, per_probe, q


def lanczos_block(apply, V, t):
    """``lanczos`` for every column of V at once, for a B given only as a product:
    ``apply(W)`` returns B W for an n-by-s block.  Column c runs its own recurrence
    from V[:, c] / |V[:, c]| with full reorthogonalisation against its own basis, so
    each of the t steps costs one block product instead of s single ones.  Returns
    one (diag, offdiag) pair per column; a column stops early on an invariant
    subspace like ``lanczos`` (its later columns of the block are zero)."""
    V = np.asarray(V, dtype=np.float64)
    n, s = V.shape
    Q = np.zeros((s, t, n))
    alpha = np.zeros((s, t))
    beta = np.zeros((s, t))
    m = np.full(s, t)
    cur = V / np.linalg.norm(V, axis=0)[None, :]
    live = np.ones(s, dtype=bool)
    for k in range(t):
        Q[:, k, :] = cur.T
        W = apply(cur)
        for c in range(s):
            if not live[c]:
                continue
            w = W[:, c]
            alpha[c, k] = cur[:, c] @ w
            Qc = Q[c, :k + 1]
            w = w - Qc.T @ (Qc @ w)
            w = w - Qc.T @ (Qc @ w)
            beta[c, k] = np.linalg.norm(w)
            if k + 1 == t:
                continue
            if beta[c, k] <= 1e-14 * max(1.0, abs(alpha[c, k])):
                m[c] = k + 1
                live[c] = False
                cur[:, c] = 0.0
                continue
            cur[:, c] = w / beta[c, k]
    return [(alpha[c, :m[c]], beta[c, :m[c] - 1]) for c in range(s)]


def estimate_lanczos_block(apply, logdet_P, Z, k, t):
    """Algorithm 1 taken literally for a B given as a block product (``lanczos_block``
    then ``step3_quadforms`` per probe).  Returns (estimate, per-probe brackets, q,
    the per-probe tridiagonals)."""
    _, _, sigma = coeffs.rk_coeffs(k)
    Z = np.asarray(Z, dtype=np.float64)
    tri = lanczos_block(apply, Z, t)
    q = np.empty((Z.shape[1], len(sigma)))
    for i, (a, bt) in enumerate(tri):
        q[i] = step3_quadforms(a, bt, np.linalg.norm(Z[:, i]), sigma)
    est, per_probe = combine(logdet_P, Z, q, k)
    return est, per_probe, q, tri


def estimate_slq(B, logdet_P, Z, t):
    """Stochastic Lanczos quadrature (Ubaru, Chen & Saad 2017), the comparison
    method of Section 3: t Lanczos steps per probe, T = V diag(theta) V^T,
    z^T log(B) z ~ |z|^2 sum_k (e_1^T v_k)^2 log(theta_k).  Returns the estimate
    log det P + (1/s) sum_i of those forms, and the per-probe forms."""
    Z = np.asarray(Z, dtype=np.float64)
    per = np.empty(Z.shape[1])
    for i in range(Z.shape[1]):
        v = Z[:, i]
        a, bt, _ = lanczos(B, v, t)
        per[i] = slq_form(a, bt, float(v @ v))
    return float(logdet_P + np.mean(per)), per


def slq_form(a, bt, vn2):
    """Gauss quadrature of v^T log(B) v from the Lanczos tridiagonal T of (B, v),
    |v|^2 = vn2: T = V diag(theta) V^T, |v|^2 sum_k (e_1^T v_k)^2 log(theta_k)."""
    T = np.diag(a) + np.diag(bt, 1) + np.diag(bt, -1)
    theta, V = np.linalg.eigh(T)
    return vn2 * float(np.sum(V[0] ** 2 * np.log(theta)))


def cg_tridiagonal(B, z, t):
    """The Lanczos tridiagonal of (B, z) rebuilt from t steps of plain CG on B x = z
    (the equivalence behind Section 2's multi-shift reading of Algorithm 1): with the CG
    step sizes a_k and ratios b_k = rho_{k+1} / rho_k,

        T_kk = 1 / a_k + b_{k-1} / a_{k-1}   (no second term for k = 0),
        T_k,k+1 = sqrt(b_k) / a_k.

    Returns (diag, offdiag) like ``lanczos``."""
    B = np.asarray(B, dtype=np.float64)
    r = np.asarray(z, dtype=np.float64).copy()
    p = r.copy()
    rho = float(r @ r)
    a = np.zeros(t)
    b = np.zeros(t)
    for k in range(t):
        Bp = B @ p
        a[k] = rho / float(p @ Bp)
        r = r - a[k] * Bp
        rho_next = float(r @ r)
        b[k] = rho_next / rho
        p = r + b[k] * p
        rho = rho_next
    diag = 1.0 / a
    diag[1:] += b[:-1] / a[:-1]
    return diag, np.sqrt(b[:-1]) / a[:-1]


def multishift_cg(B, z, deltas, iters):
    """Shifted solves x_j ~ (B + delta_j I)^-1 z from one CG run on the seed system B x = z
    (Section 2's multi-shift paragraph, after Jegerlehner): the shifted residuals stay
    collinear with the seed residual, r^j_k = zeta^j_k r_k, and

        zeta^j_{k+1} = zeta^j_k zeta^j_{k-1} a_{k-1}
                       / (a_k b_{k-1} (zeta^j_{k-1} - zeta^j_k) + zeta^j_{k-1} a_{k-1} (1 + delta_j a_k)),
        a^j_k = a_k zeta^j_{k+1} / zeta^j_k,   b^j_k = b_k (zeta^j_{k+1} / zeta^j_k)^2,
        x^j += a^j_k p^j_k,   p^j_{k+1} = zeta^j_{k+1} r_{k+1} + b^j_k p^j_k,

    with a_k, b_k the seed system's CG coefficients, zeta^j_{-1} = zeta^j_0 = 1, a_{-1} = 1,
    b_{-1} = 0.  Returns the len(deltas)-by-n shifted iterates after `iters` steps, or fewer
    once the seed residual is below 1e-16 |z| (the iterates are converged there, and further
    steps would drive the zeta to underflow)."""
    B = np.asarray(B, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    deltas = np.asarray(deltas, dtype=np.float64)
    m = len(deltas)
    r = z.copy()
    p = z.copy()
    rho = float(r @ r)
    xs = np.zeros((m, len(z)))
    ps = np.tile(z, (m, 1))
    zeta, zeta_prev = np.ones(m), np.ones(m)
    a_prev, b_prev = 1.0, 0.0
    rho0 = rho
    for _ in range(iters):
        if rho <= 1e-32 * rho0:
            break
        Bp = B @ p
        a = rho / float(p @ Bp)
        zeta_next = zeta * zeta_prev * a_prev / (a * b_prev * (zeta_prev - zeta)
                                                 + zeta_prev * a_prev * (1.0 + deltas * a))
        xs += (a * zeta_next / zeta)[:, None] * ps
        r = r - a * Bp
        rho_next = float(r @ r)
        b = rho_next / rho
        ps = zeta_next[:, None] * r[None, :] + (b * (zeta_next / zeta) ** 2)[:, None] * ps
        p = r + b * p
        zeta_prev, zeta = zeta, zeta_next
        a_prev, b_prev, rho = a, b, rho_next
    return xs


def rk_bias(B, k):
    """Exact r_k bias of the trace term: sum_i [log lam_i(B) - r_k(lam_i(B))]."""
    lam = np.linalg.eigvalsh(B)
    return float(np.sum(np.log(lam) - coeffs.rk_eval_pf(k, lam)))


def trace_rk(B, k):
    """tr r_k(B) = sum_i r_k(lam_i(B)) from the eigenvalues."""
    return float(np.sum(coeffs.rk_eval_pf(k, np.linalg.eigvalsh(B))))
