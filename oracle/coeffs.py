"""Rational approximations to log z (Eq. 1) and their partial fractions (Table 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. 1 gives r_k = N_k(z) / D_k(z) with deg N_k = deg D_k = k.  Section 2 and
Algorithm 1 need r_k in partial-fraction form

    r_k(x) = b + sum_j c_j / (x + sigma_j),     sigma_j > 0,  c_j < 0,

(Table 1 writes every term as ``- |c_j| / (x + sigma_j)``; Algorithm 1 writes
the poles as alpha_j = -sigma_j).  The oracle derives (b, c_j, sigma_j) from the
Eq. 1 polynomials by the textbook route: b is the ratio of leading
coefficients, -sigma_j are the roots of D_k (real and negative, Section 2 citing
Kelisky & Rivlin), and c_j = N_k(-sigma_j) / D_k'(-sigma_j) is the residue at a
simple pole.  Roots come from ``numpy.roots`` and are polished by Newton steps.
"""
from fractions import Fraction

import numpy as np

# Eq. 1, odd orders (the even orders are dropped in Section 1 because they add
# little accuracy).  Coefficients highest power first, as exact rationals.
_EQ1 = {
    1: (Fraction(2), [1, -1], [1, 1]),
    3: (Fraction(2, 3), [7, 27, -27, -7], [1, 15, 15, 1]),
    5: (Fraction(2, 15), [43, 825, 1150, -1150, -825, -43], [1, 45, 210, 210, 45, 1]),
}

ORDERS = (1, 3, 5)


def eq1_polynomials(k):
    """Exact numerator and denominator coefficients of r_k (Eq. 1), highest first."""
    scale, num, den = _EQ1[k]
    return [scale * a for a in num], [Fraction(a) for a in den]


def _horner(coefs, x):
    acc = 0.0
    for a in coefs:
        acc = acc * x + a
    return acc


def _deriv(coefs):
    k = len(coefs) - 1
    return [a * (k - i) for i, a in enumerate(coefs[:-1])]


def rk_coeffs(k):
    """Partial-fraction form of r_k (Table 1): returns (b, c, sigma) as float64.

    ``c`` and ``sigma`` are numpy arrays sorted by increasing sigma, so that
    r_k(x) = b + sum_j c[j] / (x + sigma[j]).
    """
    num, den = eq1_polynomials(k)
    numf = [float(a) for a in num]
    denf = [float(a) for a in den]
    dden = _deriv(denf)
    b = float(num[0] / den[0])
    roots = np.roots(denf)
    if np.max(np.abs(roots.imag)) > 1e-8:
        raise ValueError("denominator of r_%d has complex roots" % k)
    roots = np.sort(roots.real)[::-1]  # -sigma, so increasing sigma
    polished = []
    for x in roots:
        for _ in range(6):
            x = x - _horner(denf, x) / _horner(dden, x)
        polished.append(x)
    sigma = -np.array(polished)
    c = np.array([_horner(numf, -s) / _horner(dden, -s) for s in sigma])
    return b, c, sigma


def rk_eval_pf(k, z):
    """r_k(z) from the partial fractions (the form Algorithm 1 uses)."""
    b, c, sigma = rk_coeffs(k)
    z = np.asarray(z, dtype=np.float64)
    out = np.full_like(z, b)
    for cj, sj in zip(c, sigma):
        out = out + cj / (z + sj)
    return out


def rk_eval_closed(k, z):
    """r_k(z) = N_k(z)/D_k(z) straight from Eq. 1, in float64."""
    num, den = eq1_polynomials(k)
    z = np.asarray(z, dtype=np.float64)
    return _horner([float(a) for a in num], z) / _horner([float(a) for a in den], z)


def rk_exact_rational(k, z):
    """r_k(z) as an exact Fraction for rational z (Eq. 1 evaluated exactly)."""
    num, den = eq1_polynomials(k)
    z = Fraction(z)
    n = Fraction(0)
    for a in num:
        n = n * z + a
    d = Fraction(0)
    for a in den:
        d = d * z + a
    return n / d
