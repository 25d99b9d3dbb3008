"""Pins for oracle/coeffs.py: Eq. 1, Table 1 and the properties stated in Section 1."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import coeffs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def _table1():
    """Parse tests/golden/table1.txt (Table 1, Section 2)."""
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            k = int(parts[0])
            val = [float(Fraction(p)) for p in parts[2:]]
            entry = out.setdefault(k, {"b": None, "terms": []})
            if parts[1] == "b":
                entry["b"] = val[0]
            else:
                entry["terms"].append((val[0], val[1]))
    return out


@pytest.mark.parametrize("k", coeffs.ORDERS)
def test_partial_fractions_match_table1(k):
    tab = _table1()[k]
    b, c, sigma = coeffs.rk_coeffs(k)
    assert b == pytest.approx(tab["b"], rel=1e-15)
    terms = sorted(tab["terms"], key=lambda t: t[1])
    assert len(terms) == len(c) == k
    for (abs_c, sig), cj, sj in zip(terms, c, sigma):
        assert cj < 0 and sj > 0
        assert sj == pytest.approx(sig, rel=1e-13)
        assert -cj == pytest.approx(abs_c, rel=1e-13)


def test_r3_closed_form_roots_and_residues():
    # r_3's denominator is (z + 1)(z^2 + 14 z + 1): roots -1 and -7 +- 4 sqrt(3);
    # residues from N(-s)/D'(-s) worked by hand: -224/9 -+ 128 sqrt(3)/9 and -20/9.
    _, c, sigma = coeffs.rk_coeffs(3)
    r3 = math.sqrt(3.0)
    np.testing.assert_allclose(sigma, [7 - 4 * r3, 1.0, 7 + 4 * r3], rtol=1e-14)
    np.testing.assert_allclose(c, [-224 / 9 + 128 * r3 / 9, -20 / 9, -224 / 9 - 128 * r3 / 9],
                               rtol=1e-12)


def test_r5_roots_from_palindromic_quartic():
    # z^5+45z^4+210z^3+210z^2+45z+1 = (z+1)(z^4+44z^3+166z^2+44z+1); the quartic is
    # palindromic, so w = z + 1/z solves w^2 + 44 w + 164 = 0, w = -22 +- 8 sqrt(5).
    _, _, sigma = coeffs.rk_coeffs(5)
    roots = [1.0]
    for w in (-22 + 8 * math.sqrt(5), -22 - 8 * math.sqrt(5)):
        disc = math.sqrt(w * w - 4)
        roots += [-(w + disc) / 2, -(w - disc) / 2]
    np.testing.assert_allclose(np.sort(sigma), np.sort(roots), rtol=1e-13)


@pytest.mark.parametrize("k", coeffs.ORDERS)
def test_partial_fractions_equal_closed_form(k):
    z = np.logspace(-3, 3, 2001)
    pf = coeffs.rk_eval_pf(k, z)
    cf = coeffs.rk_eval_closed(k, z)
    np.testing.assert_allclose(pf, cf, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("k,z", [(1, 2), (3, 2), (5, 2), (3, Fraction(1, 3)), (5, 7), (1, Fraction(5, 4))])
def test_exact_rationals(k, z):
    exact = coeffs.rk_exact_rational(k, z)
    assert float(coeffs.rk_eval_pf(k, float(z))) == pytest.approx(float(exact), rel=1e-14)


def test_known_exact_values_at_two():
    assert coeffs.rk_exact_rational(1, 2) == Fraction(2, 3)
    assert coeffs.rk_exact_rational(3, 2) == Fraction(206, 297)
    assert coeffs.rk_exact_rational(5, 2) == Fraction(34966, 50445)


@pytest.mark.parametrize("k", coeffs.ORDERS)
def test_section1_properties(k):
    # r(1) = 0 and r(z) = -r(1/z) (Section 1); r'(1) = 1 because z r'(z) - 1 is
    # minimised to 0 at z = 1; r(0) = -b and r(inf) = b follow from the symmetry.
    b, _, _ = coeffs.rk_coeffs(k)
    assert abs(float(coeffs.rk_eval_pf(k, 1.0))) < 1e-14
    z = np.logspace(-4, 4, 333)
    np.testing.assert_allclose(coeffs.rk_eval_pf(k, z), -coeffs.rk_eval_pf(k, 1.0 / z), rtol=1e-12,
                               atol=1e-13)
    h = 1e-5
    d = (coeffs.rk_eval_pf(k, 1 + h) - coeffs.rk_eval_pf(k, 1 - h)) / (2 * h)
    assert float(d) == pytest.approx(1.0, abs=1e-9)
    assert float(coeffs.rk_eval_pf(k, 0.0)) == pytest.approx(-b, rel=1e-14)
    assert float(coeffs.rk_eval_pf(k, 1e12)) == pytest.approx(b, rel=1e-10)


# Taylor series of log(1+h) - r_k(1+h) at h = 0, expanded by hand from Eq. 1:
# contact of order k+2, with these first three coefficients.
_SERIES = {
    1: [(3, 1 / 12), (4, -1 / 8), (5, 11 / 80)],
    3: [(5, -1 / 320), (6, 1 / 128), (7, -89 / 7168)],
    5: [(7, -1 / 21504), (8, 1 / 6144), (9, -53 / 147456)],
}


@pytest.mark.parametrize("k", coeffs.ORDERS)
def test_order_of_contact_with_log(k):
    # A wrong partial-fraction coefficient changes the low-order terms at once.
    for h in (0.02, 0.04, -0.03):
        err = math.log1p(h) - float(coeffs.rk_eval_pf(k, 1 + h))
        ref = sum(c * h ** p for p, c in _SERIES[k])
        assert err == pytest.approx(ref, rel=2e-2)


def test_error_curve_values():
    # log z - r_k(z) at a few points (the curve plotted in Figure 1): computed from
    # the exact rationals of Eq. 1 and math.log, independent of the partial fractions.
    for k, z in [(1, 2), (3, 2), (5, 2), (3, Fraction(1, 10)), (3, 10)]:
        ref = math.log(float(z)) - float(coeffs.rk_exact_rational(k, z))
        got = math.log(float(z)) - float(coeffs.rk_eval_pf(k, float(z)))
        assert got == pytest.approx(ref, rel=1e-9)
    assert math.log(2) - float(coeffs.rk_exact_rational(3, 2)) == pytest.approx(-4.55513e-4, rel=1e-5)
    assert math.log(2) - float(coeffs.rk_exact_rational(1, 2)) == pytest.approx(0.0264805, rel=1e-5)
