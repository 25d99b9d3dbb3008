"""Pins for oracle/splitmix.py against the published SplitMix64 sequence."""
import numpy as np
import pytest

from oracle import splitmix


def test_published_seed0_sequence():
    # First outputs of SplitMix64 seeded with 0 (Steele, Lea & Flood 2014; the
    # same values as the widely used reference splitmix64.c by S. Vigna).
    got = [int(x) for x in splitmix.splitmix64(0, [0, 1, 2])]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_counter_based_equals_sequential_state():
    # Advancing a state by GAMMA k times equals the closed-form counter access.
    seed = 0x1234_5678_9ABC_DEF0
    state = seed
    seq = []
    for _ in range(50):
        state = (state + 0x9E3779B97F4A7C15) % (1 << 64)
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) % (1 << 64)
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) % (1 << 64)
        seq.append(z ^ (z >> 31))
    got = [int(x) for x in splitmix.splitmix64(seed, np.arange(50))]
    assert got == seq


def test_rademacher_block_layout_and_balance():
    n, s = 1000, 7
    Z = splitmix.rademacher_block(42, n, s)
    assert Z.shape == (n, s)
    assert set(np.unique(Z)) == {-1.0, 1.0}
    # column c, row i uses counter c*n + i
    k = 3 * n + 17
    bit = int(splitmix.splitmix64(42, [k])[0]) >> 63
    assert Z[17, 3] == (1.0 if bit == 0 else -1.0)
    # a later column block continues the same counter space
    Z2 = splitmix.rademacher_block(42, n, 3, col0=4)
    np.testing.assert_array_equal(Z2, Z[:, 4:7])
    big = splitmix.rademacher_block(7, 200000, 1)
    assert abs(big.mean()) < 0.01


def test_gaussian_block_is_standard_normal():
    from scipy import stats
    Z = splitmix.gaussian_block(9, 200000, 2)
    assert Z.shape == (200000, 2)
    # Kolmogorov-Smirnov against N(0, 1) and the first two moments
    assert stats.kstest(Z[:, 0], "norm").pvalue > 1e-3
    assert abs(Z.mean()) < 0.01 and abs(Z.var() - 1.0) < 0.01
    # entry (i, c) is Box-Muller of counters 2k, 2k+1 with k = c n + i
    n = 200000
    k = 1 * n + 123
    u1 = (float(int(splitmix.splitmix64(9, [2 * k])[0]) >> 11) + 0.5) * 2.0 ** -53
    u2 = (float(int(splitmix.splitmix64(9, [2 * k + 1])[0]) >> 11) + 0.5) * 2.0 ** -53
    import math
    assert Z[123, 1] == math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2)


def test_orthogonal_block_structure():
    # columns mutually orthogonal, each of squared norm |h_c|^2 (h_c the chi_n column),
    # and Z^T G upper triangular with a positive diagonal (Q is G's QR factor, not
    # another orthonormal basis of its span)
    n, s = 300, 12
    Z = splitmix.orthogonal_block(4, n, s, col0=5)
    G = splitmix.gaussian_block(4, n, s, col0=5)
    H = splitmix.gaussian_block(4, n, s, col0=splitmix.ORF_NORM_COL0 + 5)
    gram = Z.T @ Z
    h2 = (H ** 2).sum(axis=0)
    np.testing.assert_allclose(np.diag(gram), h2, rtol=1e-12)
    off = gram - np.diag(np.diag(gram))
    assert np.abs(off).max() < 1e-11 * h2.max()
    ZG = Z.T @ G
    assert np.abs(np.tril(ZG, -1)).max() < 1e-10 * np.abs(ZG).max()
    assert (np.diag(ZG) > 0).all()
    # G lies in the span of Z
    coef = np.linalg.lstsq(Z, G, rcond=None)[0]
    np.testing.assert_allclose(Z @ coef, G, atol=1e-10)


def test_orthogonal_block_complete_basis_gives_exact_trace():
    # with s = n the directions form an orthonormal basis: sum_c z_c^T A z_c / |z_c|^2 = tr A
    n = 40
    Z = splitmix.orthogonal_block(8, n, n)
    A = np.random.default_rng(0).standard_normal((n, n))
    A = A + A.T
    val = sum(Z[:, c] @ A @ Z[:, c] / (Z[:, c] @ Z[:, c]) for c in range(n))
    assert val == pytest.approx(np.trace(A), abs=1e-10)


def test_orthogonal_block_marginals_are_standard_normal():
    # each column is marginally N(0, I_n): moments over many blocks, and
    # E |z|^2 = n (chi_n squared)
    from scipy import stats
    n, s = 64, 16
    Z = np.concatenate([splitmix.orthogonal_block(3, n, s, col0=s * b) for b in range(200)], axis=1)
    assert stats.kstest(Z.ravel(), "norm").pvalue > 1e-3
    assert abs(Z.mean()) < 0.01 and abs(Z.var() - 1.0) < 0.01
    assert abs((Z ** 2).sum(axis=0).mean() / n - 1.0) < 0.02
