"""SplitMix64 counter-based generator and the Rademacher draws made from it.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Algorithm 1 step 1 draws s probe vectors with i.i.d. entries from a mean-0,
variance-1 distribution; Section 3 uses Rademacher entries (+1 or -1 with
probability 1/2).  When the device draws probes itself it cannot be handed the
host's numbers, so both sides implement one published counter-based
generator, written independently from its definition:

SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): the state advances by the odd constant
GAMMA = 0x9E3779B97F4A7C15 and each output is the state passed through the
"mix64" finaliser (xor-shift 30, multiply, xor-shift 27, multiply,
xor-shift 31).  The k-th output (k = 0, 1, ...) of the stream seeded with
``seed`` is therefore mix64(seed + (k + 1) * GAMMA) mod 2^64, which makes the
generator counter-based.

Entry (i, c) of an n-by-s block (column-major, probe c, row i) uses counter
k = c * n + i and is +1 when bit 63 of the output is 0, else -1.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MUL1 = np.uint64(0xBF58476D1CE4E5B9)
MUL2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, counters):
    """k-th outputs of the SplitMix64 stream for an array of counters k."""
    k = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (k + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * MUL1
        z = (z ^ (z >> np.uint64(27))) * MUL2
        z = z ^ (z >> np.uint64(31))
    return z


def rademacher_block(seed, n, s, col0=0):
    """n-by-s Rademacher block (float64, +-1) for columns col0 .. col0+s-1."""
    cols = np.arange(col0, col0 + s, dtype=np.uint64)
    rows = np.arange(n, dtype=np.uint64)
    k = cols[None, :] * np.uint64(n) + rows[:, None]
    bits = splitmix64(seed, k) >> np.uint64(63)
    return 1.0 - 2.0 * bits.astype(np.float64)


def uniform_open(seed, counters):
    """(0, 1) uniforms from the top 53 bits of the SplitMix64 outputs: (m + 0.5) 2^-53."""
    m = splitmix64(seed, counters) >> np.uint64(11)
    return (m.astype(np.float64) + 0.5) * 2.0 ** -53


def gaussian_block(seed, n, s, col0=0):
    """n-by-s N(0, 1) block by the Box-Muller transform (Box & Muller 1958): entry
    (i, c) uses the uniforms of counters 2k and 2k + 1, k = (col0 + c) n + i, and is
    sqrt(-2 ln u1) cos(2 pi u2)."""
    cols = np.arange(col0, col0 + s, dtype=np.uint64)
    rows = np.arange(n, dtype=np.uint64)
    k = cols[None, :] * np.uint64(n) + rows[:, None]
    u1 = uniform_open(seed, np.uint64(2) * k)
    u2 = uniform_open(seed, np.uint64(2) * k + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


ORF_NORM_COL0 = 1 << 30


def orthogonal_block(seed, n, s, col0=0):
    """n-by-s block of normal orthogonal probes (the Appendix's probe type, an
    application of Orthogonal Monte Carlo, Yu et al. 2016): W = S Q.

    Reading: Q has the orthonormal columns of the QR factorisation, R's diagonal
    taken positive, of the Gaussian block of columns col0 .. col0+s-1 (a Haar
    distributed set of s orthonormal vectors); S is diagonal with chi_n entries,
    column c's being the Euclidean norm of the Gaussian column
    ORF_NORM_COL0 + col0 + c of the same stream.  Requires s <= n."""
    G = gaussian_block(seed, n, s, col0)
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))
    H = gaussian_block(seed, n, s, ORF_NORM_COL0 + col0)
    return Q * np.sqrt(np.einsum("ij,ij->j", H, H))
