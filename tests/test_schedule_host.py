"""The block schedule of the symmetric kernel product, checked exhaustively on the
host: CTA I visits J = (I + b) mod NB for b < T(I), with T = NB/2 + 1 for odd NB and,
for even NB, NB/2 + 1 when I < NB/2 else NB/2 (the block at distance NB/2 goes to
the smaller I only).  Every unordered pair of 128-row blocks, the diagonal blocks
included, must be evaluated exactly once, and the work per CTA differs by at most
one block."""
import numpy as np
import pytest


def visit_counts(NB):
    H = NB // 2
    I = np.arange(NB)
    T = np.full(NB, H + 1) if NB % 2 else np.where(I < H, H + 1, H)
    b = np.arange(H + 1)
    II = np.broadcast_to(I[:, None], (NB, H + 1))
    JJ = (II + b[None, :]) % NB
    take = b[None, :] < T[:, None]
    lo, hi = np.minimum(II, JJ)[take], np.maximum(II, JJ)[take]
    return np.bincount(lo * NB + hi, minlength=NB * NB).reshape(NB, NB), T


@pytest.mark.parametrize("NB", list(range(1, 130)) + [512, 1023, 8192])  # 8192: n = 2^20
def test_every_block_pair_once(NB):
    counts, T = visit_counts(NB)
    upper = np.triu(np.ones((NB, NB), dtype=bool))
    assert np.all(counts[upper] == 1)
    assert np.all(counts[~upper] == 0)
    assert T.max() - T.min() <= 1
