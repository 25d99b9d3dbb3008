"""Shared-memory and image layouts of the tcgen05 kernel products, checked on the
host.  The operands use the canonical no-swizzle K-major layout: 8-row x 16-byte
core matrices, LBO = 128 bytes between core matrices along K, SBO = 1024 bytes
between 8-row groups (for a 64-wide K tile).  Element (row r, k) of a 128 x 64
half-precision tile sits at (r // 8) SBO + (k // 8) LBO + (r % 8) 16 + (k % 8) 2."""
import numpy as np
import pytest

LBO, SBO = 128, 1024


def tile_offset(r, k):
    return (r >> 3) * SBO + (k >> 3) * LBO + (r & 7) * 16 + (k & 7) * 2


def test_tile_layout_is_a_bijection_onto_the_tile():
    r, k = np.meshgrid(np.arange(128), np.arange(64), indexing="ij")
    off = tile_offset(r, k).ravel()
    assert np.array_equal(np.sort(off), np.arange(0, 128 * 64 * 2, 2))


def test_store_of_8_consecutive_k_is_one_16_byte_row_of_a_core_matrix():
    # the eval warps store 8 consecutive k of one row as one 16-byte vector
    for r in (0, 7, 8, 77, 127):
        for kq in range(8):
            offs = [tile_offset(r, 8 * kq + q) for q in range(8)]
            assert offs == list(range(offs[0], offs[0] + 16, 2)) and offs[0] % 16 == 0


@pytest.mark.parametrize("N", [16, 48, 64, 144, 256])
def test_operand_image_of_V_is_a_bijection(N):
    # N columns of V (rows of the B operand) x 64 K values per tile
    col, jj = np.meshgrid(np.arange(N), np.arange(64), indexing="ij")
    off = ((col >> 3) * SBO + (jj >> 3) * LBO + (col & 7) * 16 + (jj & 7) * 2).ravel()
    assert np.array_equal(np.sort(off), np.arange(0, N * 64 * 2, 2))


def test_stored_M_thread_mapping():
    # stored-M mode: warp w, lane l, unit k -> row 16 w + 8 (k >> 1) + l % 8 and column
    # block 4 (k & 1) + l // 8 (8 floats); every (row, block) of the 128 x 64 tile once,
    # each warp-wide load spans 8 rows x one 128-byte line, and each 8-lane phase of the
    # 16-byte shared stores writes 8 rows with distinct r % 8 (distinct banks)
    seen = np.zeros((128, 8), dtype=int)
    for w in range(8):
        for k in range(4):
            lines = set()
            for lane in range(32):
                r = 16 * w + 8 * (k >> 1) + (lane & 7)
                q = 4 * (k & 1) + (lane >> 3)
                seen[r, q] += 1
                lines.add((r, (q * 32) // 128))
            assert len(lines) == 8
            for phase in range(4):
                rows = {(16 * w + 8 * (k >> 1) + (lane & 7)) & 7 for lane in range(8 * phase, 8 * phase + 8)}
                banks = {(tile_offset(r, 0) // 4) % 32 for r in rows}
                assert len(rows) == 8 and len(banks) == 8
    assert np.all(seen == 1)
