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


# ---- stored M fed by tensor copies (dense_tma.cu): each 128 x 64 fp32 tile of M arrives
# as two boxes of 128 rows x 32 floats in the 128-byte swizzled layout, box b at byte
# 16384 b, row r at 128 r, 16-byte chunk c of the row at chunk c ^ (r % 8).
def tma_tile_offset(r, col):
    b, c = col // 32, (col % 32) // 4
    return b * 16384 + r * 128 + ((c ^ (r % 8)) * 16) + (col % 4) * 4


def test_swizzled_M_tile_is_a_bijection_onto_32_KB():
    r, col = np.meshgrid(np.arange(128), np.arange(64), indexing="ij")
    off = tma_tile_offset(r, col).ravel()
    assert np.array_equal(np.sort(off), np.arange(0, 128 * 64 * 4, 4))


def test_swizzled_M_reads_of_the_eval_threads():
    # the eval thread of unit k (row 16 w + 8 (k >> 1) + l % 8, columns 8 q .. 8 q + 7 with
    # q = 4 (k & 1) + l // 8) reads its 8 floats as two 16-byte loads at
    # box q // 4, row r, chunks 2 (q % 4) and + 1 swizzled by r % 8: the same bytes the
    # tensor copy wrote there, and every 8-lane phase of a load hits 8 distinct 16-byte
    # bank groups (no conflicts)
    for w in range(8):
        for k in range(4):
            for which in (0, 1):
                for phase in range(4):
                    groups = set()
                    for lane in range(8 * phase, 8 * phase + 8):
                        r = 16 * w + 8 * (k >> 1) + (lane & 7)
                        q = 4 * (k & 1) + (lane >> 3)
                        c0 = 2 * (q & 3) + which
                        kern = (q >> 2) * 16384 + r * 128 + ((c0 ^ (r & 7)) << 4)
                        assert kern == tma_tile_offset(r, 8 * q + 4 * which)
                        assert kern + 16 <= 128 * 64 * 4
                        groups.add((kern // 16) % 8)
                    assert len(groups) == 8


def _dense_tma_smem(N, nprod, stages):
    # barriers (1 KB), M stages (32 KB each), two V image stages, two fp16 operand tiles, slack
    b = (2 if nprod == 3 else 1) * N * 64 * 2
    vstage = (b + 1023) // 1024 * 1024
    return 1024 + stages * 32768 + 2 * vstage + 2 * (2 if nprod == 3 else 1) * 16384 + 1024


@pytest.mark.parametrize("nprod", [1, 3])
def test_dense_tma_shared_memory_fits_with_at_least_three_M_stages(nprod):
    # 16 <= N <= 128 columns per launch: the stage count the host picks (most of 6..2 under
    # 226 KB) leaves at least 3 M stages and stays within the 227 KB a CTA may use; every
    # region starts 1024-aligned (the 128-byte swizzle needs it for the M stages)
    for N in range(16, 129, 16):
        stages = next(s for s in (6, 5, 4, 3, 2) if _dense_tma_smem(N, nprod, s) <= 226 * 1024)
        assert stages >= 3 and _dense_tma_smem(N, nprod, stages) <= 232448
        assert (2 if nprod == 3 else 1) * N * 64 * 2 % 16 == 0  # bulk copy of the V image


@pytest.mark.parametrize("ntiles", [2, 3, 16, 17, 1024, 1025])
@pytest.mark.parametrize("split", [1, 2])
def test_split_row_blocks_cover_every_tile_once(ntiles, split):
    # part p of a row block takes tiles [ntiles p / split, ntiles (p + 1) / split)
    tiles = []
    for p in range(split):
        t0, t1 = ntiles * p // split, ntiles * (p + 1) // split
        assert t1 > t0
        tiles += range(t0, t1)
    assert tiles == list(range(ntiles))
