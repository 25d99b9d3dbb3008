"""Parity of the kernel product W = (K + noise I) V against the oracle."""
import numpy as np
import pytest

from gpu_util import assert_elementwise, cuda, host, product_scale, torch
from oracle import kernels, splitmix, coeffs
from paper_2405_03474_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [api.RBF, api.MATERN52])
@pytest.mark.parametrize("n,d,c", [(1000, 2, 16), (333, 3, 5), (777, 4, 33), (64, 1, 1), (300, 12, 4), (257, 20, 3)])
def test_kz_fp64_matches_dense_oracle(kind, n, d, c):
    X = inputs.points(n, d, "uniform", seed=3)
    V = inputs.gaussian(n, c, seed=4)
    k = api.Kernel(kind, 0.2, 1.3, 1e-2)
    W = host(api.ld_kz(cuda(X), cuda(V), k, "fp64"))
    M = kernels.kernel_matrix(X, kind, 0.2, 1.3, 1e-2)
    assert_elementwise(W, M @ V, product_scale(M, V), 1e-13)


@pytest.mark.parametrize("kind", [api.RBF, api.MATERN52])
def test_kz_fp32_matches_dense_oracle(kind):
    n, d, c = 1500, 4, 20
    X = inputs.points(n, d, "uniform", seed=5)
    V = inputs.gaussian(n, c, seed=6)
    k = api.Kernel(kind, 0.3, 1.0, 1e-2)
    W = host(api.ld_kz(cuda(X), cuda(V, torch.float32), k, "fp32"))
    M = kernels.kernel_matrix(X, kind, 0.3, 1.0, 1e-2)
    # fp32 sums of n terms: a few sqrt(n) 2^-24 of the sum of magnitudes, plus the input rounding
    assert_elementwise(W, M @ V, product_scale(M, V), FP32_TOL(n))


def test_kz_fp32_sampled_rows_at_large_n():
    n, d, c = 1 << 17, 4, 16
    X = inputs.points(n, d, "uniform", seed=0)
    V = inputs.gaussian(n, c, seed=7)
    k = api.Kernel(api.MATERN52, 0.1, 1.0, 1e-2)
    W = host(api.ld_kz(cuda(X), cuda(V, torch.float32), k, "fp32"))
    rows = np.random.default_rng(0).choice(n, 24, replace=False)
    rows = np.concatenate([rows, [0, n - 1]])
    ref = kernels.kz_rows(X, V, rows, api.MATERN52, 0.1, 1.0, 1e-2)
    scale = kernels.kz_rows(X, np.abs(V), rows, api.MATERN52, 0.1, 1.0, 1e-2)
    assert_elementwise(W[rows], ref, scale, FP32_TOL(n))


@pytest.mark.parametrize("kind", [api.RBF, api.MATERN52])
def test_kz_dl_fp64_matches_oracle(kind):
    n, d, c = 600, 2, 7
    X = inputs.points(n, d, "uniform", seed=8)
    V = inputs.gaussian(n, c, seed=9)
    k = api.Kernel(kind, 0.25, 0.8, 0.0)
    W, Wdl = api.ld_kz_dl(cuda(X), cuda(V), k, "fp64")
    K = kernels.kernel_matrix(X, kind, 0.25, 0.8, 0.0)
    dK = kernels.dkernel_dl_matrix(X, kind, 0.25, 0.8)
    assert_elementwise(host(W), K @ V, product_scale(K, V), 1e-13)
    assert_elementwise(host(Wdl), dK @ V, product_scale(dK, V), 1e-13)


def test_rademacher_bit_exact_with_oracle_splitmix():
    n, s = 10007, 24
    Z = host(api.ld_rademacher(12345, n, s, col0=3))
    ref = splitmix.rademacher_block(12345, n, s, col0=3)
    np.testing.assert_array_equal(Z.astype(np.float64), ref)


@pytest.mark.parametrize("k", [1, 3, 5])
def test_library_coefficients_match_oracle(k):
    b, c, s = api.rk_coeffs(k)
    bo, co, so = coeffs.rk_coeffs(k)
    assert b == bo
    np.testing.assert_allclose(s, so, rtol=2e-15)
    np.testing.assert_allclose(c, co, rtol=2e-14)


# Tensor-core tolerances from the rounding of the operands: fp16 keeps 11 bits
# (2^-11 relative per element), bf16 8 bits (2^-8), and the hi/lo fp16 split
# keeps ~22 bits (2^-21 per product after dropping K_lo V_lo); fp32 accumulation
# over n terms adds ~sqrt(n) 2^-24.
TC_TOL = {"f16_tc": 2.0 ** -9, "bf16_tc": 2.0 ** -6, "f16x3_tc": 2.0 ** -16}


def FP32_TOL(n):
    """Elementwise bound (relative to |K| |V|) of an fp32 product over n terms."""
    return 4 * np.sqrt(n) * 2.0 ** -24 + 2.0 ** -21


@pytest.mark.parametrize("prec", ["f16x3_tc", "f16_tc", "bf16_tc"])
@pytest.mark.parametrize("kind", [api.RBF, api.MATERN52])
@pytest.mark.parametrize("n,d,c", [(1000, 2, 16), (777, 4, 48), (300, 3, 5), (2000, 4, 256), (640, 1, 300),
                                   (1000, 4, 512), (700, 3, 264)])
def test_kz_tensor_core_matches_oracle(prec, kind, n, d, c):
    # (256 < c <= 512 in fp16 / bf16 runs the one-pass wide kernel; hi/lo fp16 above 48 columns
    # the general kernel in 256-column chunks)
    X = inputs.points(n, d, "uniform", seed=11)
    V = inputs.gaussian(n, c, seed=12)
    k = api.Kernel(kind, 0.15, 1.7, 1e-2)
    W = host(api.ld_kz(cuda(X), cuda(V, torch.float32), k, prec))
    M = kernels.kernel_matrix(X, kind, 0.15, 1.7, 1e-2)
    assert_elementwise(W, M @ V, product_scale(M, V), TC_TOL[prec])


def test_kz_wide_sketch_sampled_rows_at_large_n():
    # the sketch product as the preconditioner build calls it: 512 columns, fp16, n = 2^18
    n, d, c = 1 << 18, 4, 512
    X = inputs.points(n, d, "uniform", seed=0)
    V = inputs.gaussian(n, c, seed=8)
    k = api.Kernel(api.MATERN52, 0.1, 1.0, 1e-2)
    W = host(api.ld_kz(cuda(X), cuda(V, torch.float32), k, "f16_tc"))
    rows = np.concatenate([np.random.default_rng(2).choice(n, 12, replace=False), [0, n - 1]])
    ref = kernels.kz_rows(X, V, rows, api.MATERN52, 0.1, 1.0, 1e-2)
    scale = kernels.kz_rows(X, np.abs(V), rows, api.MATERN52, 0.1, 1.0, 1e-2)
    assert_elementwise(W[rows], ref, scale, TC_TOL["f16_tc"])


@pytest.mark.parametrize("c", [270, 512])
def test_kz_wide_two_j_chunks_sampled_rows(c):
    # n just over 1024 j-tiles of 64 points: two grid rows whose partial sums are added into W
    # (vector reductions for c % 4 == 0, per-element ones for c = 270)
    n, d = 66000, 3
    X = inputs.points(n, d, "uniform", seed=4)
    V = inputs.gaussian(n, c, seed=9)
    k = api.Kernel(api.RBF, 0.05, 1.3, 2e-2)
    W = host(api.ld_kz(cuda(X), cuda(V, torch.float32), k, "f16_tc"))
    rows = np.concatenate([np.random.default_rng(5).choice(n, 10, replace=False), [0, n - 1]])
    ref = kernels.kz_rows(X, V, rows, api.RBF, 0.05, 1.3, 2e-2)
    scale = kernels.kz_rows(X, np.abs(V), rows, api.RBF, 0.05, 1.3, 2e-2)
    assert_elementwise(W[rows], ref, scale, TC_TOL["f16_tc"])


def test_kz_f16x3_sampled_rows_at_large_n():
    n, d, c = 1 << 18, 4, 16
    X = inputs.points(n, d, "uniform", seed=0)
    V = inputs.gaussian(n, c, seed=7)
    k = api.Kernel(api.MATERN52, 0.1, 1.0, 1e-2)
    W = host(api.ld_kz(cuda(X), cuda(V, torch.float32), k, "f16x3_tc"))
    rows = np.concatenate([np.random.default_rng(1).choice(n, 24, replace=False), [0, n - 1]])
    ref = kernels.kz_rows(X, V, rows, api.MATERN52, 0.1, 1.0, 1e-2)
    scale = kernels.kz_rows(X, np.abs(V), rows, api.MATERN52, 0.1, 1.0, 1e-2)
    assert_elementwise(W[rows], ref, scale, FP32_TOL(n) + 2.0 ** -19)


def test_kz_bench_workload_sampled_rows():
    # the product exactly as the timed estimate calls it: n = 2^20 Matern-5/2 points
    # in [0,1]^4, lengthscale 0.1, 16 columns (symmetric kernel), hi/lo fp16
    from paper_2405_03474_gb300.inputs import WORKLOADS
    w = WORKLOADS["matern_n1048576_d4"]
    n, d, c = w["n"], w["d"], w["probes"]
    X = inputs.points(n, d, w["dist"], seed=inputs.SEED_POINTS)
    V = inputs.gaussian(n, c, seed=7)
    k = api.Kernel(w["kind"], w["lengthscale"], w["variance"], w["noise"])
    W = host(api.ld_kz(cuda(X), cuda(V, torch.float32), k, "f16x3_tc"))
    rows = np.concatenate([np.random.default_rng(3).choice(n, 30, replace=False), [0, 127, 128, n - 1]])
    ref = kernels.kz_rows(X, V, rows, w["kind"], w["lengthscale"], w["variance"], w["noise"])
    scale = kernels.kz_rows(X, np.abs(V), rows, w["kind"], w["lengthscale"], w["variance"], w["noise"])
    assert_elementwise(W[rows], ref, scale, FP32_TOL(n) + 2.0 ** -19)


# The symmetric product (c <= 48; compiled for 16 and 48 columns): one CTA per
# 128-row block visits half of the blocks, so cover NB = 2 (even, tie rule), odd
# NB, a ragged last block, 1..48 columns on both widths, c * 4 not a multiple of 16
# (per-element adds instead of vector adds) and a dimension above 4 (the generic-d
# instance).
@pytest.mark.parametrize("prec", ["f16x3_tc", "f16_tc", "bf16_tc"])
@pytest.mark.parametrize("kind", [api.RBF, api.MATERN52])
@pytest.mark.parametrize("n,d,c", [(256, 2, 16), (257, 3, 7), (384, 4, 1), (4133, 4, 16), (1536, 1, 12), (700, 6, 9),
                                   (1000, 2, 48), (513, 3, 33), (4133, 4, 17), (2560, 4, 40)])
def test_kz_symmetric_tensor_core_matches_oracle(prec, kind, n, d, c):
    X = inputs.points(n, d, "uniform", seed=31)
    V = inputs.gaussian(n, c, seed=32)
    k = api.Kernel(kind, 0.2, 0.9, 3e-2)
    W = host(api.ld_kz(cuda(X), cuda(V, torch.float32), k, prec))
    M = kernels.kernel_matrix(X, kind, 0.2, 0.9, 3e-2)
    assert_elementwise(W, M @ V, product_scale(M, V), TC_TOL[prec])


# The gradient's derivative pass on the tensor cores: K V and dK/dl V from one sweep,
# 64 columns per launch (100 columns: two launches), ragged n, d up to 6.
@pytest.mark.parametrize("prec", ["f16x3_tc", "f16_tc", "bf16_tc"])
@pytest.mark.parametrize("kind", [api.RBF, api.MATERN52])
@pytest.mark.parametrize("n,d,c", [(1000, 2, 16), (777, 4, 48), (300, 3, 5), (2000, 4, 100), (129, 1, 64),
                                   (700, 6, 7)])
def test_kz_dl_tensor_core_matches_oracle(prec, kind, n, d, c):
    X = inputs.points(n, d, "uniform", seed=13)
    V = inputs.gaussian(n, c, seed=14)
    k = api.Kernel(kind, 0.2, 1.3, 0.0)
    W, Wdl = api.ld_kz_dl(cuda(X), cuda(V, torch.float32), k, prec)
    K = kernels.kernel_matrix(X, kind, 0.2, 1.3, 0.0)
    dK = kernels.dkernel_dl_matrix(X, kind, 0.2, 1.3)
    assert_elementwise(host(W), K @ V, product_scale(K, V), TC_TOL[prec], "K V")
    assert_elementwise(host(Wdl), dK @ V, product_scale(dK, V), TC_TOL[prec], "dK/dl V")


# Repetition: the general, wide and derivative products reduce in a fixed order, so the same
# call must give the same bits every time; a race between the evaluation and MMA sides shows
# up as an occasional wrong tile.  (The symmetric product adds transposed blocks in arrival
# order, so it is repeated against the oracle instead.)
@pytest.mark.parametrize("prec,c", [("bf16_tc", 300), ("f16_tc", 300), ("f16_tc", 264), ("f16x3_tc", 100)])
def test_deterministic_products_repeat_bit_for_bit(prec, c):
    n, d = 5000, 4
    X = cuda(inputs.points(n, d, "uniform", seed=21))
    V = cuda(inputs.gaussian(n, c, seed=23), torch.float32)
    k = api.Kernel(api.RBF, 0.15, 1.2, 1e-2)
    first = api.ld_kz(X, V, k, prec).clone()
    for rep in range(30):
        assert torch.equal(api.ld_kz(X, V, k, prec), first), (prec, c, rep)
    W1, G1 = api.ld_kz_dl(X, V[:, :48].contiguous(), k, "f16x3_tc")
    for rep in range(10):
        W2, G2 = api.ld_kz_dl(X, V[:, :48].contiguous(), k, "f16x3_tc")
        assert torch.equal(W1, W2) and torch.equal(G1, G2), rep


def test_symmetric_product_repeats_against_oracle():
    n, d, c = 5000, 4, 16
    Xh = inputs.points(n, d, "uniform", seed=24)
    Vh = inputs.gaussian(n, c, seed=25)
    k = api.Kernel(api.RBF, 0.15, 1.2, 1e-2)
    M = kernels.kernel_matrix(Xh, api.RBF, 0.15, 1.2, 1e-2)
    X, V = cuda(Xh), cuda(Vh, torch.float32)
    ref, scale = M @ Vh, product_scale(M, Vh)
    for rep in range(15):
        assert_elementwise(host(api.ld_kz(X, V, k, "f16x3_tc")), ref, scale, TC_TOL["f16x3_tc"], "repeat %d" % rep)


# Far blocks of the symmetric product: lengthscale 0.03 over 4133 points in [0,1]^2
# makes 33 Morton-ordered 128-point tiles, most pairs of them far apart, and those
# blocks are rounded once to fp16 instead of split hi/lo.  A far block holds only
# entries <= 2^-10 of the variance, so the error is bounded by the hi/lo bound over
# |M||V|, plus one fp16 rounding (2^-11 relative) of every entry that small, plus the
# spacing of fp16 subnormals (2^-25 of the 2^15-scaled values) for the tiniest ones.
@pytest.mark.parametrize("kind", [api.RBF, api.MATERN52])
@pytest.mark.parametrize("c", [16, 48])
def test_kz_symmetric_far_blocks_within_one_fp16_rounding(kind, c):
    n, d, ell, v, nu = 4133, 2, 0.03, 1.1, 1e-2
    X = inputs.points(n, d, "uniform", seed=41)
    V = inputs.gaussian(n, c, seed=42)
    W = host(api.ld_kz(cuda(X), cuda(V, torch.float32), api.Kernel(kind, ell, v, nu), "f16x3_tc"))
    M = kernels.kernel_matrix(X, kind, ell, v, nu)
    K = np.abs(M - nu * np.eye(n))
    small = np.where(K <= v * 2.0 ** -10, K, 0.0)
    assert (K <= v * 2.0 ** -10).mean() > 0.9  # most pairs are that small (94-96% here)
    bound = (TC_TOL["f16x3_tc"] * product_scale(M, V) + 2.0 ** -11 * (small @ np.abs(V))
             + 2.0 ** -40 * v * np.abs(V).sum(axis=0))
    err = np.abs(W - M @ V)
    assert np.all(err <= bound), float(np.max(err / bound))
