"""Stored dense M = K + noise I (the rbf_n65536_d3 workload keeps M in HBM) against the oracle."""
import numpy as np
import pytest

from gpu_util import assert_elementwise, cuda, host, product_scale, relerr, torch
from oracle import estimator, kernels, precond
from oracle.splitmix import rademacher_block
from paper_2405_03474_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [api.RBF, api.MATERN52])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-14), ("fp32", 1e-6)])
def test_materialize_and_product_match_oracle(kind, prec, tol):
    n, d, c = 1000, 3, 24
    X = inputs.points(n, d, "normal", seed=1)
    k = api.Kernel(kind, 0.5, 1.3, 1e-3)
    M = api.ld_dense_materialize(cuda(X), k, prec)
    Mo = kernels.kernel_matrix(X, kind, 0.5, 1.3, 1e-3)
    assert np.abs(host(M) - Mo).max() < tol * 10
    V = inputs.gaussian(n, c, seed=2)
    dt = torch.float64 if prec == "fp64" else torch.float32
    W = api.ld_dense_kz(M, cuda(V, dt), prec)
    assert_elementwise(host(W), Mo @ V, product_scale(Mo, V), tol * 10)


@pytest.mark.parametrize("order", [1, 3, 5])
def test_dense_estimate_equals_matrix_free_and_oracle(order):
    n, s = 2000, 8
    X = inputs.points(n, 3, "normal", seed=0)
    k = api.Kernel(api.RBF, 0.5, 1.0, 1e-2)
    M = kernels.kernel_matrix(X, kernels.RBF, 0.5, 1.0, 1e-2)
    A, D = precond.build(M, rademacher_block(2, n, 32), 2, 1e-2)
    F = precond.factors(A, D)
    Z = inputs.rademacher(n, s, seed=1)
    P = api.Precond.import_(A, D, "fp64")
    common = dict(precond=P, probes=cuda(Z), order=order, num_probes=s, precision="fp64", rel_tol=1e-12,
                  max_iters=3000)
    rd = api.logdet_estimate(cuda(X), k, dense=True, **common)
    rf = api.logdet_estimate(cuda(X), k, dense=False, **common)
    assert rd["logdet"] == pytest.approx(rf["logdet"], rel=1e-12)
    est, _, _ = estimator.estimate_converged(precond.operator_B(M, F), F["logdet_P"], Z.astype(np.float64), order)
    assert rd["logdet"] == pytest.approx(est, rel=1e-10)


def test_dense_fp32_estimate_within_1e4():
    n, s = 4096, 16
    X = inputs.points(n, 3, "normal", seed=0)
    k = api.Kernel(api.RBF, 0.5, 1.0, 1e-3)
    M = kernels.kernel_matrix(X, kernels.RBF, 0.5, 1.0, 1e-3)
    A, D = precond.build(M, rademacher_block(2, n, 64), 2, 1e-3)
    F = precond.factors(A, D)
    Z = inputs.rademacher(n, s, seed=1)
    P = api.Precond.import_(A, D, "fp32")
    r = api.logdet_estimate(cuda(X), k, precond=P, probes=cuda(Z), order=3, num_probes=s, precision="fp32",
                            rel_tol=1e-6, max_iters=3000, dense=True)
    est, _, _ = estimator.estimate_converged(precond.operator_B(M, F), F["logdet_P"], Z.astype(np.float64), 3)
    assert r["logdet"] == pytest.approx(est, rel=1e-4)


# Tensor-core product of a stored M: the same rounding as the computed kernel values
# (fp16 11 bits, bf16 8 bits, hi/lo fp16 ~22 bits), plus the fp32 rounding of M itself.
TC_TOL = {"f16_tc": 2.0 ** -9, "bf16_tc": 2.0 ** -6, "f16x3_tc": 2.0 ** -16}


@pytest.mark.parametrize("prec", ["f16x3_tc", "f16_tc", "bf16_tc"])
@pytest.mark.parametrize("n,c,variance", [(1000, 16, 1.3), (777, 5, 1.3), (2049, 64, 0.7), (300, 300, 1.0),
                                          (128, 1, 1.0), (640, 130, 2.5), (1500, 24, 1e-3), (1100, 64, 1.0),
                                          (2052, 96, 0.9), (4100, 128, 1.1), (516, 48, 1.0)])
def test_dense_tensor_core_product_matches_oracle(prec, n, c, variance):
    # n % 4 == 0 with n >= 128 and at most 128 columns streams M by tensor copies (the
    # last tile of n = 1100 has a second box wholly past column n, n = 2052 leaves 4
    # columns in its last tile, 4100 rows end 4 into a row block; 96 and 128 columns
    # use the 512-column accumulator and two stages with the hi/lo split); other n read
    # M per thread (n % 4 != 0 per element); 300 columns run two 256-column chunks; 130
    # columns (N = 144) accumulate hi/lo without drains; a variance of 1e-3 checks the
    # power-of-two scale taken from the diagonal
    kind = api.MATERN52 if n % 2 else api.RBF
    X = inputs.points(n, 3, "normal", seed=5)
    k = api.Kernel(kind, 0.4, variance, 1e-2 * variance)
    M = api.ld_dense_materialize(cuda(X), k, "fp32")
    V = inputs.gaussian(n, c, seed=6)
    W = host(api.ld_dense_kz(M, cuda(V, torch.float32), prec))
    Mo = kernels.kernel_matrix(X, kind, 0.4, variance, 1e-2 * variance)
    assert_elementwise(W, Mo @ V, product_scale(Mo, V), TC_TOL[prec])


@pytest.mark.parametrize("order", [1, 3, 5])
def test_dense_tensor_core_estimate_matches_oracle(order):
    n, s = 2000, 16
    X = inputs.points(n, 3, "normal", seed=0)
    k = api.Kernel(api.RBF, 0.5, 1.0, 1e-2)
    M = kernels.kernel_matrix(X, kernels.RBF, 0.5, 1.0, 1e-2)
    A, D = precond.build(M, rademacher_block(2, n, 32), 2, 1e-2)
    F = precond.factors(A, D)
    Z = inputs.rademacher(n, s, seed=1)
    P = api.Precond.import_(A, D, "fp32")
    r = api.logdet_estimate(cuda(X), k, precond=P, probes=cuda(Z), order=order, num_probes=s, precision="f16x3_tc",
                            rel_tol=1e-6, max_iters=3000, dense=True)
    est, _, _ = estimator.estimate_converged(precond.operator_B(M, F), F["logdet_P"], Z.astype(np.float64), order)
    assert r["logdet"] == pytest.approx(est, rel=1e-4)


def test_rbf_n65536_stored_dense_at_full_size():
    # The stored-dense workload at its stated size: n = 65536 points N(0, I_3), RBF,
    # lengthscale 0.5, noise 1e-3, M in fp32 (16 GiB), 64 probes, rank 256.  The oracle
    # checks sampled rows of M and of M V; the FP32 and hi/lo fp16 tensor-core estimates
    # (same probes, preconditioner and t) must agree to the reduced-precision bar.
    import time
    from paper_2405_03474_gb300.inputs import SEED_POINTS, SEED_PROBES, WORKLOADS
    w = WORKLOADS["rbf_n65536_d3"]
    n, d, s = w["n"], w["d"], w["probes"]
    X = inputs.points(n, d, w["dist"], seed=SEED_POINTS)
    k = api.Kernel(w["kind"], w["lengthscale"], w["variance"], w["noise"])
    Xt = cuda(X)
    M = api.ld_dense_materialize(Xt, k, "fp32")
    rows = np.concatenate([np.random.default_rng(4).choice(n, 20, replace=False), [0, n - 1]])
    Mrows = kernels.kernel_of_r2(kernels.sqdist(X[rows], X), w["kind"], w["lengthscale"], w["variance"])
    Mrows[np.arange(len(rows)), rows] += w["noise"]
    assert np.abs(host(M[torch.as_tensor(rows).cuda()]) - Mrows).max() < 1e-5
    V = inputs.gaussian(n, s, seed=2)
    Vt = cuda(V, torch.float32)
    ref = kernels.kz_rows(X, V, rows, w["kind"], w["lengthscale"], w["variance"], w["noise"])
    scale = kernels.kz_rows(X, np.abs(V), rows, w["kind"], w["lengthscale"], w["variance"], w["noise"])
    fp32_bound = 4 * np.sqrt(n) * 2.0 ** -24 + 2.0 ** -21
    tol = {"fp32": fp32_bound, "f16x3_tc": fp32_bound + 2.0 ** -19, "f16_tc": TC_TOL["f16_tc"],
           "bf16_tc": TC_TOL["bf16_tc"]}
    for prec in ("fp32", "f16x3_tc", "f16_tc", "bf16_tc"):
        W = api.ld_dense_kz(M, Vt, prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        W = api.ld_dense_kz(M, Vt, prec)
        torch.cuda.synchronize()
        ms = 1e3 * (time.perf_counter() - t0)
        err = relerr(host(W)[rows], ref)
        print("dense product n=%d c=%d %s: %.2f ms (%.0f GB/s of M), rel err %.2e"
              % (n, s, prec, ms, 4.0 * n * n / ms / 1e6, err))
        assert_elementwise(host(W)[rows], ref, scale, tol[prec], what=prec)
    del M, W
    P = api.Precond.build(Xt, k, w["rank"], power_iters=w["power_iters"], seed=2, precision="f16_tc")
    Z = cuda(inputs.rademacher(n, s, seed=SEED_PROBES))
    res = {}
    for prec in ("fp32", "f16x3_tc"):
        t0 = time.perf_counter()
        res[prec] = api.logdet_estimate(Xt, k, precond=P, probes=Z, order=w["order"], num_probes=s, precision=prec,
                                        fixed_iters=40, max_iters=40, dense=True)
        print("dense estimate %s: log det %.6f (trace %.6f), %.2f s"
              % (prec, res[prec]["logdet"], res[prec]["trace_est"], time.perf_counter() - t0))
    assert res["f16x3_tc"]["logdet"] == pytest.approx(res["fp32"]["logdet"], rel=1e-4)


def test_rbf_n65536_orders_and_precisions_against_fp64():
    # The stored-dense workload as stated: r_1, r_3 and r_5 with a rank-256 preconditioner
    # and 64 probes, M stored (fp64 for the reference, fp32 for the others), the estimate
    # in FP32 (CUDA-core GEMM), hi/lo fp16 and bf16 on the tensor cores, each against the
    # FP64 estimate on the same probes, preconditioner and t (the FP64 path matches the
    # oracle to 1e-10 at every size it can check).
    import time
    from paper_2405_03474_gb300.inputs import SEED_POINTS, SEED_PROBES, WORKLOADS
    w = WORKLOADS["rbf_n65536_d3"]
    n, d, s, t = w["n"], w["d"], w["probes"], 40
    X = inputs.points(n, d, w["dist"], seed=SEED_POINTS)
    k = api.Kernel(w["kind"], w["lengthscale"], w["variance"], w["noise"])
    Xt = cuda(X)
    P32 = api.Precond.build(Xt, k, w["rank"], power_iters=w["power_iters"], seed=2, precision="f16_tc")
    A, D, _ = P32.export()
    P64 = api.Precond.import_(A, D, "fp64")
    del A, D
    Z = cuda(inputs.rademacher(n, s, seed=SEED_PROBES))
    from paper_2405_03474_gb300 import _lib
    for order in (1, 3, 5):
        res = {}
        for prec in ("fp64", "fp32", "f16x3_tc", "bf16_tc"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                res[prec] = api.logdet_estimate(Xt, k, precond=P64 if prec == "fp64" else P32, probes=Z,
                                                order=order, num_probes=s, precision=prec, fixed_iters=t,
                                                max_iters=t, dense=True)
            except _lib.LogdetError as e:
                # bf16 kernel values (8 bits) perturb M by ~2^-9 of its row sums, far above the
                # noise 1e-3: the operator is not positive definite and CG says so
                assert prec == "bf16_tc" and e.status == _lib.LD_ERR_NOT_SPD, (prec, str(e))
                print("rbf_n65536 r_%d %s: %s" % (order, prec, e))
                continue
            sec = time.perf_counter() - t0
            ref = res["fp64"]["logdet"]
            print("rbf_n65536 r_%d %s: log det %.6f, %.2f s, rel err vs FP64 %.2e"
                  % (order, prec, res[prec]["logdet"], sec, abs(res[prec]["logdet"] / ref - 1)))
        for prec in ("fp32", "f16x3_tc"):
            assert res[prec]["logdet"] == pytest.approx(res["fp64"]["logdet"], rel=1e-4), (order, prec)
