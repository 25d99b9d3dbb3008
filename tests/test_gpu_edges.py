"""Edge cases of the CUDA path against the oracle: empty inputs, a single point,
sizes below, at and just past one tile, the largest dimension of the
tensor-core path, one probe per block."""
import ctypes

import numpy as np
import pytest

from gpu_util import assert_elementwise, cuda, host, product_scale, torch
from oracle import estimator, kernels, precond
from oracle.splitmix import rademacher_block
from paper_2405_03474_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu

# elementwise, relative to |K| |V| (see gpu_util.assert_elementwise)
TOL = {"fp64": 1e-12, "fp32": 1e-5, "f16x3_tc": 2.0 ** -16, "f16_tc": 2.0 ** -9}


def test_empty_inputs_are_refused():
    lib = _lib.load()
    X = cuda(inputs.points(10, 2, "uniform", seed=1))
    V = torch.zeros((10, 1), dtype=torch.float32, device="cuda")
    W = torch.empty_like(V)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, c in ((0, 1), (10, 0)):
        st = lib.ld_kz(ctypes.c_void_p(X.data_ptr()), n, 2, api.Kernel(api.RBF, 0.3).c(), ctypes.c_void_p(V.data_ptr()),
                       ctypes.c_void_p(W.data_ptr()), c, api.PRECISIONS["fp32"], None, 0, stream)
        assert st == _lib.LD_ERR_INVALID


def test_single_point_estimate_is_exact():
    # n = 1 with the diagonal preconditioner: P = M, B = 1, r_k(1) = 0, log det M = log(v + nu)
    X = cuda(np.array([[0.3, 0.7]]))
    k = api.Kernel(api.MATERN52, 0.5, 1.7, 0.2)
    P = api.Precond.build(X, k, 0, precision="fp64")
    res = api.logdet_estimate(X, k, precond=P, order=3, num_probes=2, probes_per_block=1, precision="fp64",
                              rel_tol=1e-12, max_iters=10)
    assert res["logdet"] == pytest.approx(np.log(1.7 + 0.2), rel=1e-14)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16x3_tc"])
@pytest.mark.parametrize("n", [1, 2, 63, 127, 129, 255, 257])
def test_sizes_around_one_tile(prec, n):
    X = inputs.points(n, 3, "uniform", seed=n)
    V = inputs.gaussian(n, 16, seed=n + 1)
    k = api.Kernel(api.MATERN52, 0.3, 1.2, 5e-2)
    dt = torch.float64 if prec == "fp64" else torch.float32
    W = host(api.ld_kz(cuda(X), cuda(V, dt), k, prec))
    M = kernels.kernel_matrix(X, api.MATERN52, 0.3, 1.2, 5e-2)
    assert_elementwise(W, M @ V, product_scale(M, V), TOL[prec])


@pytest.mark.parametrize("n,c", [(129, 300), (257, 512), (300, 49)])
def test_wide_and_general_products_just_past_a_tile(n, c):
    X = inputs.points(n, 2, "uniform", seed=c)
    V = inputs.gaussian(n, c, seed=c + 1)
    k = api.Kernel(api.RBF, 0.2, 1.0, 1e-2)
    prec = "f16_tc" if c > 256 else "f16x3_tc"
    W = host(api.ld_kz(cuda(X), cuda(V, torch.float32), k, prec))
    M = kernels.kernel_matrix(X, api.RBF, 0.2, 1.0, 1e-2)
    assert_elementwise(W, M @ V, product_scale(M, V), TOL[prec])


def test_largest_tensor_core_dimension():
    n, d, c = 700, 8, 16
    X = inputs.points(n, d, "uniform", seed=8)
    V = inputs.gaussian(n, c, seed=9)
    k = api.Kernel(api.MATERN52, 0.8, 1.0, 1e-2)
    W = host(api.ld_kz(cuda(X), cuda(V, torch.float32), k, "f16x3_tc"))
    M = kernels.kernel_matrix(X, api.MATERN52, 0.8, 1.0, 1e-2)
    assert_elementwise(W, M @ V, product_scale(M, V), TOL["f16x3_tc"])


def test_one_probe_per_block_matches_oracle():
    n, s, r = 600, 3, 12
    X = inputs.points(n, 2, "uniform", seed=10)
    M = kernels.kernel_matrix(X, api.RBF, 0.3, 1.0, 3e-2)
    A, D = precond.build(M, rademacher_block(2, n, r), 2, 3e-2)
    F = precond.factors(A, D)
    Z = inputs.rademacher(n, s, seed=11)
    P = api.Precond.import_(A, D, "fp64")
    res = api.logdet_estimate(cuda(X), api.Kernel(api.RBF, 0.3, 1.0, 3e-2), precond=P, probes=cuda(Z), order=5,
                              num_probes=s, probes_per_block=1, precision="fp64", rel_tol=1e-13, max_iters=3000)
    est, _, _ = estimator.estimate_converged(precond.operator_B(M, F), F["logdet_P"], Z.astype(np.float64), 5)
    assert res["logdet"] == pytest.approx(est, rel=1e-10)
