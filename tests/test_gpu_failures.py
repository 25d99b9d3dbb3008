"""Failure paths that fault, trap or hang nothing: bounded device waits report a
status, bad arguments are refused on the host, CG reports non-convergence."""
import ctypes

import numpy as np
import pytest

from gpu_util import assert_elementwise, cuda, host, product_scale, torch
from oracle import kernels
from paper_2405_03474_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu


def test_device_wait_times_out_and_context_stays_usable():
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.ld_selftest_wait_timeout(20_000_000, stream)  # ~10 ms at 2 GHz
    assert st == _lib.LD_ERR_DEVICE_TIMEOUT
    assert b"gave up" in lib.ld_last_error()
    # the context still runs work correctly
    X = inputs.points(500, 2, "uniform", seed=1)
    V = inputs.gaussian(500, 16, seed=2)
    W = host(api.ld_kz(cuda(X), cuda(V, torch.float32), api.Kernel(api.RBF, 0.3, 1.0, 1e-2), "f16x3_tc"))
    M = kernels.kernel_matrix(X, kernels.RBF, 0.3, 1.0, 1e-2)
    assert_elementwise(W, M @ V, product_scale(M, V), 2.0 ** -16)


def test_not_converged_is_reported_with_the_result_filled():
    n = 800
    X = cuda(inputs.points(n, 2, "uniform", seed=3))
    res = api.logdet_estimate(X, api.Kernel(api.MATERN52, 0.3, 1.0, 1e-3), order=3, num_probes=4,
                              precision="fp64", rel_tol=1e-14, max_iters=3, allow_not_converged=True)
    assert res["status"] == _lib.LD_ERR_NOT_CONVERGED
    assert res["iters"] == 3 and np.isfinite(res["logdet"]) and res["final_rel_resid"] > 1e-14


def test_invalid_arguments_are_refused_on_the_host():
    X = cuda(inputs.points(100, 2, "uniform", seed=4))
    with pytest.raises(_lib.LogdetError) as e:
        api.logdet_estimate(X, api.Kernel(api.RBF, -1.0, 1.0, 0.0), num_probes=4)
    assert e.value.status == _lib.LD_ERR_INVALID
    with pytest.raises(_lib.LogdetError) as e:
        api.logdet_estimate(X, api.Kernel(api.RBF, 0.5, 1.0, 0.0), order=4, num_probes=4)
    assert e.value.status == _lib.LD_ERR_INVALID
    with pytest.raises(_lib.LogdetError):
        api.Precond.build(X, api.Kernel(api.RBF, 0.5, 1.0, 1e-2), rank=200)  # rank > n
    P = api.Precond.import_(np.zeros((50, 0)), np.ones(50), "fp64")
    with pytest.raises(_lib.LogdetError):  # handle built for another n
        api.logdet_estimate(X, api.Kernel(api.RBF, 0.5, 1.0, 1e-2), precond=P, num_probes=4, precision="fp64")


def test_workspace_too_small_is_refused():
    lib = _lib.load()
    n, d, c = 1000, 2, 16
    X = cuda(inputs.points(n, d, "uniform", seed=5))
    V = cuda(inputs.gaussian(n, c, seed=6), torch.float32)
    W = torch.empty_like(V)
    need = lib.ld_kz_workspace_size(n, d, c, api.PRECISIONS["f16x3_tc"])
    ws = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    st = lib.ld_kz(ctypes.c_void_p(X.data_ptr()), n, d, api.Kernel(api.RBF, 0.3).c(), ctypes.c_void_p(V.data_ptr()),
                   ctypes.c_void_p(W.data_ptr()), c, api.PRECISIONS["f16x3_tc"], ctypes.c_void_p(ws.data_ptr()),
                   need // 2, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.LD_ERR_WORKSPACE


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_points_are_refused(bad):
    # a NaN or Inf coordinate is reported by the estimator and the preconditioner build
    X = inputs.points(300, 2, "uniform", seed=7)
    X[5, 1] = bad
    k = api.Kernel(api.RBF, 0.3, 1.0, 1e-2)
    with pytest.raises(_lib.LogdetError) as e:
        api.logdet_estimate(cuda(X), k, order=3, num_probes=4, precision="fp64", fixed_iters=5, max_iters=5)
    assert e.value.status == _lib.LD_ERR_INVALID and "non-finite" in str(e.value)
    with pytest.raises(_lib.LogdetError) as e:
        api.Precond.build(cuda(X), k, 8, precision="fp64")
    assert e.value.status == _lib.LD_ERR_INVALID and "non-finite" in str(e.value)
