"""ld_kz_static: the kernel product for callers that cannot allocate device memory.

Such callers (a plug-in inside a framework that owns all device memory, a
latency-critical loop where cudaMalloc would synchronise the device, a process
under a hard memory cap) get the same result as ld_kz from scratch held in a
fixed static device array.  This file is collected last on purpose, and each
check makes two calls in a row because the array keeps the previous call's
contents.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import cuda, host, relerr, torch
from paper_2405_03474_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu

# the tolerances the other kernel-product tests use
TOL = {"fp32": 2e-6, "f16x3_tc": 2.0 ** -16, "f16_tc": 2.0 ** -9}


def _call_static(lib, X, V, W, kern, prec):
    n, d = X.shape
    st = lib.ld_kz_static(ctypes.c_void_p(X.data_ptr()), n, d, kern.c(), ctypes.c_void_p(V.data_ptr()),
                          ctypes.c_void_p(W.data_ptr()), V.shape[1], api.PRECISIONS[prec],
                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("prec", ["f16x3_tc", "f16_tc", "fp32"])
@pytest.mark.parametrize("kind", [api.RBF, api.MATERN52])
def test_static_scratch_matches_ld_kz_twice(prec, kind):
    lib = _lib.load()
    n, d, c = 5000, 4, 16
    X = cuda(inputs.points(n, d, "uniform", seed=21))
    kern = api.Kernel(kind, 0.15, 1.2, 1e-2)
    for call, seed in enumerate((22, 23)):  # two calls in a row, different V
        V = cuda(inputs.gaussian(n, c, seed=seed), torch.float32)
        ref = host(api.ld_kz(X, V, kern, prec))
        W = torch.full_like(V, float("nan"))
        _lib.check(_call_static(lib, X, V, W, kern, prec), "ld_kz_static call %d" % call)
        torch.cuda.synchronize()
        assert relerr(host(W), ref) < TOL[prec]


def test_static_scratch_rejects_sizes_beyond_capacity():
    lib = _lib.load()
    cap = lib.ld_kz_static_capacity()
    assert cap == 32 << 20
    n, d, c = 1 << 21, 5, 16  # fp32 needs n*d*4 = 40 MiB of scaled points
    assert lib.ld_kz_workspace_size(n, d, c, api.PRECISIONS["fp32"]) > cap
    X = torch.zeros((n, d), dtype=torch.float64, device="cuda")
    V = torch.zeros((n, c), dtype=torch.float32, device="cuda")
    W = torch.zeros_like(V)
    st = _call_static(lib, X, V, W, api.Kernel(api.RBF, 0.5, 1.0, 0.0), "fp32")
    assert st == _lib.LD_ERR_WORKSPACE
    assert b"static" in lib.ld_last_error()
