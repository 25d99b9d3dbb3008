"""ld_kz_static: the kernel product for callers that cannot allocate device memory.

Such callers (a plug-in inside a framework that owns all device memory, a
latency-critical loop where cudaMalloc would synchronise the device, a process
under a hard memory cap) get the same result as ld_kz from scratch held in a
fixed static device array.  This file is collected last on purpose.  Each check
makes two calls in a row with different column counts, so the second call runs
over what the first left in the shared array, laid out differently (symmetric,
general, wide and SIMT products), and compares both calls with ld_kz (the
tolerance the other kernel-product tests use) and, element by element, with the
CPU FP64 oracle.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import assert_elementwise, cuda, host, product_scale, torch
from oracle import kernels
from paper_2405_03474_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu

# the tolerances the other kernel-product tests use (elementwise, relative to |K| |V|)
TOL = {"fp64": 1e-13, "fp32": 4 * np.sqrt(5000) * 2.0 ** -24 + 2.0 ** -21, "f16x3_tc": 2.0 ** -16,
       "f16_tc": 2.0 ** -9, "bf16_tc": 2.0 ** -6}

# (precision, columns) of two calls in a row: symmetric (<= 48 columns), general
# (49..256 in hi/lo fp16), one-pass wide (257..512 in fp16/bf16) and SIMT products
PAIRS = [
    (("f16x3_tc", 16), ("f16x3_tc", 100)),
    (("f16x3_tc", 100), ("f16x3_tc", 48)),
    (("f16_tc", 300), ("f16_tc", 16)),
    (("bf16_tc", 40), ("bf16_tc", 300)),
    (("fp64", 16), ("fp64", 7)),
    (("fp32", 16), ("f16x3_tc", 33)),
]


def _call_static(lib, X, V, W, kern, prec):
    n, d = X.shape
    st = lib.ld_kz_static(ctypes.c_void_p(X.data_ptr()), n, d, kern.c(), ctypes.c_void_p(V.data_ptr()),
                          ctypes.c_void_p(W.data_ptr()), V.shape[1], api.PRECISIONS[prec],
                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("pair", PAIRS, ids=["%s%d-%s%d" % (a[0], a[1], b[0], b[1]) for a, b in PAIRS])
@pytest.mark.parametrize("kind", [api.RBF, api.MATERN52])
def test_static_scratch_matches_ld_kz_and_oracle_twice(pair, kind):
    lib = _lib.load()
    n, d = 5000, 4
    Xh = inputs.points(n, d, "uniform", seed=21)
    X = cuda(Xh)
    kern = api.Kernel(kind, 0.15, 1.2, 1e-2)
    M = kernels.kernel_matrix(Xh, kind, 0.15, 1.2, 1e-2)
    for call, ((prec, c), seed) in enumerate(zip(pair, (22, 23))):
        Vh = inputs.gaussian(n, c, seed=seed)
        dt = torch.float64 if prec == "fp64" else torch.float32
        V = cuda(Vh, dt)
        ref = host(api.ld_kz(X, V, kern, prec))
        W = torch.full_like(V, float("nan"))
        _lib.check(_call_static(lib, X, V, W, kern, prec), "ld_kz_static call %d" % call)
        torch.cuda.synchronize()
        got = host(W)
        scale = product_scale(M, Vh)
        assert_elementwise(got, ref, scale, TOL[prec], "call %d (%s, %d columns) vs ld_kz" % (call, prec, c))
        assert_elementwise(got, M @ Vh, scale, TOL[prec], "call %d (%s, %d columns) vs oracle" % (call, prec, c))


def test_static_scratch_accepts_ld_kz_dimensions():
    # FP32 / FP64 take d up to 32 like ld_kz; the tensor-core precisions d <= 8
    lib = _lib.load()
    n, d, c = 600, 12, 5
    Xh = inputs.points(n, d, "uniform", seed=24)
    Vh = inputs.gaussian(n, c, seed=25)
    kern = api.Kernel(api.RBF, 0.9, 1.0, 1e-2)
    M = kernels.kernel_matrix(Xh, api.RBF, 0.9, 1.0, 1e-2)
    V = cuda(Vh, torch.float32)
    W = torch.empty_like(V)
    _lib.check(_call_static(lib, cuda(Xh), V, W, kern, "fp32"), "ld_kz_static d = 12")
    torch.cuda.synchronize()
    assert_elementwise(host(W), M @ Vh, product_scale(M, Vh), 1e-5, "d = 12 fp32")
    assert _call_static(lib, cuda(Xh), V, W, kern, "f16x3_tc") == _lib.LD_ERR_INVALID


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
