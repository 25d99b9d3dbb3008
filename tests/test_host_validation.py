"""Host-side logic of the C ABI, run without a GPU: argument checks that return a
status before any device work, and the host-computed r_k coefficients against
the oracle.  (Fake device pointers below are never dereferenced: every call
returns at its argument check.)"""
import ctypes

import numpy as np
import pytest

from oracle import coeffs
from paper_2405_03474_gb300 import _lib, api

FAKE = ctypes.c_void_p(0x1000)  # non-NULL, never touched


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


@pytest.mark.parametrize("k", [1, 3, 5])
def test_rk_coefficients_match_oracle(lib, k):
    b = ctypes.c_double()
    c = (ctypes.c_double * k)()
    sigma = (ctypes.c_double * k)()
    assert lib.ld_rk_coeffs(k, ctypes.byref(b), c, sigma) == _lib.LD_OK
    b0, c0, s0 = coeffs.rk_coeffs(k)
    assert b.value == pytest.approx(b0, rel=1e-14)
    np.testing.assert_allclose(np.array(c[:]), c0, rtol=1e-13)
    np.testing.assert_allclose(np.array(sigma[:]), s0, rtol=1e-13)
    assert lib.ld_rk_coeffs(2, ctypes.byref(b), c, sigma) == _lib.LD_ERR_INVALID


def test_kernel_product_argument_checks(lib):
    kern = api.Kernel(api.RBF, 0.3).c()
    fp32 = api.PRECISIONS["fp32"]
    for n, d, c, prec in ((0, 2, 4, fp32), (10, 2, 0, fp32), (10, 0, 4, fp32), (10, 33, 4, fp32),
                          (10, 9, 4, api.PRECISIONS["f16x3_tc"]), (10, 2, 4097, fp32), (10, 2, 4, 9)):
        st = lib.ld_kz(FAKE, n, d, kern, FAKE, ctypes.c_void_p(0x2000), c, prec, None, 0, None)
        assert st == _lib.LD_ERR_INVALID, (n, d, c, prec)
    assert b"ld_kz" in lib.ld_last_error()
    # W aliasing V
    assert lib.ld_kz(FAKE, 10, 2, kern, FAKE, FAKE, 4, fp32, None, 0, None) == _lib.LD_ERR_INVALID
    bad = api.Kernel(api.RBF, -0.3).c()
    assert lib.ld_kz(FAKE, 10, 2, bad, FAKE, ctypes.c_void_p(0x2000), 4, fp32, None, 0, None) == _lib.LD_ERR_INVALID


def test_static_product_rejects_sizes_beyond_its_array(lib):
    cap = lib.ld_kz_static_capacity()
    assert cap == 32 << 20
    kern = api.Kernel(api.MATERN52, 0.3).c()
    st = lib.ld_kz_static(FAKE, 1 << 22, 4, kern, FAKE, ctypes.c_void_p(0x2000), 16, api.PRECISIONS["f16x3_tc"],
                          None)
    assert st == _lib.LD_ERR_WORKSPACE and b"static" in lib.ld_last_error()


def test_estimator_option_checks(lib):
    kern = api.Kernel(api.MATERN52, 0.3, 1.0, 1e-2).c()
    res = _lib.LdResult()
    good = dict(order=3, num_probes=16, precision="fp32")
    cases = [dict(good, order=4), dict(good, num_probes=12, probes_per_block=8), dict(good, max_iters=0),
             dict(good, probes_per_block=300, num_probes=300), dict(good, precision="f16x3_tc"),  # d = 9 below
             dict(good, probe_kind=3), dict(good, probe_kind="orthogonal", num_probes=64, probes_per_block=64)]
    for i, kw in enumerate(cases):
        o = api.make_options(**kw)
        d = 9 if i == 4 else 2
        n = 32 if i == 6 else 1000  # orthogonal probes need probes_per_block <= n
        st = lib.logdet_estimate(FAKE, n, d, kern, None, ctypes.byref(o), None, None, None, 0, None, ctypes.byref(res))
        assert st == _lib.LD_ERR_INVALID, kw


def test_preconditioner_import_checks(lib):
    n, r = 6, 2
    A = np.ones((n, r))
    handle = ctypes.c_void_p()
    for D in (np.array([1, 1, 0, 1, 1, 1.0]), np.array([1, 1, -2, 1, 1, 1.0]), np.array([1, 1, np.nan, 1, 1, 1.0])):
        st = lib.precond_import(A.ctypes.data_as(ctypes.c_void_p), D.ctypes.data_as(ctypes.c_void_p), n, r,
                                api.PRECISIONS["fp64"], None, ctypes.byref(handle))
        assert st == _lib.LD_ERR_INVALID
    st = lib.precond_import(A.ctypes.data_as(ctypes.c_void_p), np.ones(n).ctypes.data_as(ctypes.c_void_p), n, n + 1,
                            api.PRECISIONS["fp64"], None, ctypes.byref(handle))
    assert st == _lib.LD_ERR_INVALID


def test_profile_kernel_id_check(lib):
    ms, nl, pairs, flops = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    for bad in (-1, 6):
        assert lib.ld_profile_kernel(bad, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(pairs),
                                     ctypes.byref(flops)) == _lib.LD_ERR_INVALID
    for good in (1, 5):  # the symmetric product, the tensor-core derivative pass
        assert lib.ld_profile_kernel(good, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(pairs),
                                     ctypes.byref(flops)) == _lib.LD_OK


def test_dense_product_argument_checks(lib):
    W = ctypes.c_void_p(0x2000)
    f16x3 = api.PRECISIONS["f16x3_tc"]
    for n, c, prec in ((0, 4, f16x3), (10, 0, f16x3), (10, 4, 9), (10, 4, -1), (10, 4097, f16x3)):
        assert lib.ld_dense_kz(FAKE, n, FAKE, W, c, prec, None) == _lib.LD_ERR_INVALID, (n, c, prec)
    assert b"ld_dense_kz" in lib.ld_last_error()
    assert lib.ld_dense_kz(FAKE, 10, FAKE, FAKE, 4, f16x3, None) == _lib.LD_ERR_INVALID  # W aliasing V


def test_dense_binding_checks_dtypes_and_shapes():
    torch = pytest.importorskip("torch")
    M32, V32 = torch.zeros(6, 6), torch.zeros(6, 2)
    with pytest.raises(ValueError, match="M must be"):
        api.ld_dense_kz(M32.double(), V32, "f16x3_tc")
    with pytest.raises(ValueError, match="M must be"):
        api.ld_dense_kz(torch.zeros(6, 5), V32, "fp32")
    with pytest.raises(ValueError, match="V must be"):
        api.ld_dense_kz(M32, torch.zeros(5, 2), "fp32")
    with pytest.raises(ValueError, match="V must be"):
        api.ld_dense_kz(M32.double(), V32, "fp64")
    with pytest.raises(ValueError, match="CUDA"):  # well-formed, but host tensors
        api.ld_dense_kz(M32, V32, "bf16_tc")
