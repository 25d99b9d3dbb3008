"""The C-ABI library loads and exports every function include/logdet.h declares
(no GPU needed: only dlopen and symbol lookup)."""
import ctypes
import os

import pytest

from paper_2405_03474_gb300 import _lib


def test_header_declares_the_boundary():
    names = _lib.header_functions()
    for must in ("logdet_estimate", "logdet_grad", "precond_build", "ld_kz", "surrogate_train"):
        assert must in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2405_03474_gb300 import build
        build.build()
    lib = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in _lib.header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    lib = _lib.load()
    assert lib.ld_status_string(0) == b"ok"
    assert lib.ld_status_string(-3) == b"not converged"
    assert lib.ld_version() >= 1


def test_coefficients_from_library_match_table1_without_gpu():
    # ld_rk_coeffs is host code: it runs without a device.
    from paper_2405_03474_gb300 import api
    import numpy as np
    b, c, s = api.rk_coeffs(3)
    assert b == pytest.approx(14 / 3)
    np.testing.assert_allclose(s, [0.0717967697244908, 1.0, 13.92820323027551], rtol=1e-14)
    np.testing.assert_allclose(-c, [0.2552774034648563, 20 / 9, 49.52250037431294], rtol=1e-13)
