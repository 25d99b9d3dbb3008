"""Algorithm 1 at n = 2^15, matrix-free, against the value the CPU FP64 oracle stored.

The stored case (tests/golden/estimate_matern_n32768_d4.txt, written by
tests/golden/make_estimate_matern_n32768_d4.py from oracle/ only) is the literal
Algorithm 1 of Section 2: t = 20 Lanczos steps per probe, Thomas per shift of r_3,
the Hutchinson mean over 16 Rademacher probes, on Matern-5/2 points in [0,1]^4
(lengthscale 0.1, noise 1e-2) with a rank-128 randomized-SVD preconditioner that
the oracle builds matrix-free.  This test rebuilds that preconditioner with the
same oracle code (its log det P must reproduce the stored value), imports it on
the device, runs the estimator with the same probes and t, and compares: FP64
within 1e-10 (per-probe brackets and SLQ as well), FP32 and the hi/lo fp16
tensor-core product within 1e-4.
"""
import importlib.util
import os

import numpy as np
import pytest

from gpu_util import cuda, torch
from paper_2405_03474_gb300 import api

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden_module():
    path = os.path.join(HERE, "golden", "make_estimate_matern_n32768_d4.py")
    spec = importlib.util.spec_from_file_location("make_estimate_matern_n32768_d4", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def case():
    g = _golden_module()
    stored = g.read()
    X, Z, A, D, F, _ = g.problem()
    # the rebuilt preconditioner is the stored one
    assert F["logdet_P"] == pytest.approx(stored["logdet_P"], rel=1e-12)
    return g.CONFIG, stored, X, Z, A, D


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4), ("f16x3_tc", 1e-4)])
def test_estimate_matches_stored_oracle_algorithm1(case, prec, tol):
    cfg, stored, X, Z, A, D = case
    P = api.Precond.import_(A, D, "fp64" if prec == "fp64" else "fp32")
    kern = api.Kernel(cfg["kind"], cfg["lengthscale"], cfg["variance"], cfg["noise"])
    res = api.logdet_estimate(cuda(X), kern, precond=P, probes=cuda(Z.astype(np.int8)), order=cfg["order"],
                              num_probes=cfg["probes"], precision=prec, fixed_iters=cfg["t"], max_iters=cfg["t"])
    print("n=%d %s: log det %.12f, oracle %.12f, rel %.2e; SLQ %.12f, oracle %.12f"
          % (cfg["n"], prec, res["logdet"], stored["estimate"], abs(res["logdet"] / stored["estimate"] - 1),
             res["slq_logdet"], stored["slq"]))
    assert res["iters"] == cfg["t"]
    assert res["logdet_P"] == pytest.approx(stored["logdet_P"], rel=1e-12 if prec == "fp64" else 1e-5)
    assert res["logdet"] == pytest.approx(stored["estimate"], rel=tol)
    assert res["slq_logdet"] == pytest.approx(stored["slq"], rel=tol)
    if prec == "fp64":
        np.testing.assert_allclose(res["per_probe"], stored["bracket"], rtol=1e-9)
