"""Gradient of the estimator (hand-written adjoint) at the gradient workload's scales:
parity with the oracle's frozen-P gradient and the exact FP64 gradient at n = 4096,
central finite differences of the FP64 estimate at n = 32768 and at the workload's
n = 131072, the reduced precisions against FP64 at n = 131072, and the
torch.autograd.Function."""
import numpy as np
import pytest

from gpu_util import cuda, host, torch
from oracle import gradient, kernels, precond
from oracle.splitmix import rademacher_block
from paper_2405_03474_gb300 import api, autograd, inputs

pytestmark = pytest.mark.gpu


def test_grad_n4096_matches_oracle_and_exact_gradient():
    n, s = 4096, 32
    th = (0.2, 1.0, 1e-2)
    X = inputs.points(n, 2, "uniform", seed=0)
    M = kernels.kernel_matrix(X, kernels.RBF, *th)
    A, D = precond.build(M, rademacher_block(2, n, 64), 2, th[2])
    Z = inputs.rademacher(n, s, seed=1)
    P = api.Precond.import_(A, D, "fp64")
    res = api.logdet_grad(cuda(X), api.Kernel(api.RBF, *th), precond=P, probes=cuda(Z), order=3,
                          num_probes=s, precision="fp64", rel_tol=1e-12, max_iters=3000)
    g_or = gradient.estimator_grad(X, kernels.RBF, *th, A, D, Z.astype(np.float64), 3)
    np.testing.assert_allclose(res["grad"], g_or, rtol=1e-8)
    g_exact = gradient.exact_grad(X, kernels.RBF, *th)
    # Hutchinson noise with 32 probes after a rank-64 preconditioner: a few percent
    np.testing.assert_allclose(res["grad"], g_exact, rtol=0.05)


def _fd_check(n, prec, th, h_rel, rtol, rank=128, s=16):
    th = np.array(th)
    Xt = cuda(inputs.points(n, 2, "uniform", seed=0))
    P = api.Precond.build(Xt, api.Kernel(api.RBF, *th), rank, power_iters=2, seed=2,
                          precision="fp64" if prec == "fp64" else "fp32")
    Zt = cuda(inputs.rademacher(n, s, seed=1))
    opts = dict(order=3, num_probes=s, precision=prec, rel_tol=1e-11 if prec == "fp64" else 1e-6,
                max_iters=3000)
    g = api.logdet_grad(Xt, api.Kernel(api.RBF, *th), precond=P, probes=Zt, **opts)["grad"]
    fd = []
    for a in range(3):
        e = np.zeros(3)
        e[a] = h_rel * th[a]
        fp = api.logdet_estimate(Xt, api.Kernel(api.RBF, *(th + e)), precond=P, probes=Zt, **opts)["logdet"]
        fm = api.logdet_estimate(Xt, api.Kernel(api.RBF, *(th - e)), precond=P, probes=Zt, **opts)["logdet"]
        fd.append((fp - fm) / (2 * e[a]))
    if rtol is not None:
        np.testing.assert_allclose(g, fd, rtol=rtol)
    return g


def test_grad_central_differences_fp64():
    # Differences of the converged fp64 estimate (P and probes frozen) against the adjoint.
    _fd_check(32768, "fp64", (0.2, 1.0, 1e-2), 1e-4, 1e-6)


def test_grad_central_differences_fp64_n131072():
    # The gradient workload's size (RBF, 2^17 points in [0,1]^2); theta = (0.2, 1, 0.1),
    # where FP64 CG converges in tens of steps; 8 probes, P and probes frozen.
    _fd_check(131072, "fp64", (0.2, 1.0, 0.1), 1e-4, 1e-5, rank=128, s=8)


def _grads_n131072(th, precs, s=8):
    import time
    n = 131072
    Xt = cuda(inputs.points(n, 2, "uniform", seed=0))
    Zt = cuda(inputs.rademacher(n, s, seed=1))
    P64 = api.Precond.build(Xt, api.Kernel(api.RBF, *th), 128, power_iters=2, seed=2, precision="fp64")
    A, D, _ = P64.export()
    P32 = api.Precond.import_(A, D, "fp32")
    out = {}
    for prec in precs:
        P, tol = (P64, 1e-10) if prec == "fp64" else (P32, 1e-6)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = api.logdet_grad(Xt, api.Kernel(api.RBF, *th), precond=P, probes=Zt, order=3, num_probes=s,
                            precision=prec, rel_tol=tol, max_iters=3000, residual_check=True)
        out[prec] = r
        print("grad n=%d theta=%s %s: %.2f s, %d iterations, grad %s, residual check %s"
              % (n, th, prec, time.perf_counter() - t0, r["iters"], r["grad"], r["max_resid"][:3]))
    return out


def test_grad_fp32_adjoint_matches_fp64_adjoint_n131072():
    # The gradient workload's size: n = 2^17 points in [0,1]^2.  The fp32 estimate is
    # too noisy for central differences at this size (its fp32 CG moves the value by
    # more than 2 h g), so the fp32 adjoint is held against the fp64 adjoint on the
    # same probes and preconditioner, whose differences are checked above.  At
    # lengthscale 0.2 a row of K sums to ~ n 2 pi l^2 = 3.3e4 while the noise is 1e-2:
    # fp32 rounding of the kernel values (~2^-24 each) moves the smallest eigenvalues
    # of M, which the shifted solutions x_ij weight most, by up to ~2e-3, and the
    # adjoint (which uses x_ij directly) inherits that; the log det is far less
    # sensitive.
    out = _grads_n131072((0.2, 1.0, 1e-2), ("fp64", "fp32"))
    np.testing.assert_allclose(out["fp32"]["grad"], out["fp64"]["grad"], rtol=2e-2)


def test_grad_tensor_core_adjoint_n131072():
    # The tensor-core derivative pass at the gradient workload's size, where the hi/lo
    # fp16 rounding of K (~2^-22 per entry) times the row sum of K (~3.3e4) stays well
    # below the noise: noise 0.1 (the top of the workload's noise range).  With noise
    # 1e-2 that perturbation reaches the noise level and the reduced-precision operator
    # stops being reliably positive definite (CG reports not converged).
    out = _grads_n131072((0.2, 1.0, 0.1), ("fp64", "fp32", "f16x3_tc"))
    np.testing.assert_allclose(out["fp32"]["grad"], out["fp64"]["grad"], rtol=2e-2)
    np.testing.assert_allclose(out["f16x3_tc"]["grad"], out["fp64"]["grad"], rtol=2e-2)


def test_autograd_function_backpropagates_the_adjoint():
    n, s = 1500, 8
    th = (0.3, 1.2, 5e-2)
    X = cuda(inputs.points(n, 2, "uniform", seed=3))
    P = api.Precond.build(X, api.Kernel(api.MATERN52, *th), 32, power_iters=2, seed=2, precision="fp64")
    Z = cuda(inputs.rademacher(n, s, seed=4))
    opts = dict(order=3, num_probes=s, precision="fp64", rel_tol=1e-12, max_iters=3000)
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    val = autograd.logdet(theta, X, api.MATERN52, precond=P, probes=Z, **opts)
    (3.0 * val).backward()
    ref = api.logdet_grad(X, api.Kernel(api.MATERN52, *th), precond=P, probes=Z, **opts)
    assert val.detach().item() == pytest.approx(ref["logdet"], rel=1e-14)
    np.testing.assert_allclose(theta.grad.numpy(), 3.0 * ref["grad"], rtol=1e-14)
    # and it agrees with a central difference of the forward value
    h = 1e-6
    for a in range(3):
        e = torch.zeros(3, dtype=torch.float64)
        e[a] = h * th[a]
        fp = float(autograd.logdet(theta.detach() + e, X, api.MATERN52, precond=P, probes=Z, **opts))
        fm = float(autograd.logdet(theta.detach() - e, X, api.MATERN52, precond=P, probes=Z, **opts))
        assert ref["grad"][a] == pytest.approx((fp - fm) / (2 * h * th[a]), rel=1e-6)


@pytest.mark.parametrize("prec", ["f16x3_tc", "fp32"])
def test_grad_reduced_precision_n4096_against_oracle(prec):
    # the same case as the FP64 test above, in FP32 SIMT and on the tensor cores (hi/lo
    # fp16 derivative pass); the printed residual check is the true relative residual
    # of the shifted solutions the adjoint uses
    n, s = 4096, 32
    th = (0.2, 1.0, 1e-2)
    X = inputs.points(n, 2, "uniform", seed=0)
    M = kernels.kernel_matrix(X, kernels.RBF, *th)
    A, D = precond.build(M, rademacher_block(2, n, 64), 2, th[2])
    Z = inputs.rademacher(n, s, seed=1)
    P = api.Precond.import_(A, D, "fp32")
    res = api.logdet_grad(cuda(X), api.Kernel(api.RBF, *th), precond=P, probes=cuda(Z), order=3,
                          num_probes=s, precision=prec, rel_tol=1e-6, max_iters=3000, residual_check=True)
    g_or = gradient.estimator_grad(X, kernels.RBF, *th, A, D, Z.astype(np.float64), 3)
    rel = np.abs(res["grad"] / g_or - 1)
    print("grad %s n=%d: rel err vs oracle %s, true residuals %s, iters %d"
          % (prec, n, rel, res["max_resid"][:3], res["iters"]))
    np.testing.assert_allclose(res["grad"], g_or, rtol=3e-4)
