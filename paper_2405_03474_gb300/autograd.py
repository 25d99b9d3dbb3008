"""torch.autograd.Function over the C-ABI estimator.

``LogDet.apply(theta, X, kind, precond, probes, options)`` returns the estimate of
log det (K(X, X; l, v) + nu I) for theta = (l, v, nu) (a float64 tensor of 3) and
backpropagates the hand-written adjoint of ``logdet_grad``: with P and the probes
held fixed, d/dtheta = (1/s) sum_i sum_j (-c_j) y_ij^T (dM/dtheta) y_ij.  Both the
value and the gradient come from one call of the library (the shifted solves are
shared); backward only scales the saved gradient.
"""
import torch

from . import api


class LogDet(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, X, kind, precond, probes, options):
        th = [float(v) for v in theta.detach().cpu().tolist()]
        kern = api.Kernel(kind, th[0], th[1], th[2])
        res = api.logdet_grad(X, kern, precond=precond, probes=probes, **(options or {}))
        ctx.save_for_backward(torch.as_tensor(res["grad"], dtype=theta.dtype, device=theta.device))
        return torch.as_tensor(res["logdet"], dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None, None, None, None


def logdet(theta, X, kind, precond=None, probes=None, **options):
    """Differentiable log det estimate in theta = (lengthscale, variance, noise)."""
    return LogDet.apply(theta, X, kind, precond, probes, options)
