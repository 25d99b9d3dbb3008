"""FP64 reference for the surrogate MLP (forward, backward, Adam).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The surrogate maps hyperparameters (log lengthscale, log variance, log noise,
log n) to a standardised log det.  Architecture: 4 -> 128 -> 128 -> 128 -> 1,
GELU after each hidden layer (exact form x * Phi(x), Phi the standard normal
CDF), mean-squared-error loss, Adam (Kingma & Ba 2015) updates.  Weights are
stored as W_l with shape (out, in) and biases b_l with shape (out,).
"""
import numpy as np
from scipy.special import erf

SIZES = (4, 128, 128, 128, 1)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    phi = np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * phi


def n_params(sizes=SIZES):
    return sum(o * i + o for i, o in zip(sizes[:-1], sizes[1:]))


def unflatten(flat, sizes=SIZES):
    """Flat parameter vector -> list of (W, b); layout W_1, b_1, W_2, b_2, ..."""
    flat = np.asarray(flat, dtype=np.float64)
    out, off = [], 0
    for i, o in zip(sizes[:-1], sizes[1:]):
        W = flat[off:off + o * i].reshape(o, i)
        off += o * i
        b = flat[off:off + o]
        off += o
        out.append((W, b))
    return out


def forward(flat, X):
    """Returns y (N,) and the per-layer pre-activations (for backward)."""
    layers = unflatten(flat)
    h = np.asarray(X, dtype=np.float64)
    cache = [h]
    for li, (W, b) in enumerate(layers):
        z = h @ W.T + b
        cache.append(z)
        h = gelu(z) if li + 1 < len(layers) else z
    return h[:, 0], cache


def loss_and_grads(flat, X, y):
    """MSE loss, its gradient w.r.t. the flat parameters, and d pred / d X."""
    layers = unflatten(flat)
    pred, cache = forward(flat, X)
    N = pred.shape[0]
    loss = float(np.mean((pred - y) ** 2))
    dz = (2.0 / N) * (pred - y)[:, None]
    din = np.ones((N, 1))  # for d pred / d X
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        zin = cache[li]
        hin = gelu(zin) if li > 0 else zin
        grads.append((dz.T @ hin, dz.sum(axis=0)))
        dh = dz @ W
        dinh = din @ W
        if li > 0:
            gp = gelu_grad(zin)
            dz = dh * gp
            din = dinh * gp
        else:
            dX = dinh
    grads.reverse()
    flat_g = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat_g, dX


def adam_step(flat, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (flat, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return flat - lr * mhat / (np.sqrt(vhat) + eps), m, v
