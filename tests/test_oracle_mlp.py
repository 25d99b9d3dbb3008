"""Pins for oracle/mlp.py: parameter count, GELU values, finite-difference gradients, Adam."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_param_count_and_gelu():
    assert mlp.n_params() == 33793
    # GELU(x) = x Phi(x); Phi(1) = 0.8413447460685429 (standard normal CDF table value)
    assert float(mlp.gelu(np.array(1.0))) == pytest.approx(0.8413447460685429, rel=1e-14)
    assert float(mlp.gelu(np.array(0.0))) == 0.0
    x = np.linspace(-4, 4, 41)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), rtol=1e-7,
                               atol=1e-9)


def _setup(N=7, seed=0):
    rng = np.random.default_rng(seed)
    flat = rng.standard_normal(mlp.n_params()) * 0.1
    X = rng.standard_normal((N, 4))
    y = rng.standard_normal(N)
    return flat, X, y


def test_parameter_gradient_matches_fd():
    flat, X, y = _setup()
    _, g, _ = mlp.loss_and_grads(flat, X, y)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(mlp.n_params(), 40, replace=False), [0, 512, 640, 33792]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (mlp.loss_and_grads(flat + e, X, y)[0] - mlp.loss_and_grads(flat - e, X, y)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_input_gradient_matches_fd():
    flat, X, y = _setup()
    _, _, dX = mlp.loss_and_grads(flat, X, y)
    h = 1e-6
    for a in range(4):
        e = np.zeros_like(X)
        e[:, a] = h
        fd = (mlp.forward(flat, X + e)[0] - mlp.forward(flat, X - e)[0]) / (2 * h)
        np.testing.assert_allclose(dX[:, a], fd, rtol=1e-6, atol=1e-10)


def test_first_adam_step_is_lr_times_sign():
    # After one step, m_hat = g and v_hat = g^2, so the update is lr g / (|g| + eps).
    g = np.array([0.5, -2.0, 1e-3])
    p, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert math.isclose(m[0], 0.05) and math.isclose(v[1], 0.004)
