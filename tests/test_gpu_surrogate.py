"""The surrogate MLP's CUDA kernels against the FP64 oracle MLP (oracle/mlp.py)."""
import numpy as np
import pytest

from gpu_util import assert_elementwise, cuda, host, torch
from oracle import mlp
from paper_2405_03474_gb300 import api

pytestmark = pytest.mark.gpu


def _data(N, seed):
    rng = np.random.default_rng(seed)
    flat = (rng.standard_normal(mlp.n_params()) * 0.1).astype(np.float32)
    X = rng.standard_normal((N, 4)).astype(np.float32)
    y = rng.standard_normal(N).astype(np.float32)
    return flat, X, y


def test_loss_and_parameter_gradient_match_oracle():
    flat, X, y = _data(300, 0)
    S = api.Surrogate(seed=1)
    S.set_params(flat)
    loss, g = S.loss_grad(cuda(X), cuda(y))
    lo, go, _ = mlp.loss_and_grads(flat.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    assert loss == pytest.approx(lo, rel=1e-5)
    # fp32 sums over the batch: each entry within 1e-5 of the largest gradient entry
    assert_elementwise(g, go, np.full(go.shape, np.abs(go).max()), 1e-5, "parameter gradient")


def test_inference_and_input_gradient_match_oracle():
    flat, X, _ = _data(1000, 2)
    S = api.Surrogate(seed=1)
    S.set_params(flat)
    out, dout = S.infer(cuda(X), want_grad=True)
    ref, _ = mlp.forward(flat.astype(np.float64), X.astype(np.float64))
    _, _, dX = mlp.loss_and_grads(flat.astype(np.float64), X.astype(np.float64), np.zeros(1000))
    assert_elementwise(host(out), ref, np.full(ref.shape, np.abs(ref).max()), 1e-5, "network output")
    assert_elementwise(host(dout), dX, np.full(dX.shape, np.abs(dX).max()), 1e-5, "input gradient")


def test_adam_steps_match_oracle():
    # one epoch of full-batch Adam steps on normalised data, against the oracle's Adam
    flat, X, y = _data(256, 3)
    S = api.Surrogate(seed=1)
    S.set_params(flat)
    S.train(cuda(X), cuda(y), epochs=3, batch=256, lr=1e-3)
    Xn = (X.astype(np.float64) - X.mean(0)) / X.std(0)
    yn = (y.astype(np.float64) - y.mean()) / y.std()
    p = flat.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for step in range(1, 4):
        _, g, _ = mlp.loss_and_grads(p, Xn, yn)
        p, m, v = mlp.adam_step(p, g, m, v, step, 1e-3)
    np.testing.assert_allclose(S.get_params(), p, rtol=1e-4, atol=1e-6)


def test_training_fits_a_smooth_function():
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (2048, 4)).astype(np.float32)
    y = (np.sin(X[:, 0]) + X[:, 1] * X[:, 2] - 0.5 * X[:, 3] ** 2).astype(np.float32)
    S = api.Surrogate(seed=5)
    loss = S.train(cuda(X), cuda(y), epochs=300, batch=256, lr=3e-3)
    assert loss < 1e-3  # normalised MSE
    Xt = rng.uniform(-1, 1, (512, 4)).astype(np.float32)
    yt = np.sin(Xt[:, 0]) + Xt[:, 1] * Xt[:, 2] - 0.5 * Xt[:, 3] ** 2
    assert np.abs(host(S.infer(cuda(Xt))) - yt).max() < 0.1


def test_surrogate_gain_over_the_estimator():
    # Train on estimator labels at n = 2048 (Matern-5/2, d = 3) over the hyperparameter box,
    # then measure what the network gains: accuracy against fresh estimator values on
    # held-out hyperparameters, and time per query against running the estimator.
    import time
    from paper_2405_03474_gb300 import inputs, surrogate
    n = 2048
    X = cuda(inputs.points(n, 3, "uniform", seed=0))
    est = surrogate.Estimator(X, api.MATERN52, rank=32, power_iters=1, probes=16, t=20)
    thetas = inputs.sobol_theta(256, seed=0)
    labels = surrogate.generate_labels(est, thetas)
    hs = surrogate.HyperSurrogate(est, seed=3)
    hs.fit(thetas, labels, epochs=600, batch=64, lr=2e-3)
    test = inputs.sobol_theta(48, seed=11)
    t0 = time.perf_counter()
    ref = np.array([est(t) for t in test])
    t_est = (time.perf_counter() - t0) / len(test)
    many = inputs.sobol_theta(4096, seed=12)
    hs.predict(many)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs.predict(many)
    t_sur = (time.perf_counter() - t0) / len(many)
    pred, outside = hs.predict(test)
    assert not outside.any()
    err = np.abs(pred - ref)
    spread = labels.max() - labels.min()
    print("surrogate: max abs err %.4g (label spread %.3g), %.3g s/query vs estimator %.3g s/query"
          % (err.max(), spread, t_sur, t_est))
    assert err.max() < 0.01 * spread
    assert t_est / t_sur > 100
    # outside the box the estimator answers
    far = np.array([[3.0, 1.0, 0.05]])
    p, out = hs.predict(far)
    # (the symmetric kernel product adds the blocks of different CTAs in arrival order,
    # so two estimates of one theta agree to fp32 rounding of the sums, not bit for bit)
    assert out[0] and p[0] == pytest.approx(est(far[0]), rel=1e-6)


def test_checkpoint_round_trip(tmp_path):
    # a trained network saved (parameters + normalisation) and restored into a fresh handle
    # predicts bit for bit what the original predicts
    rng = np.random.default_rng(4)
    theta = rng.uniform(-1, 1, size=(512, 4)).astype(np.float32)
    y = (np.sin(theta[:, 0]) + theta[:, 1] * theta[:, 2] + 3.0).astype(np.float32)
    net = api.Surrogate(seed=5)
    net.train(cuda(theta), cuda(y), epochs=20, batch=64, lr=2e-3)
    q = cuda(rng.uniform(-1, 1, size=(300, 4)).astype(np.float32))
    ref = host(net.infer(q))
    path = str(tmp_path / "surrogate.npz")
    net.save(path)
    other = api.Surrogate(seed=99)
    other.load(path)
    np.testing.assert_array_equal(host(other.infer(q)), ref)
    np.testing.assert_array_equal(other.get_norm(), net.get_norm())
