"""Pins of the FP64 cost-model oracle (oracle/mlp.py) against things other than
itself: central finite differences, the linear regime where the network
collapses to one affine map, Adam's closed-form first step, dead units, and
a batch the network already fits."""
import numpy as np
import pytest

from oracle import mlp
from paper_1011_4046_gb300 import inputs


def _rand(seed, *shape, scale=1.0):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(shape)


def test_parameter_count_and_layout():
    assert mlp.N_PARAMS == 5313 == inputs.MLP_PARAMS
    theta = np.arange(mlp.N_PARAMS, dtype=np.float64)
    p = mlp.unpack(theta)
    assert p["W1"][1, 0] == 16 and p["b1"][0] == 1024 and p["W2"][0, 1] == 1089
    assert p["b3"][0] == mlp.N_PARAMS - 1
    assert np.array_equal(mlp.pack(p), theta)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_central_differences(seed):
    theta = inputs.mlp_init(seed).astype(np.float64) + _rand(seed + 10, mlp.N_PARAMS, scale=0.05)
    X = _rand(seed + 20, 9, 16)
    y = _rand(seed + 30, 9)
    _, g = mlp.loss_and_grad(theta, X, y)
    rng = np.random.default_rng(seed)
    idx = np.concatenate([rng.choice(1024, 40, replace=False), 1024 + rng.choice(64, 10, replace=False),
                          1088 + rng.choice(4096, 60, replace=False), 5184 + rng.choice(64, 10, replace=False),
                          5248 + rng.choice(64, 20, replace=False), [5312]])
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (mlp.loss_and_grad(tp, X, y)[0] - mlp.loss_and_grad(tm, X, y)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_linear_regime_is_one_affine_map():
    """With positive inputs, weights and biases every unit is active, so the
    network is the affine map x -> (W3 W2 W1) x + (W3 W2 b1 + W3 b2 + b3), and
    the gradient of W3 is the mean residual-weighted hidden activation."""
    rng = np.random.default_rng(5)
    p = {"W1": rng.uniform(0.1, 0.5, (64, 16)), "b1": rng.uniform(0.1, 0.2, 64),
         "W2": rng.uniform(0.0, 0.1, (64, 64)), "b2": rng.uniform(0.1, 0.2, 64),
         "W3": rng.uniform(-1, 1, 64), "b3": np.array([0.3])}
    theta = mlp.pack(p)
    X = rng.uniform(0.0, 1.0, (7, 16))
    M = np.linalg.multi_dot([p["W3"][None, :], p["W2"], p["W1"]])[0]
    c = p["W3"] @ (p["W2"] @ p["b1"]) + p["W3"] @ p["b2"] + p["b3"][0]
    yhat, _ = mlp.forward(theta, X)
    assert np.allclose(yhat, X @ M + c, rtol=1e-13, atol=1e-13)
    y = rng.uniform(-1, 1, 7)
    _, g = mlp.loss_and_grad(theta, X, y)
    r = (X @ M + c) - y
    # d/db3 of mean r^2 is 2 mean(r); d/dW1 = 2 mean(r x) outer (W3 W2)
    assert np.isclose(g[-1], 2 * r.mean(), rtol=1e-12)
    gW1 = np.outer(p["W3"] @ p["W2"], 2 * (r[:, None] * X).mean(axis=0))
    assert np.allclose(g[:1024].reshape(64, 16), gW1, rtol=1e-11, atol=1e-13)


def test_dead_units_pass_no_gradient():
    """Units whose pre-activation is negative for every sample get zero
    gradient on their incoming weights and biases."""
    theta = inputs.mlp_init(7).astype(np.float64)
    p = mlp.unpack(theta)
    p["b1"][:8] = -1e3  # first 8 first-layer units dead
    p["b2"][-4:] = -1e3  # last 4 second-layer units dead
    theta = mlp.pack(p)
    X = _rand(8, 11, 16)
    _, g = mlp.loss_and_grad(theta, X, _rand(9, 11))
    gp = mlp.unpack(g)
    assert np.all(gp["W1"][:8] == 0) and np.all(gp["b1"][:8] == 0)
    assert np.all(gp["W2"][-4:] == 0) and np.all(gp["b2"][-4:] == 0) and np.all(gp["W3"][-4:] == 0)
    assert np.all(gp["W2"][:, :8] == 0)


def test_zero_residual_gives_zero_loss_and_gradient():
    theta = inputs.mlp_init(4).astype(np.float64)
    X = _rand(1, 5, 16)
    yhat, _ = mlp.forward(theta, X)
    loss, g = mlp.loss_and_grad(theta, X, yhat)
    assert loss == 0.0 and np.all(g == 0)


def test_adam_first_step_is_lr_times_sign():
    """From m = v = 0 the bias-corrected first step is g / (|g| + eps): each
    parameter with |g| >> eps moves by exactly lr against its gradient."""
    theta = np.zeros(6)
    g = np.array([3.0, -2.0, 1e-3, -5e-2, 0.0, 7.0])
    t1, m, v = mlp.adam_step(theta, g, np.zeros(6), np.zeros(6), 1, lr=0.01)
    expect = -0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(t1, expect, rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # second step with the same gradient: still lr per parameter (m-hat = g, v-hat = g^2)
    t2, _, _ = mlp.adam_step(t1, g, m, v, 2, lr=0.01)
    assert np.allclose(t2 - t1, expect, rtol=1e-9, atol=1e-15)


def test_training_fits_an_affine_target():
    """A learnable target (an affine function of the features) is fitted:
    the loss falls by two orders of magnitude in 40 epochs."""
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, (256, 16))
    y = X @ rng.uniform(-1, 1, 16) + 0.5
    theta = inputs.mlp_init(11)
    order = inputs.epoch_orders(11, len(y), 40)
    theta1, losses = mlp.train(theta, X, y, order, batch=32, lr=3e-3)
    first = float(np.mean(losses[:8]))
    last = float(np.mean(losses[-8:]))
    assert last < 1e-2 * first, (first, last)
