"""FP64 oracle of the region cost model (test infrastructure only).

Only the tests may import this module; the product library never calls it and
shares no code with it.

The paper's manager hands out regions so that the expensive ones are not
left for last (Sec. 4, and the uneven region costs of the matter-era runs,
Sec. 6); here a small network predicts a region's cost from 16 features so
that the device queue can issue predicted-expensive regions first.  The
network and its training are plain definitions, written out:

* network: x (16) -> h1 = relu(W1 x + b1) (64) -> h2 = relu(W2 h1 + b2) (64)
  -> yhat = W3 h2 + b3 (1);
* loss of a minibatch: L = mean over its samples of (yhat - y)^2, y being the
  log of the measured region time;
* gradient: reverse-mode differentiation of L (relu'(z) = 1 for z > 0, else 0);
* Adam (Kingma & Ba 2015): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
  theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
* training: epochs of minibatches in a given order (the permutation is an
  input), one Adam step per minibatch.

Parameter vector (flat): W1 [64][16] row-major (output index first), b1 [64],
W2 [64][64], b2 [64], W3 [64], b3 [1]: 5313 numbers.

Pins: ``tests/test_mlp_oracle.py`` (finite differences, the linear regime,
Adam's first step, dead units, a zero-residual batch).
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 16, 64
SIZES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("W3", (N_HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (N_PARAMS,)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def forward(theta, X):
    """Predictions for the rows of X (n x 16) and the intermediate values."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    yhat = h2 @ p["W3"] + p["b3"][0]
    return yhat, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, y):
    """Mean squared error of a minibatch and its gradient (flat, like theta)."""
    p = unpack(theta)
    yhat, (X, z1, h1, z2, h2) = forward(theta, X)
    n = X.shape[0]
    r = yhat - np.asarray(y, dtype=np.float64)
    loss = float(np.mean(r * r))
    g_out = 2.0 * r / n                       # dL/dyhat per sample
    g = {"W3": h2.T @ g_out, "b3": np.array([g_out.sum()])}
    g_h2 = np.outer(g_out, p["W3"])
    g_z2 = g_h2 * (z2 > 0.0)
    g["W2"] = g_z2.T @ h1
    g["b2"] = g_z2.sum(axis=0)
    g_h1 = g_z2 @ p["W2"]
    g_z1 = g_h1 * (z1 > 0.0)
    g["W1"] = g_z1.T @ X
    g["b1"] = g_z1.sum(axis=0)
    return loss, pack(g)


def adam_step(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def train(theta, X, y, order, batch, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam over the minibatches given by ``order`` (concatenated epoch
    permutations of the sample indices, cut into consecutive groups of
    ``batch``; a short last group of an epoch is its own minibatch).
    ``order`` is a list of index arrays, one per epoch.  Returns
    (theta, losses of every minibatch before its step)."""
    theta = np.asarray(theta, dtype=np.float64).copy()
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    t = 0
    losses = []
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    for perm in order:
        for s in range(0, len(perm), batch):
            idx = perm[s:s + batch]
            loss, g = loss_and_grad(theta, X[idx], y[idx])
            t += 1
            theta, m, v = adam_step(theta, g, m, v, t, lr, beta1, beta2, eps)
            losses.append(loss)
    return theta, losses
