"""Rank predictor oracle (test infrastructure only): plain numpy, FP64.

A three-layer perceptron of width 64 maps the features of one scaled block
(Sec. 3.1: the block row G^-1 [A_sn A_sw] that the compression step of
Algorithm 1 factors) to the fraction r / s of its numerical rank.  Nothing in
the paper fixes the network; this module is the reference its CUDA
forward / backward / Adam kernels are checked against.

Parameter vector (float, NPARAM entries, the layout both sides use):
  W1 (64 x 8, row-major), b1 (64), W2 (64 x 64, row-major), b2 (64),
  w3 (64), b3 (1).
Network:  h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = w3 . h2 + b3.
Loss over a batch of B samples:  L = (1/B) sum_b (y_b - t_b)^2.
ReLU'(0) is taken as 0.
Adam (Kingma and Ba, 2015): m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
theta <- theta - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

NIN, NH = 8, 64
SHAPES = (("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)), ("b3", (1,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)
BETA1, BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


def unpack(theta):
    """Flat parameter vector -> dict of views (the layout above)."""
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(theta, X):
    """X: B x 8 -> (y (B), cache) with the hidden activations."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (X, a1, h1, a2, h2)


def loss_and_grad(theta, X, t):
    """Mean squared error and its gradient (backpropagation, layer by layer)."""
    p = unpack(theta)
    y, (X, a1, h1, a2, h2) = forward(theta, X)
    B = X.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    L = float(np.mean(r * r))
    gy = 2.0 * r / B                      # dL/dy
    g = {}
    g["w3"] = h2.T @ gy
    g["b3"] = np.array([gy.sum()])
    ga2 = np.outer(gy, p["w3"]) * (a2 > 0.0)
    g["W2"] = ga2.T @ h1
    g["b2"] = ga2.sum(axis=0)
    ga1 = (ga2 @ p["W2"]) * (a1 > 0.0)
    g["W1"] = ga1.T @ X
    g["b1"] = ga1.sum(axis=0)
    return L, pack(g)


def adam_step(theta, grad, m, v, step, lr):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = BETA1 * m + (1.0 - BETA1) * grad
    v = BETA2 * v + (1.0 - BETA2) * grad * grad
    mh = m / (1.0 - BETA1 ** step)
    vh = v / (1.0 - BETA2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def train_steps(theta, X, t, order, batch, lr):
    """Minibatch Adam: step k uses samples order[k*batch:(k+1)*batch] (the
    order array is an input, so both implementations see the same batches).
    Returns (theta, per-step losses before each update)."""
    order = np.asarray(order).reshape(-1, batch)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    losses = []
    for step, idx in enumerate(order, start=1):
        L, g = loss_and_grad(theta, X[idx], t[idx])
        theta, m, v = adam_step(theta, g, m, v, step, lr)
        losses.append(L)
    return theta, np.array(losses)
