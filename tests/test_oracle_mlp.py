"""Pins of the rank-predictor oracle (numpy MLP) against facts that do not
come from the oracle itself: central finite differences of the loss, a
network built by hand to compute a known function, the closed form of the
first Adam step, and loss descent on a learnable target."""
import numpy as np
import pytest

from oracle import mlp
from paper_1811_11248_gb300 import inputs


def rand_theta(seed, scale=0.5):
    return np.random.default_rng(seed).standard_normal(mlp.NPARAM) * scale


def test_layout_size():
    assert mlp.NPARAM == 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1 == 4801
    th = np.arange(mlp.NPARAM, dtype=float)
    assert np.array_equal(mlp.pack(mlp.unpack(th)), th)
    assert mlp.unpack(th)["W1"][1, 0] == 8.0  # row-major (out x in)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    th = rand_theta(seed)
    X = rng.standard_normal((7, 8))
    t = rng.standard_normal(7)
    _, g = mlp.loss_and_grad(th, X, t)
    h = 1e-6
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    # every parameter group is probed
    idx = np.concatenate([idx, [0, 511, 512, 600, 576 + 4095, 4736, 4799, 4800]])
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        lp, _ = mlp.loss_and_grad(th + e, X, t)
        lm, _ = mlp.loss_and_grad(th - e, X, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_hand_built_network_computes_abs():
    """h1 = relu(+x0), relu(-x0); h2 copies them; y = h2_0 + h2_1 = |x0| + 0.25."""
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    p["W1"][0, 0], p["W1"][1, 0] = 1.0, -1.0
    p["W2"][0, 0], p["W2"][1, 1] = 1.0, 1.0
    p["w3"][0], p["w3"][1] = 1.0, 1.0
    p["b3"][0] = 0.25
    X = np.random.default_rng(3).standard_normal((20, 8))
    y, _ = mlp.forward(mlp.pack(p), X)
    np.testing.assert_allclose(y, np.abs(X[:, 0]) + 0.25, rtol=0, atol=1e-15)


def test_zero_network_gradient_is_bias_only():
    """All weights zero: y = b3, so only b3 has a gradient, 2 mean(b3 - t)."""
    th = np.zeros(mlp.NPARAM)
    th[-1] = 0.5
    X = np.ones((4, 8))
    t = np.array([0.0, 1.0, 2.0, 3.0])
    L, g = mlp.loss_and_grad(th, X, t)
    assert L == pytest.approx(np.mean((0.5 - t) ** 2))
    assert g[-1] == pytest.approx(2.0 * np.mean(0.5 - t))
    assert not g[:-1].any()


def test_first_adam_step_closed_form():
    """Step 1: m_hat = g and v_hat = g^2, so theta moves by lr * g / (|g| + eps)."""
    th = rand_theta(4)
    g = np.random.default_rng(5).standard_normal(mlp.NPARAM)
    z = np.zeros(mlp.NPARAM)
    th1, m, v = mlp.adam_step(th, g, z, z, 1, 1e-3)
    np.testing.assert_allclose(th1, th - 1e-3 * g / (np.abs(g) + mlp.ADAM_EPS), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_training_fits_a_learnable_target():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((512, 8))
    t = np.maximum(X[:, 0], 0.0) + 0.5 * X[:, 1] - 0.2 * X[:, 2] * (X[:, 3] > 0)
    th0 = inputs.mlp_init_params(0)
    L0, _ = mlp.loss_and_grad(th0, X, t)
    order = inputs.mlp_batch_order(512, 64, 30, seed=1)
    th, losses = mlp.train_steps(th0, X, t, order, 64, 3e-3)
    L1, _ = mlp.loss_and_grad(th, X, t)
    assert L1 < 0.05 * L0, (L0, L1)
