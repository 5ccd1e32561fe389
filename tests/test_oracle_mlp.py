"""Pins of the reference MLP: gradient by central finite differences, a network whose
answer is known in closed form, and the Adam step written out."""
import numpy as np

from oracle import mlp


def test_param_count():
    assert mlp.N_PARAMS == 5378


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(1) * 0.5 + 0.01 * rng.standard_normal(mlp.N_PARAMS)
    X = rng.standard_normal((7, 16))
    Y = rng.standard_normal((7, 2))
    L, g = mlp.loss_grad(theta, X, Y)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss(theta + e, X, Y) - mlp.loss(theta - e, X, Y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_linear_network_closed_form():
    """With identity-like weights and positive inputs the ReLUs pass everything, so the
    network is the product of the three affine maps."""
    rng = np.random.default_rng(2)
    W1 = np.abs(rng.standard_normal((64, 16)))
    W2 = np.abs(rng.standard_normal((64, 64)))
    W3 = rng.standard_normal((2, 64))
    b1, b2, b3 = np.ones(64), np.ones(64), np.array([0.5, -0.5])
    theta = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    X = np.abs(rng.standard_normal((5, 16)))
    y, _ = mlp.forward(theta, X)
    ref = ((X @ W1.T + b1) @ W2.T + b2) @ W3.T + b3
    assert np.allclose(y, ref, rtol=1e-12)


def test_adam_first_step_is_signed_lr():
    """At t = 1 with zero moments, Adam moves each parameter by -lr * g/(|g| + eps')."""
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(th, -0.01 * np.sign(g))
