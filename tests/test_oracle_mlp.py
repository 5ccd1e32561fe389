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


def test_adam_three_steps_hand_computed():
    """Steps t = 1, 2, 3 of Adam (Kingma & Ba 2015, Algorithm 1) on two parameters, with
    beta1 = 1/2, beta2 = 3/4, lr = 1/10, eps = 1/100, worked out by hand in exact fractions:

      parameter 0, gradients 2, 4, -2, theta_0 = 1:
        t=1: m = 1,    v = 1,      m^ = 2,    v^ = 4
        t=2: m = 5/2,  v = 19/4,   m^ = 10/3, v^ = 76/7
        t=3: m = 1/4,  v = 73/16,  m^ = 2/7,  v^ = 292/37
      parameter 1, gradients -1, 3, 1/2, theta_0 = -1/2:
        t=1: m = -1/2, v = 1/4,    m^ = -1,   v^ = 1
        t=2: m = 5/4,  v = 39/16,  m^ = 5/3,  v^ = 39/7
        t=3: m = 7/8,  v = 121/64, m^ = 1,    v^ = 121/37
      theta_t = theta_{t-1} - lr m^ / (sqrt(v^) + eps).
    beta1 and beta2 differ and the bias corrections 1 - beta^t change with t, so swapping
    the betas, dropping a correction or using the wrong power fails at t = 2 or 3."""
    expect = {1: [0.900497512437811, -0.400990099009901],
              2: [0.7996407712601878, -0.47130209453229205],
              3: [0.7895063677291949, -0.526295832219544]}
    grads = {1: [2.0, -1.0], 2: [4.0, 3.0], 3: [-2.0, 0.5]}
    th, m, v = np.array([1.0, -0.5]), np.zeros(2), np.zeros(2)
    for t in (1, 2, 3):
        th, m, v = mlp.adam_step(th, np.array(grads[t]), m, v, t, lr=0.1, beta1=0.5, beta2=0.75, eps=0.01)
        assert np.allclose(th, expect[t], rtol=0, atol=1e-14), (t, th)
    assert np.allclose(m, [0.25, 0.875], rtol=0, atol=1e-15)
    assert np.allclose(v, [73 / 16, 121 / 64], rtol=0, atol=1e-15)
