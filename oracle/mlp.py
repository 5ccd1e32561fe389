"""Reference MLP for learned Krylov sizing (oracle; test infrastructure).

The network maps 16 features of the first outer Krylov coefficients to 2 outputs
(log k*, log l*): 16 -> 64 -> 64 -> 2, ReLU after the two hidden layers, mean
squared error loss. This is the plain definition in double precision, with the
gradient by the chain rule written out layer by layer, and one Adam step
(Kingma & Ba 2015, with bias correction).

Parameter vector layout (5378 entries): W1 [64][16], b1 [64], W2 [64][64], b2 [64],
W3 [2][64], b3 [2] (row-major, out x in).
"""
import numpy as np

SIZES = [(64, 16), (64, 64), (2, 64)]
N_PARAMS = sum(o * i + o for o, i in SIZES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out = []
    p = 0
    for o, i in SIZES:
        W = theta[p:p + o * i].reshape(o, i)
        p += o * i
        b = theta[p:p + o]
        p += o
        out.append((W, b))
    return out


def forward(theta, X):
    """Returns (outputs, cache) for inputs X of shape (n, 16)."""
    (W1, b1), (W2, b2), (W3, b3) = unpack(theta)
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ W3.T + b3
    return y, (X, z1, a1, z2, a2)


def loss(theta, X, Y):
    y, _ = forward(theta, X)
    return float(np.mean(np.sum((y - Y) ** 2, axis=1)))


def loss_grad(theta, X, Y):
    """Mean over samples of the squared error summed over the 2 outputs, and its gradient."""
    (W1, b1), (W2, b2), (W3, b3) = unpack(theta)
    y, (X, z1, a1, z2, a2) = forward(theta, X)
    n = X.shape[0]
    d3 = 2.0 * (y - Y) / n
    gW3 = d3.T @ a2
    gb3 = d3.sum(0)
    d2 = (d3 @ W3) * (z2 > 0)
    gW2 = d2.T @ a1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (z1 > 0)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return float(np.mean(np.sum((y - Y) ** 2, axis=1))), g


def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed):
    """He-style uniform initialisation (deterministic)."""
    rng = np.random.default_rng(seed)
    parts = []
    for o, i in SIZES:
        lim = np.sqrt(6.0 / i)
        parts.append(rng.uniform(-lim, lim, o * i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)
