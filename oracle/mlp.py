"""Cost-model network of the config selection, in float64 (test only).

The paper has no learned component; the library adds one: a multilayer
perceptron that predicts a contraction step's log2 time per pass from its
features, so that a kernel configuration can be chosen per step without
measuring it.  This module is the plain definition of that network and of
its training step, written from the textbook definitions:

    z1 = W1 x + b1,   a1 = relu(z1)
    z2 = W2 a1 + b2,  a2 = relu(z2)
    y  = w3 . a2 + b3
    L  = (1/n) sum_i (y_i - t_i)^2

backward by the chain rule (relu'(z) taken as 1 for z > 0, else 0), and
one Adam step (Kingma and Ba, 2015: exponential moving averages of the
gradient and its square, both divided by (1 - beta^t) before the update
p -= lr * m_hat / (sqrt(v_hat) + eps)).

Parameters travel as one flat vector in the order W1 [H][D] (row j = hidden
unit j), b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1] -- the layout of the
library's FP32 parameter array.  D and H are free here.

Pins (tests/test_oracle_pins.py): central finite differences of L against
the analytic gradient; a hand-evaluated two-unit network; the first Adam
step, which moves every parameter with a non-zero gradient by exactly
lr * sign(g) (up to eps).
"""

import numpy as np


def n_params(d: int, h: int) -> int:
    return h * d + h + h * h + h + h + 1


def unpack(p: np.ndarray, d: int, h: int):
    p = np.asarray(p, np.float64)
    assert p.size == n_params(d, h)
    i = 0
    W1 = p[i:i + h * d].reshape(h, d); i += h * d
    b1 = p[i:i + h]; i += h
    W2 = p[i:i + h * h].reshape(h, h); i += h * h
    b2 = p[i:i + h]; i += h
    w3 = p[i:i + h]; i += h
    b3 = p[i]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2), np.ravel(w3),
                           np.atleast_1d(b3)]).astype(np.float64)


def forward(p, X, d: int, h: int, keep: bool = False):
    """Network outputs y (n,) for inputs X (n, d); with keep, also the
    pre-activations needed by the backward pass."""
    W1, b1, W2, b2, w3, b3 = unpack(p, d, h)
    X = np.asarray(X, np.float64)
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ w3 + b3
    if keep:
        return y, (X, z1, a1, z2, a2)
    return y


def loss(p, X, t, d: int, h: int) -> float:
    y = forward(p, X, d, h)
    e = y - np.asarray(t, np.float64)
    return float(np.mean(e * e))


def grad(p, X, t, d: int, h: int):
    """(dL/dp as a flat vector in the parameter layout, L)."""
    W1, b1, W2, b2, w3, b3 = unpack(p, d, h)
    y, (X, z1, a1, z2, a2) = forward(p, X, d, h, keep=True)
    n = X.shape[0]
    e = y - np.asarray(t, np.float64)
    dy = 2.0 * e / n                        # dL/dy_i
    g_w3 = a2.T @ dy
    g_b3 = dy.sum()
    dz2 = np.outer(dy, w3) * (z2 > 0)       # dL/dz2
    g_W2 = dz2.T @ a1
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (z1 > 0)             # dL/dz1
    g_W1 = dz1.T @ X
    g_b1 = dz1.sum(axis=0)
    return pack(g_W1, g_b1, g_W2, g_b2, g_w3, g_b3), float(np.mean(e * e))


def adam_step(p, g, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update; returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
