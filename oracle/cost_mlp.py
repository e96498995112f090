"""Double-precision reference of the learned tick-cost model (test
infrastructure: only the tests import it; the CUDA model never does).

A multilayer perceptron 5 -> 64 -> 64 -> 1 with ReLU hidden layers, mean
squared error, and full-batch Adam (Kingma and Ba, 2015: beta1 0.9, beta2
0.999, eps 1e-8, bias-corrected moments), written out step by step in numpy
float64.  Parameter vector layout (the same as the C ABI's): W1[64][5],
b1[64], W2[64][64], b2[64], W3[64], b3.  Pinned in the CPU tests: the forward
pass by a network whose output is worked out by hand, one Adam step by
bias-corrected moments worked out by hand, and the gradient by finite
differences of the (pinned) loss.
"""
from __future__ import annotations

import numpy as np

IN, H = 5, 64
SIZES = [("W1", H * IN), ("b1", H), ("W2", H * H), ("b2", H), ("W3", H), ("b3", 1)]
P = sum(n for _, n in SIZES)


def unpack(p):
    out, o = {}, 0
    for name, n in SIZES:
        out[name] = p[o:o + n]
        o += n
    out["W1"] = out["W1"].reshape(H, IN)
    out["W2"] = out["W2"].reshape(H, H)
    return out


def init(seed: int) -> np.ndarray:
    """He-uniform weights, zero biases (float64)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(P)
    q = unpack(p)
    q["W1"][:] = rng.uniform(-1, 1, (H, IN)) * np.sqrt(6.0 / IN)
    q["W2"][:] = rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / H)
    q["W3"][:] = rng.uniform(-1, 1, H) * np.sqrt(6.0 / H)
    return p


def forward(p, X):
    q = unpack(np.asarray(p, np.float64))
    a1 = X @ q["W1"].T + q["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ q["W2"].T + q["b2"]
    h2 = np.maximum(a2, 0.0)
    out = h2 @ q["W3"] + q["b3"][0]
    return out, (a1, h1, a2, h2)


def loss(p, X, y):
    out, _ = forward(p, X)
    return float(np.mean((out - y) ** 2))


def grad(p, X, y):
    """Gradient of the mean squared error by backpropagation."""
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    q = unpack(np.asarray(p, np.float64))
    out, (a1, h1, a2, h2) = forward(p, X)
    n = X.shape[0]
    dout = 2.0 * (out - y) / n                       # d loss / d out
    g = {"W3": h2.T @ dout, "b3": np.array([dout.sum()])}
    d2 = np.outer(dout, q["W3"]) * (a2 > 0)          # d loss / d a2
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(0)
    d1 = (d2 @ q["W2"]) * (a1 > 0)                   # d loss / d a1
    g["W1"] = d1.T @ X
    g["b1"] = d1.sum(0)
    return np.concatenate([g[name].reshape(-1) for name, _ in SIZES])


BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def adam_step(p, g, m, v, t, lr):
    """One Adam update (Kingma and Ba 2015, Algorithm 1) at step t >= 1 with
    gradient g: moments m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
    bias-corrected m^ = m / (1 - b1^t), v^ = v / (1 - b2^t), and
    p <- p - lr m^ / (sqrt(v^) + eps).  Returns (p, m, v)."""
    m = BETA1 * m + (1.0 - BETA1) * g
    v = BETA2 * v + (1.0 - BETA2) * g * g
    mhat = m / (1.0 - BETA1 ** t)
    vhat = v / (1.0 - BETA2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + EPS), m, v


def adam(p, X, y, epochs, lr, m=None, v=None, step0=0):
    """`epochs` full-batch Adam steps; returns (p, m, v, loss before the last step)."""
    p = np.array(p, np.float64)
    m = np.zeros(P) if m is None else np.array(m, np.float64)
    v = np.zeros(P) if v is None else np.array(v, np.float64)
    last = None
    for e in range(epochs):
        last = loss(p, X, y)
        p, m, v = adam_step(p, grad(p, X, y), m, v, step0 + e + 1, lr)
    return p, m, v, last
