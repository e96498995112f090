"""Pins of the double-precision cost-model reference (oracle/cost_mlp.py):
its backpropagated gradient against central finite differences of the loss,
and Adam reducing the loss of a learnable target.  No GPU."""
import numpy as np

from oracle import cost_mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = cost_mlp.init(1) * 0.5
    X = rng.normal(size=(17, 5))
    y = rng.normal(size=17)
    g = cost_mlp.grad(p, X, y)
    idx = rng.choice(cost_mlp.P, size=60, replace=False)
    idx = np.concatenate([idx, [cost_mlp.P - 1, 0, 64 * 5]])        # b3, W1[0][0], b1[0]
    h = 1e-6
    for i in idx:
        e = np.zeros(cost_mlp.P)
        e[i] = h
        fd = (cost_mlp.loss(p + e, X, y) - cost_mlp.loss(p - e, X, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_adam_learns_a_smooth_target():
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, size=(200, 5))
    y = 0.5 * X[:, 0] - X[:, 1] ** 2 + 0.3 * X[:, 2] * X[:, 3]
    p0 = cost_mlp.init(3)
    l0 = cost_mlp.loss(p0, X, y)
    p, _, _, _ = cost_mlp.adam(p0, X, y, epochs=300, lr=3e-3)
    assert cost_mlp.loss(p, X, y) < 0.1 * l0


def test_parameter_layout_size():
    assert cost_mlp.P == 64 * 5 + 64 + 64 * 64 + 64 + 64 + 1
