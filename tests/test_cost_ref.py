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


def _hand_network():
    """A network whose output is worked out by hand (only a few weights are
    non-zero; the rest of the 64 units stay at zero):
      layer 1: a1[0] = x0, a1[1] = -x1, a1[2] = 1 (bias only)
      layer 2: a2[0] = 2 h1[1], a2[1] = 3 h1[0], a2[2] = -h1[2],
               a2[3] = h1[2] - 2, a2[4] = -h1[0]
      output : h2[0] + h2[1] + 5 h2[2] + 7 h2[3] + 10 h2[4] + 0.5
    Sample (1, -2): h1 = (1, 2, 1), a2 = (4, 3, -1, -1, -1), h2 = (4, 3, 0, 0, 0),
      out = 4 + 3 + 0.5 = 7.5.
    Sample (-1, 3): a1 = (-1, -3, 1), h1 = (0, 0, 1), a2 = (0, 0, -1, -1, 0),
      h2 = 0, out = 0.5.
    A transposed W2 gives 6 + 2 + 0.5 = 8.5 on the first sample; no ReLU on
    layer 2 gives 4 + 3 - 5 - 7 - 10 + 0.5 = -14.5; no ReLU on layer 1 gives
    a2[4] = 1 on the second sample, out 10.5; b1 added as a weight column or
    b3 left out shifts both samples."""
    p = np.zeros(cost_mlp.P)
    q = cost_mlp.unpack(p)
    q["W1"][0, 0] = 1.0
    q["W1"][1, 1] = -1.0
    q["b1"][2] = 1.0
    q["W2"][0, 1] = 2.0
    q["W2"][1, 0] = 3.0
    q["W2"][2, 2] = -1.0
    q["W2"][3, 2] = 1.0
    q["b2"][3] = -2.0
    q["W2"][4, 0] = -1.0
    q["W3"][:5] = [1.0, 1.0, 5.0, 7.0, 10.0]
    q["b3"][0] = 0.5
    X = np.array([[1.0, -2.0, 0.0, 0.0, 0.0], [-1.0, 3.0, 0.0, 0.0, 0.0]])
    return p, X


def test_forward_matches_a_hand_worked_network():
    p, X = _hand_network()
    out, _ = cost_mlp.forward(p, X)
    np.testing.assert_allclose(out, [7.5, 0.5], rtol=0, atol=1e-12)
    # mean squared error against y = (7, 1): ((0.5)^2 + (-0.5)^2) / 2
    assert abs(cost_mlp.loss(p, X, np.array([7.0, 1.0])) - 0.25) < 1e-12


def test_gradient_of_the_hand_worked_network():
    """d loss / d b3 = mean(2 (out - y)); for y = (7, 0): (2 * 0.5 + 2 * 0.5) / 2 = 1.
    d loss / d W3[0] = mean(2 (out - y) h2[0]) = (2 * 0.5 * 4 + 0) / 2 = 2, and
    d loss / d W3[2] = 0 (h2[2] is 0 on both samples)."""
    p, X = _hand_network()
    g = cost_mlp.unpack(cost_mlp.grad(p, X, np.array([7.0, 0.0])))
    assert abs(g["b3"][0] - 1.0) < 1e-12
    assert abs(g["W3"][0] - 2.0) < 1e-12
    assert g["W3"][2] == 0.0


def test_one_adam_step_worked_by_hand():
    """Kingma and Ba (2015), Algorithm 1, at t = 3 with g = 0.5, m = 0.2,
    v = 0.01, lr = 0.01:
      m' = 0.9 * 0.2 + 0.1 * 0.5 = 0.23
      v' = 0.999 * 0.01 + 0.001 * 0.25 = 0.01024
      m^ = 0.23 / (1 - 0.9^3) = 0.23 / 0.271 = 0.8487084870848708...
      v^ = 0.01024 / (1 - 0.999^3) = 0.01024 / 0.002997001 = 3.4167489433603792...
      step = 0.01 * m^ / (sqrt(v^) + 1e-8) = 0.01 * 0.84870848708 / 1.84844501685
           = 0.0045914727208371812..."""
    p, m, v = cost_mlp.adam_step(np.array([1.0]), np.array([0.5]), np.array([0.2]), np.array([0.01]), 3, 0.01)
    assert abs(m[0] - 0.23) < 1e-15
    assert abs(v[0] - 0.01024) < 1e-15
    assert abs((1.0 - p[0]) - 0.0045914727208371812) < 1e-15


def test_first_adam_step_moves_by_lr_times_sign():
    """At t = 1 from zero moments the bias correction makes m^ = g and
    v^ = g^2, so every parameter moves by lr * sign(g) (up to eps): without
    the correction the step would be lr * 0.1 / sqrt(0.001) = 3.16 lr.
    (Swapped betas cancel at t = 1; the t = 3 step above catches them.)"""
    g = np.array([3.0, -0.02, 1e-3, -250.0])
    p, m, v = cost_mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-4)


def test_adam_eps_is_added_outside_the_square_root():
    """g = 1e-8 at t = 1: m^ = 1e-8, v^ = 1e-16, sqrt(v^) = 1e-8, so the step
    is lr * 1e-8 / (1e-8 + 1e-8) = lr / 2 (eps inside the root would give
    lr * 1e-8 / sqrt(1e-8 + 1e-16) = lr * 1e-4)."""
    p, _, _ = cost_mlp.adam_step(np.zeros(1), np.array([1e-8]), np.zeros(1), np.zeros(1), 1, 0.01)
    assert abs(p[0] + 0.005) < 1e-12
