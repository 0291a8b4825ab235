"""Pins of the FP64 reference network (no GPU): back-propagation equals central
finite differences of the loss, and the packed layout round-trips."""
import numpy as np

from oracle import mlp


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = rng.standard_normal(mlp.NW) * 0.3
    w[mlp.NTRAIN + 16:mlp.NTRAIN + 32] = rng.uniform(0.5, 2.0, 16)      # sd > 0
    w[mlp.NTRAIN + 32:] = rng.uniform(0.5, 2.0, 4)                      # os > 0
    X = rng.standard_normal((9, mlp.F))
    Yt = rng.standard_normal((9, mlp.O))
    loss, g = mlp.loss_and_grad(w, X, Yt)
    for p in rng.choice(mlp.NTRAIN, 60, replace=False):
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[p] += h
        wm[p] -= h
        fd = (mlp.loss_and_grad(wp, X, Yt)[0] - mlp.loss_and_grad(wm, X, Yt)[0]) / (2 * h)
        assert abs(fd - g[p]) <= 1e-7 * max(1.0, abs(g[p]))


def test_forward_consistent_with_loss():
    rng = np.random.default_rng(1)
    w = rng.standard_normal(mlp.NW) * 0.2
    w[mlp.NTRAIN:] = 1.0
    X = rng.standard_normal((5, mlp.F))
    Y = mlp.forward(w, X)
    loss, _ = mlp.loss_and_grad(w, X, Y)
    assert loss < 1e-24


def test_closed_forms_of_degenerate_networks():
    """Zero hidden weights and biases: every hidden unit is tanh(0) = 0, so the output is
    b3 * os whatever the input.  One hidden path (single nonzero weights): the output is
    os * w3 * tanh(w2 * tanh(w1 (x - mu)/sd + b1))."""
    rng = np.random.default_rng(2)
    w = np.zeros(mlp.NW)
    p = mlp.unpack(w)                       # views into w
    p["b3"][:] = rng.standard_normal(mlp.O)
    p["mu"][:] = rng.standard_normal(mlp.F)
    p["sd"][:] = rng.uniform(0.5, 2.0, mlp.F)
    p["os"][:] = rng.uniform(0.5, 2.0, mlp.O)
    X = rng.standard_normal((7, mlp.F))
    np.testing.assert_array_equal(mlp.forward(w, X), np.tile(p["b3"] * p["os"], (7, 1)))
    p["b3"][:] = 0.0
    p["W1"][5, 3], p["b1"][5], p["W2"][9, 5], p["W3"][2, 9] = 0.7, -0.2, 1.3, -0.9
    y = mlp.forward(w, X)
    xs = (X[:, 3] - p["mu"][3]) / p["sd"][3]
    expect = p["os"][2] * -0.9 * np.tanh(1.3 * np.tanh(0.7 * xs - 0.2))
    np.testing.assert_allclose(y[:, 2], expect, rtol=1e-14, atol=0)
    assert np.all(y[:, [0, 1, 3]] == 0.0)
