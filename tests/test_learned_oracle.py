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
