"""Learned preconditioner: the hand-written network kernels against the FP64 reference
network (oracle/mlp.py), training, fallbacks, and what the trained network (the damping
and cutoff of the spectral correction of the block-diagonal preconditioner) gains over
the method without it."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import mlp as ref  # noqa: E402
from paper_1506_08481_b300 import api, inputs, params  # noqa: E402

WEIGHTS = os.path.join(os.path.dirname(api.__file__), "learned_pc_weights.npy")


def random_weights(rng, scale=0.3):
    w = rng.standard_normal(ref.NW) * scale
    w[ref.NTRAIN:ref.NTRAIN + 16] = rng.standard_normal(16) * 0.2            # mu
    w[ref.NTRAIN + 16:ref.NTRAIN + 32] = rng.uniform(0.5, 2.0, 16)            # sd
    w[ref.NTRAIN + 32:] = rng.uniform(0.5, 2.0, 4)                            # os
    return w.astype(np.float32)


def test_forward_and_gradient_match_reference_network():
    rng = np.random.default_rng(0)
    w = random_weights(rng)
    X = rng.standard_normal((777, 16)).astype(np.float32)
    Yt = rng.standard_normal((777, 4)).astype(np.float32)
    wt, Xt, Yt_t = (torch.tensor(a, device="cuda") for a in (w, X, Yt))
    Y = api.mlp_forward(wt, Xt).double().cpu().numpy()
    Yr = ref.forward(w.astype(np.float64), X.astype(np.float64))
    assert np.linalg.norm(Y - Yr) / np.linalg.norm(Yr) <= 1e-5
    g, loss, _ = api.mlp_grad(wt, Xt, Yt_t)
    lr, gr = ref.loss_and_grad(w.astype(np.float64), X.astype(np.float64), Yt.astype(np.float64))
    assert abs(float(loss.item()) - lr) <= 1e-5 * lr
    g = g.double().cpu().numpy()
    assert np.linalg.norm(g - gr) / np.linalg.norm(gr) <= 1e-4


def test_adam_training_reduces_the_loss():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((4096, 16)).astype(np.float32)
    Yt = np.stack([np.tanh(X[:, 0] - X[:, 3]), X[:, 1] * X[:, 2] * 0.3, np.sin(X[:, 5]), 0 * X[:, 0]], 1)
    w = random_weights(rng, 0.2)
    w[ref.NTRAIN:ref.NTRAIN + 16] = 0.0
    w[ref.NTRAIN + 16:ref.NTRAIN + 32] = 1.0
    w[ref.NTRAIN + 32:] = 1.0
    wt, Xt, Yt_t = torch.tensor(w, device="cuda"), torch.tensor(X, device="cuda"), torch.tensor(Yt.astype(np.float32), device="cuda")
    m, v = torch.zeros(api.SE_MLP_NTRAIN, device="cuda"), torch.zeros(api.SE_MLP_NTRAIN, device="cuda")
    g, l0, scratch = api.mlp_grad(wt, Xt, Yt_t)
    l0 = float(l0.item())
    for step in range(1, 301):
        g, loss, scratch = api.mlp_grad(wt, Xt, Yt_t, scratch)
        api.mlp_adam_step(wt, m, v, g, step, 3e-3)
    assert float(loss.item()) < 0.2 * l0


def _solve_ctx(cfg, precision=1, tol=1e-8, M_max=96):
    sp = params.choose(cfg.L, cfg.N, tol, M_max=M_max, a_eff=params.effective_radius(cfg.rad),
                       precision=precision)
    ctx = api.Context()
    ctx.set_params(sp.xi, sp.M, sp.P, sp.rc)
    ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
    ctx.set_option(api.SE_OPT_PRECISION, precision)
    ctx.set_option(api.SE_OPT_SIZE_MODE, 1)
    ctx.set_option(api.SE_OPT_RESTART, 100)
    ctx.set_config(cfg.pos, cfg.rad, cfg.L)
    return ctx


def test_without_weights_learned_is_the_block_preconditioner():
    cfg = inputs.lognormal(seed=7, n=300, phi=0.3)
    ctx = _solve_ctx(cfg)
    b = torch.tensor(np.random.default_rng(2).standard_normal((cfg.N, 11)), device="cuda")
    x1, i1, r1 = ctx.solve(b, rtol=1e-8, maxit=400, precond=api.SE_PRECOND_BLOCK)
    x2, i2, r2 = ctx.solve(b, rtol=1e-8, maxit=400, precond=api.SE_PRECOND_LEARNED)
    assert i1 == i2 and torch.equal(x1, x2)


def test_bad_weights_are_rejected_or_clamped():
    """Non-finite weights are rejected; weights whose outputs lie far outside the useful
    range give the clamped damping and cutoff, and the solve still converges (a correction
    that stalls falls back to the block preconditioner)."""
    cfg = inputs.mono_dense(seed=8, n=2000, phi=0.45)
    ctx = _solve_ctx(cfg, precision=0, tol=5e-7, M_max=64)
    w = random_weights(np.random.default_rng(3))
    bad = w.copy()
    bad[5] = np.nan
    with pytest.raises(api.SeError) as e:
        ctx.set_learned_weights(bad)
    assert e.value.code == api.SE_ERR_NONFINITE
    b = torch.tensor(np.random.default_rng(4).standard_normal((cfg.N, 11)), device="cuda")
    xb, ib, rb = ctx.solve(b, rtol=1e-6, maxit=800, precond=api.SE_PRECOND_BLOCK)
    for big in (-50.0, 50.0):
        w2 = w.copy()
        w2[:ref.NTRAIN] = 0.0
        w2[ref.NTRAIN - 4:ref.NTRAIN - 2] = big          # b3 of outputs 0 and 1
        ctx.set_learned_weights(w2)
        xl, il, rl = ctx.solve(b, rtol=1e-6, maxit=800, precond=api.SE_PRECOND_LEARNED)
        assert rl <= 1e-6, big


# Held-out configurations, seeds disjoint from training (train_pc.py uses 1000..1159):
# the kinds the network is trained on, including two on which the fixed default damping
# of the spectral correction stalls (monodisperse phi = 0.45 at N = 20000, bidisperse).
HELD_OUT = [("lognormal", 4000, 0.4, 5001), ("mono", 20000, 0.45, 5002), ("bidisperse", 4000, 0.3, 5003),
            ("mono", 3000, 0.2, 5004)]


def _held_out(kind, n, phi, seed):
    if kind == "lognormal":
        return inputs.lognormal(seed=seed, n=n, phi=phi)
    if kind == "mono":
        return inputs.mono_dense(seed=seed, n=n, phi=phi)
    return inputs.bidisperse(seed=seed, n=n, phi=phi)


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained weights in the package")
def test_trained_network_gain_on_held_out_configurations():
    """What the trained network gains over the method without it.  On every held-out
    configuration the learned preconditioner (the spectral correction with the network's
    damping and cutoff) needs fewer products than the plain block-diagonal preconditioner
    it corrects, and at least 1.5x fewer summed over the set; summed over the set it needs
    no more than the spectral correction with the fixed default damping and cutoff (the
    best single setting on the training set), never more than 1.25x on one configuration,
    and every solve meets the tolerance (the network only changes the iteration count)."""
    w = np.load(WEIGHTS)
    tot = {"block": 0, "learned": 0, "spectral": 0}
    for kind, n, phi, seed in HELD_OUT:
        cfg = _held_out(kind, n, phi, seed)
        ctx = _solve_ctx(cfg, precision=0, tol=5e-7, M_max=128)
        b = torch.tensor(np.random.default_rng(seed).standard_normal((cfg.N, 11)), device="cuda")
        xb, ib, rb = ctx.solve(b, rtol=1e-6, maxit=1500, precond=api.SE_PRECOND_BLOCK)
        xs, is_, rs = ctx.solve(b, rtol=1e-6, maxit=1500, precond=api.SE_PRECOND_SPECTRAL)
        ctx.set_learned_weights(w)
        xl, il, rl = ctx.solve(b, rtol=1e-6, maxit=1500, precond=api.SE_PRECOND_LEARNED)
        # every solve meets the tolerance on its FP64-equivalent residual: the network
        # changes how many products the solution takes, not the system that is solved
        assert rb <= 1e-6 and rl <= 1e-6 and rs <= 1e-6
        print(f"{kind} N={n} phi={phi}: products block {ib}, spectral default {is_}, learned {il}")
        assert il < ib, (kind, n)
        assert il <= 1.25 * is_, (kind, n)
        tot["block"] += ib
        tot["learned"] += il
        tot["spectral"] += is_
    print("summed products:", tot)
    assert tot["block"] >= 1.5 * tot["learned"]
    assert tot["learned"] <= tot["spectral"]
