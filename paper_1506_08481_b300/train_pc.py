"""Train the learned correction of the block-diagonal far-field preconditioner.

  python -m paper_1506_08481_b300.train_pc [--configs 200] [--n 96] [--epochs 400]

Training data come from the method itself: for each generated configuration (log-normal
radii, mean 1, std 0.2, volume fraction 0.4) the dense F,T,S grand mobility is assembled
column by column from FP64 Spectral Ewald products (se_mobility_apply), inverted, and the
target of sphere i is the isotropic part of [M^-1]_ii^-1 - [M]_ii, made dimensionless by
the isolated-sphere mobilities (the change that turns the plain block into the inverse of
the diagonal block of M^-1).  Features come from se_learned_features; the network is
trained with the library's kernels (se_mlp_grad, se_mlp_adam_step).  Writes
learned_pc_weights.npy (SE_MLP_NW floats) and learned_pc_weights.json next to this file.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import api, inputs, params

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "learned_pc_weights.npy")
NC = 11


def dense_mobility(ctx, N):
    import torch
    n = N * NC
    Mt = torch.empty(n, n, device="cuda", dtype=torch.float64)
    e = torch.zeros(N, NC, device="cuda", dtype=torch.float64)
    y = torch.empty_like(e)
    for col in range(n):
        e.view(-1)[col] = 1.0
        ctx.apply(e, y)
        Mt[col] = y.view(-1)
        e.view(-1)[col] = 0.0
    return Mt.T.contiguous()


def targets_for(ctx, cfg):
    """Dimensionless isotropic corrections [N, 4] and features [N, 16]."""
    import torch
    M = dense_mobility(ctx, cfg.N)
    Mi = torch.linalg.inv(M)
    N = cfg.N
    idx = torch.arange(N, device="cuda")
    blk = lambda A: A.view(N, NC, N, NC)[idx, :, idx, :]          # diagonal blocks [N, 11, 11]
    B = blk(M)
    D = torch.linalg.inv(blk(Mi)) - B
    a = torch.tensor(cfg.rad, device="cuda", dtype=torch.float64)
    iso = torch.stack([1 / (6 * math.pi * a), 1 / (8 * math.pi * a ** 3), 3 / (20 * math.pi * a ** 3)], 1)
    dF = torch.diagonal(D[:, 0:3, 0:3], dim1=1, dim2=2).mean(1)
    dT = torch.diagonal(D[:, 3:6, 3:6], dim1=1, dim2=2).mean(1)
    dS = torch.diagonal(D[:, 6:11, 6:11], dim1=1, dim2=2).mean(1)
    Y = torch.stack([dF / iso[:, 0], dT / iso[:, 1], dS / iso[:, 2], torch.zeros_like(dF)], 1)
    return Y.float(), ctx.learned_features()


def make_context(cfg, tol=1e-7, M_max=64):
    sp = params.choose(cfg.L, cfg.N, tol, M_max=M_max, a_eff=params.effective_radius(cfg.rad))
    ctx = api.Context()
    ctx.set_params(sp.xi, sp.M, sp.P, sp.rc)
    ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
    ctx.set_option(api.SE_OPT_PRECISION, 1)
    ctx.set_config(cfg.pos, cfg.rad, cfg.L)
    return ctx


def build_dataset(nconf, n, seed0, phi=0.4, log=print):
    import torch
    Xs, Ys = [], []
    t = time.time()
    for c in range(nconf):
        cfg = inputs.lognormal(seed=seed0 + c, n=n, phi=phi)
        ctx = make_context(cfg)
        Y, X = targets_for(ctx, cfg)
        ctx.close()
        Xs.append(X)
        Ys.append(Y)
        if (c + 1) % 25 == 0:
            log(f"  {c + 1}/{nconf} configurations ({time.time() - t:.0f} s)")
    return torch.cat(Xs), torch.cat(Ys)


def init_weights(X, Y, seed=0):
    """Xavier-initialised parameters, input standardisation and output scale."""
    import torch
    from math import sqrt
    rng = np.random.default_rng(seed)
    F, H, O = 16, 64, 4
    w = []
    for fan_out, fan_in in ((H, F), (H, H), (O, H)):
        w.append(rng.standard_normal(fan_out * fan_in) * sqrt(1.0 / fan_in))
        w.append(np.zeros(fan_out))
    mu = X.double().mean(0).cpu().numpy()
    sd = X.double().std(0).cpu().numpy()
    sd = np.where(sd > 1e-6, sd, 1.0)
    os_ = Y.double().std(0).cpu().numpy()
    os_ = np.where(os_ > 1e-9, os_, 1.0)
    packed = np.concatenate(w + [mu, sd, os_]).astype(np.float32)
    assert packed.size == api.SE_MLP_NW
    return torch.tensor(packed, device="cuda")


def train(X, Y, epochs=400, lr=3e-3, batch=8192, seed=0, log=print):
    import torch
    w = init_weights(X, Y, seed)
    m = torch.zeros(api.SE_MLP_NTRAIN, device="cuda")
    v = torch.zeros_like(m)
    g_rng = torch.Generator(device="cuda").manual_seed(seed)
    n = X.shape[0]
    step, scratch, history = 0, None, []
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g_rng)
        tot = 0.0
        for b0 in range(0, n, batch):
            sel = perm[b0:b0 + batch]
            g, loss, scratch = api.mlp_grad(w, X[sel].contiguous(), Y[sel].contiguous(), scratch)
            step += 1
            api.mlp_adam_step(w, m, v, g, step, lr)
            tot += float(loss.item()) * sel.numel()
        history.append(tot / n)
        if ep % 50 == 0 or ep == epochs - 1:
            log(f"  epoch {ep}: loss {history[-1]:.4e}")
    return w, history


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--configs", type=int, default=200)
    ap.add_argument("--n", type=int, default=96)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--out", default=WEIGHTS)
    args = ap.parse_args()
    t = time.time()
    X, Y = build_dataset(args.configs, args.n, args.seed0)
    t_data = time.time() - t
    w, hist = train(X, Y, epochs=args.epochs)
    np.save(args.out, w.cpu().numpy())
    meta = {"configs": args.configs, "n": args.n, "phi": 0.4, "radii": "log-normal mean 1 std 0.2",
            "seeds": [args.seed0, args.seed0 + args.configs - 1], "samples": int(X.shape[0]),
            "loss_first": hist[0], "loss_last": hist[-1], "epochs": args.epochs,
            "target_std": Y.double().std(0).cpu().tolist(), "data_seconds": t_data,
            "train_seconds": time.time() - t - t_data}
    with open(args.out.replace(".npy", ".json"), "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
