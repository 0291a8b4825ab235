"""Train the learned preconditioner: the network that sets the damping theta, the cutoff
k_c <a> and the norm cap c_max of the long-wavelength (spectral) correction of the
block-diagonal far-field preconditioner.

  python -m paper_1506_08481_b300.train_pc [--configs 160] [--epochs 300]

Training data come from the method itself.  For each generated configuration (mono-, bi-
and polydisperse suspensions, volume fractions 0.1-0.45, N from 1000 to 50000) the
library solves M x = b (11 components, FP32 products with FP64 refinement, GMRES(100) to
1e-6) with the spectral correction at every (theta, k_c <a>, c_max) of a grid and records
the products each solve took.  The configuration's target is the grid point with the
fewest products; among those within 2% of it, the smallest c_max and theta (the safer
correction).  Every particle of the configuration carries the target; the network's mean
over the particles is its prediction for the configuration.  Features come from
se_learned_features; the network is trained with the library's kernels (se_mlp_grad,
se_mlp_adam_step).  Writes learned_pc_weights.npy (SE_MLP_NW floats) and
learned_pc_weights.json (the data and the training record) next to this file.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import time

import numpy as np

from . import api, inputs, params

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "learned_pc_weights.npy")
NC = 11
THETAS = (0.9, 0.98)
KAS = (0.6, 0.9, 1.2)
CMAXS = (0.9, 0.95, 0.97, 0.985)


def config_spec(k: int, seed0: int):
    """The k-th configuration of the training set: (kind, N, phi, radius parameter, seed)."""
    rng = np.random.default_rng(seed0 + 7919 * k)
    kind = ("mono", "bidisperse", "lognormal")[k % 3]
    u = rng.uniform()
    N = int(round(math.exp(math.log(1000) + u * (math.log(20000) - math.log(1000)))))
    if k % 40 == 39:
        N = 50000
    phi = float(rng.uniform(0.1, 0.45 if kind == "mono" else 0.4))
    par = {"mono": 1.0, "bidisperse": float(rng.choice([1.5, 2.0])), "lognormal": float(rng.uniform(0.1, 0.3))}[kind]
    return kind, N, phi, par, seed0 + k


def make_config(spec):
    kind, N, phi, par, seed = spec
    rng = np.random.default_rng(seed)
    if kind == "mono":
        rad = np.ones(N)
    elif kind == "bidisperse":
        rad = inputs.radii_bidisperse(N, 1.0, par, 0.5, rng)
    else:
        rad = inputs.radii_lognormal(N, 1.0, par, rng)
    L = inputs.box_side(rad, phi)
    pos = inputs.positions_dense(rad, L, rng, sweeps=4)
    return inputs.Config(f"{kind}_n{N}_phi{phi:.2f}_s{seed}", L, pos, rad)


def solve_context(cfg, tol=5e-7, M_max=128):
    sp = params.choose(cfg.L, cfg.N, tol, M_max=M_max, a_eff=params.effective_radius(cfg.rad), precision=0)
    ctx = api.Context()
    ctx.set_params(sp.xi, sp.M, sp.P, sp.rc)
    ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
    ctx.set_option(api.SE_OPT_SIZE_MODE, 1)
    ctx.set_option(api.SE_OPT_RESTART, 100)
    ctx.set_config(cfg.pos, cfg.rad, cfg.L)
    return ctx


def products(ctx, b, precond, theta=0.0, ka=0.9, cmax=0.97, maxit=600):
    """Products of one solve to 1e-6 (maxit + 1 if it did not converge)."""
    ctx.set_option(api.SE_OPT_PC_THETA, theta)
    ctx.set_option(api.SE_OPT_PC_KA, ka)
    ctx.set_option(api.SE_OPT_PC_CMAX, cmax)
    _, it, rel = ctx.solve(b, rtol=1e-6, maxit=maxit, precond=precond, allow_not_converged=True)
    ctx.set_option(api.SE_OPT_PC_THETA, 0.0)
    ctx.set_option(api.SE_OPT_PC_KA, 0.9)
    ctx.set_option(api.SE_OPT_PC_CMAX, 0.97)
    return it if rel <= 1e-6 else maxit + 1


def label(ctx, cfg, seed):
    """Products on the (theta, k_c a, c_max) grid; the target; the block and default counts."""
    import torch
    b = torch.tensor(np.random.default_rng(seed).standard_normal((cfg.N, NC)), device="cuda")
    grid = {}
    for th in THETAS:
        for ka in KAS:
            for cm in CMAXS:
                grid[(th, ka, cm)] = products(ctx, b, api.SE_PRECOND_SPECTRAL, th, ka, cm)
    return {"target": target_of(grid), "grid": {",".join(str(v) for v in k): p for k, p in grid.items()},
            "block": products(ctx, b, api.SE_PRECOND_BLOCK), "spectral_default": products(ctx, b, api.SE_PRECOND_SPECTRAL)}


def target_of(grid):
    """The grid point with the fewest products; among those within 2% of it, the smallest
    c_max, then the smallest theta."""
    best = min(grid.values())
    return min((k for k, v in grid.items() if v <= 1.02 * best), key=lambda k: (k[2], k[0], grid[k]))


def build_dataset(specs, per_config=2000, labels=None, log=print):
    """Features and targets of every configuration; labels: records of an earlier run (their
    product grids are reused, only the features are computed again)."""
    import torch
    t = time.time()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        cfgs = pool.map(make_config, specs)
    log(f"  {len(cfgs)} configurations generated in {time.time() - t:.0f} s")
    Xs, Ys, recs = [], [], []
    rng = np.random.default_rng(0)
    t = time.time()
    old = {r["name"]: r for r in labels} if labels else {}
    for c, (cfg, spec) in enumerate(zip(cfgs, specs)):
        ctx = solve_context(cfg)
        if cfg.name in old:
            rec = dict(old[cfg.name])
            grid = {tuple(float(v) for v in k.split(",")): p for k, p in rec["grid"].items()}
            rec["target"] = target_of(grid)
        else:
            rec = label(ctx, cfg, spec[4])
        feat = ctx.learned_features()
        ctx.close()
        sel = torch.tensor(rng.choice(cfg.N, min(per_config, cfg.N), replace=False), device="cuda")
        X = feat[sel]
        Y = torch.zeros(X.shape[0], 4, device="cuda")
        Y[:, 0], Y[:, 1], Y[:, 2] = rec["target"][0], rec["target"][1], rec["target"][2]
        Xs.append(X)
        Ys.append(Y)
        rec.update({"name": cfg.name, "N": cfg.N})
        recs.append(rec)
        if (c + 1) % 20 == 0:
            log(f"  {c + 1}/{len(cfgs)} configurations labelled ({time.time() - t:.0f} s)")
    return torch.cat(Xs), torch.cat(Ys), recs


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
    os_ = Y.double().abs().max(0).values.cpu().numpy()
    os_ = np.where(os_ > 1e-9, os_, 1.0)
    packed = np.concatenate(w + [mu, sd, os_]).astype(np.float32)
    assert packed.size == api.SE_MLP_NW
    return torch.tensor(packed, device="cuda")


def train(X, Y, epochs=300, lr=2e-3, batch=8192, seed=0, log=print):
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
    ap.add_argument("--configs", type=int, default=160)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--labels-from", default=None,
                    help="a learned_pc_weights.json of an earlier run: reuse its product grids")
    args = ap.parse_args()
    t = time.time()
    specs = [config_spec(k, args.seed0) for k in range(args.configs)]
    labels = None
    if args.labels_from:
        with open(args.labels_from) as f:
            labels = json.load(f)["records"]
    X, Y, recs = build_dataset(specs, labels=labels)
    t_data = time.time() - t
    w, hist = train(X, Y, epochs=args.epochs)
    np.save(args.out, w.cpu().numpy())
    tot = {k: sum(r[k] for r in recs) for k in ("block", "spectral_default")}
    tot["best_on_grid"] = sum(min(r["grid"].values()) for r in recs)
    meta = {"configs": args.configs, "seeds": [args.seed0, args.seed0 + args.configs - 1],
            "grid": {"theta": THETAS, "k_c_a": KAS, "c_max": CMAXS}, "samples": int(X.shape[0]),
            "loss_first": hist[0], "loss_last": hist[-1], "epochs": args.epochs,
            "products_summed_over_configs": tot, "data_seconds": t_data,
            "train_seconds": time.time() - t - t_data, "records": recs}
    with open(args.out.replace(".npy", ".json"), "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps({k: v for k, v in meta.items() if k != "records"}))


if __name__ == "__main__":
    main()
