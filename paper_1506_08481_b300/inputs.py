"""Seeded synthetic inputs: sphere configurations in a cubic periodic box and
random multipole moments.

This module holds no mobility arithmetic.  It serves both the CUDA path and the
FP64 oracle (the test-suite feeds the same arrays to both), and imports nothing
from either.

Workloads (the configurations the bench and the parity tests use):
  mono_n100      N=100, a=1, phi=0.2, uniform random non-overlapping (RSA)
  bidisperse     N=2000, radii 1 and 2 (50/50 by number), phi=0.3 (RSA)
  lognormal      N=20000, log-normal radii (mean 1, std 0.2), phi=0.4
                 (FCC-lattice start, overlap removal, hard-sphere MC sweeps)
  batch64        64 boxes, N ~ U[500, 8000], radii 1 and 1.5, phi ~ U[0.1, 0.45]
  mono_n200k     N=200000, a=1, phi=0.45 (FCC-lattice subset, jitter, MC sweeps)
Moments are i.i.d. N(0, 1) per component.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.spatial import cKDTree


@dataclass
class Config:
    """A periodic configuration: positions in [0, L)^3 and radii."""
    name: str
    L: float
    pos: np.ndarray      # [N, 3] float64
    rad: np.ndarray      # [N] float64

    @property
    def N(self) -> int:
        return int(self.pos.shape[0])

    @property
    def phi(self) -> float:
        return float(4.0 / 3.0 * math.pi * np.sum(self.rad ** 3) / self.L ** 3)


def box_side(rad: np.ndarray, phi: float) -> float:
    """Side of the cubic box that holds spheres of radii rad at volume fraction phi."""
    return float((4.0 / 3.0 * math.pi * np.sum(rad ** 3) / phi) ** (1.0 / 3.0))


def radii_lognormal(n: int, mean: float, std: float, rng: np.random.Generator) -> np.ndarray:
    """Log-normal radii whose own mean and standard deviation are (mean, std)."""
    s2 = math.log(1.0 + (std / mean) ** 2)
    mu = math.log(mean) - 0.5 * s2
    return rng.lognormal(mu, math.sqrt(s2), n)


def radii_bidisperse(n: int, a1: float, a2: float, frac2: float, rng: np.random.Generator) -> np.ndarray:
    """n radii, a fraction frac2 (by number) of radius a2, the rest a1, shuffled."""
    n2 = int(round(frac2 * n))
    r = np.concatenate([np.full(n - n2, a1), np.full(n2, a2)])
    rng.shuffle(r)
    return r


def min_gap(pos: np.ndarray, rad: np.ndarray, L: float) -> float:
    """Smallest surface gap r_ij - a_i - a_j over all pairs (periodic)."""
    tree = cKDTree(np.mod(pos, L), boxsize=L)
    pairs = tree.query_pairs(2.0 * rad.max() + 1e-9, output_type="ndarray")
    if len(pairs) == 0:
        return float("inf")
    d = _pair_dist(pos, pairs, L)
    return float(np.min(d - rad[pairs[:, 0]] - rad[pairs[:, 1]]))


def _pair_dist(pos, pairs, L):
    dx = pos[pairs[:, 0]] - pos[pairs[:, 1]]
    dx -= L * np.round(dx / L)
    return np.sqrt(np.sum(dx * dx, axis=1))


def positions_rsa_sheared(rad: np.ndarray, L: float, gamma: float, rng: np.random.Generator,
                          max_tries: int = 5000) -> np.ndarray:
    """Random sequential addition (largest first, brute force: small N) in the periodic
    cell a1 = (L, 0, 0), a2 = (gamma L, L, 0), a3 = (0, 0, L): no sphere overlaps another
    or any periodic image of it (Lees-Edwards minimum image)."""
    n = rad.shape[0]
    order = np.argsort(-rad, kind="stable")
    pos = np.zeros((n, 3))
    placed: list[int] = []
    for idx in order:
        for _ in range(max_tries):
            t = rng.uniform(0.0, 1.0, 3)
            p = L * np.array([t[0] + gamma * t[1], t[1], t[2]])
            if placed:
                d = p - pos[placed]
                ny = np.round(d[:, 1] / L)
                d[:, 1] -= ny * L
                d[:, 0] -= ny * gamma * L
                d[:, 0] -= L * np.round(d[:, 0] / L)
                d[:, 2] -= L * np.round(d[:, 2] / L)
                if np.any(np.sum(d * d, axis=1) < (rad[idx] + rad[placed]) ** 2):
                    continue
            pos[idx] = p
            placed.append(idx)
            break
        else:
            raise RuntimeError("random sequential addition did not place every sphere")
    return pos


def positions_rsa(rad: np.ndarray, L: float, rng: np.random.Generator, max_tries: int = 2000) -> np.ndarray:
    """Random sequential addition (largest first), each sphere uniform in the box
    and rejected while it overlaps an already placed one."""
    n = rad.shape[0]
    order = np.argsort(-rad, kind="stable")
    amax = rad.max()
    cell = 2.0 * amax
    nc = max(1, int(L // cell))
    cs = L / nc
    grid: dict[tuple[int, int, int], list[int]] = {}
    pos = np.zeros((n, 3))
    for idx in order:
        a = rad[idx]
        for _ in range(max_tries):
            p = rng.uniform(0.0, L, 3)
            c = (p // cs).astype(int) % nc
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        key = ((c[0] + dx) % nc, (c[1] + dy) % nc, (c[2] + dz) % nc)
                        for j in grid.get(key, ()):
                            d = p - pos[j]
                            d -= L * np.round(d / L)
                            if d @ d < (a + rad[j]) ** 2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                pos[idx] = p
                grid.setdefault(tuple(c), []).append(idx)
                break
        else:
            raise RuntimeError("RSA failed to place a sphere; volume fraction too high for RSA")
    return pos


def _fcc_sites(n_min: int, L: float) -> np.ndarray:
    m = int(math.ceil((n_min / 4.0) ** (1.0 / 3.0)))
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3)
    sites = (g[:, None, :] + base[None, :, :]).reshape(-1, 3)
    return (sites + 0.25) * (L / m)


def _remove_overlaps(pos, rad, L, max_iter=5000, pad=1e-6, skin=0.3):
    """Relax a soft overlap energy: each overlapping pair is pushed apart along
    its line of centres by a quarter of its overlap per iteration.  Candidate
    pairs come from a Verlet list rebuilt when a sphere has moved skin/2."""
    reach = 2.0 * rad.max() * (1 + pad)
    pairs, ref = None, None
    for _ in range(max_iter):
        if pairs is None or np.max(np.abs(_wrap(pos - ref, L))) > 0.5 * skin / math.sqrt(3.0):
            pairs = cKDTree(pos, boxsize=L).query_pairs(reach + skin, output_type="ndarray")
            ref = pos.copy()
        if len(pairs) == 0:
            return pos, True
        dx = _wrap(pos[pairs[:, 0]] - pos[pairs[:, 1]], L)
        d = np.sqrt(np.sum(dx * dx, axis=1))
        ov = (rad[pairs[:, 0]] + rad[pairs[:, 1]]) * (1 + pad) - d
        m = ov > 0
        if not np.any(m):
            return pos, True
        u = dx[m] / np.maximum(d[m], 1e-12)[:, None]
        push = 0.25 * ov[m][:, None] * u + 1e-7 * u
        np.add.at(pos, pairs[m, 0], push)
        np.add.at(pos, pairs[m, 1], -push)
        pos = np.mod(pos, L)
    return pos, False


def _wrap(dx, L):
    return dx - L * np.round(dx / L)


def _mc_sweeps(pos, rad, L, rng, sweeps, step):
    """Hard-sphere Monte-Carlo: every particle proposes a uniform displacement;
    a move is accepted if the new position overlaps neither the old nor the new
    position of any neighbour (so all accepted moves are mutually compatible)."""
    n = pos.shape[0]
    reach = 2.0 * rad.max() + 2.0 * step * math.sqrt(3.0)
    for _ in range(sweeps):
        new = np.mod(pos + rng.uniform(-step, step, pos.shape), L)
        both = np.concatenate([pos, new])
        tree = cKDTree(both, boxsize=L)
        pairs = tree.query_pairs(reach, output_type="ndarray")
        i, j = pairs[:, 0], pairs[:, 1]
        pi_, pj = i % n, j % n
        d = _pair_dist(both, pairs, L)
        clash = (pi_ != pj) & (d < rad[pi_] + rad[pj]) & ((i >= n) | (j >= n))
        bad = np.zeros(n, dtype=bool)
        bad[pi_[clash & (i >= n)]] = True
        bad[pj[clash & (j >= n)]] = True
        pos = np.where(bad[:, None], pos, new)
    return pos


def positions_dense(rad: np.ndarray, L: float, rng: np.random.Generator, sweeps: int = 10) -> np.ndarray:
    """Non-overlapping positions at any volume fraction below jamming: a random
    subset of FCC lattice sites, radii assigned at random, residual overlaps
    removed, then hard-sphere MC sweeps to randomise."""
    n = rad.shape[0]
    sites = _fcc_sites(n, L)
    pick = rng.choice(sites.shape[0], n, replace=False)
    pos = sites[np.sort(pick)].copy()
    perm = rng.permutation(n)
    a = rad[perm]                      # sphere placed at pos[k] has radius rad[perm[k]]
    d_nn = (L / math.ceil((n / 4.0) ** (1.0 / 3.0))) / math.sqrt(2.0)
    step = max(0.02, 0.25 * (d_nn - 2.0 * a.mean()))
    pos, ok = _remove_overlaps(pos, a, L)
    scale = min(1.0, d_nn / (2.0 * a.max()))
    while not ok:
        # too dense to relax directly: grow the radii from a non-overlapping scale
        pos, ok = _remove_overlaps(pos, a * scale, L)
        if not ok:
            raise RuntimeError("could not relax the configuration; volume fraction too high")
        if scale < 1.0:
            pos = _mc_sweeps(pos, a * scale, L, rng, 1, step)
            scale = min(1.0, scale * 1.02)
            ok = False
    pos = _mc_sweeps(pos, a, L, rng, sweeps, step)
    out = np.empty_like(pos)
    out[perm] = pos
    return out


def moments(n: int, rng: np.random.Generator, ncomp: int = 12) -> np.ndarray:
    """i.i.d. N(0,1) multipoles [n, 12]; components beyond ncomp are zero."""
    x = np.zeros((n, 12))
    x[:, :ncomp] = rng.standard_normal((n, ncomp))
    return x


# ---------------- named workloads ----------------

def mono_n100(seed: int = 0) -> Config:
    rng = np.random.default_rng(seed)
    rad = np.ones(100)
    L = box_side(rad, 0.2)
    return Config("mono_n100", L, positions_rsa(rad, L, rng), rad)


def bidisperse(seed: int = 0, n: int = 2000, phi: float = 0.3) -> Config:
    rng = np.random.default_rng(seed)
    rad = radii_bidisperse(n, 1.0, 2.0, 0.5, rng)
    L = box_side(rad, phi)
    return Config(f"bidisperse_n{n}", L, positions_rsa(rad, L, rng), rad)


def lognormal(seed: int = 0, n: int = 20000, phi: float = 0.4) -> Config:
    rng = np.random.default_rng(seed)
    rad = radii_lognormal(n, 1.0, 0.2, rng)
    L = box_side(rad, phi)
    return Config(f"lognormal_n{n}", L, positions_dense(rad, L, rng), rad)


def mono_dense(seed: int = 0, n: int = 200000, phi: float = 0.45, sweeps: int = 4) -> Config:
    rng = np.random.default_rng(seed)
    rad = np.ones(n)
    L = box_side(rad, phi)
    return Config(f"mono_n{n}", L, positions_dense(rad, L, rng, sweeps=sweeps), rad)


def batch_boxes(seed: int = 0, nbox: int = 64, nmin: int = 500, nmax: int = 8000) -> list[Config]:
    rng = np.random.default_rng(seed)
    out = []
    for b in range(nbox):
        n = int(rng.integers(nmin, nmax + 1))
        phi = float(rng.uniform(0.1, 0.45))
        rad = radii_bidisperse(n, 1.0, 1.5, 0.5, rng)
        L = box_side(rad, phi)
        out.append(Config(f"box{b}_n{n}", L, positions_dense(rad, L, rng, sweeps=4), rad))
    return out
