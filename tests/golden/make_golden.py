"""Writes the stored oracle values used by the full-size parity tests and the bench.

Run from the repository root:  python tests/golden/make_golden.py
Every expected value comes from the FP64 direct-Ewald oracle (oracle/), evaluated on
sampled output rows of the seeded synthetic workloads; the positions' checksum is
stored so a consumer can verify it regenerated the same configuration.
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1506_08481_b300 import inputs  # noqa: E402

OUT = os.path.dirname(os.path.abspath(__file__))


def checksum(a):
    return float(np.sum(a * np.arange(1, a.size + 1).reshape(a.shape) % 97))


def mono_n200k(nrows=1000):
    cfg = inputs.mono_dense(seed=0, n=200000, phi=0.45)
    x = inputs.moments(cfg.N, np.random.default_rng(1), 12)
    rows = np.sort(np.random.default_rng(2).choice(cfg.N, nrows, replace=False))
    t = time.time()
    y = oracle.mobility(cfg.pos, cfg.rad, cfg.L, x, rows=rows, tol=1e-11)
    print(f"mono_n200k: {nrows} rows in {time.time() - t:.1f} s on {oracle.num_threads()} threads")
    np.savez(os.path.join(OUT, "mono_n200k_rows.npz"), rows=rows, y=y, L=cfg.L,
             pos_checksum=checksum(cfg.pos), x_checksum=checksum(x))


if __name__ == "__main__":
    oracle.build()
    mono_n200k()
