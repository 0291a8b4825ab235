"""FP64 direct-Ewald oracle for the periodic far-field grand mobility
(Wang & Brady, arXiv 1506.08481, Secs. 2.1-2.3 and Eq. uf-self).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_1506_08481_b300``) and imports nothing from it.

The arithmetic lives in ``se_oracle.c`` (plain C, FP64, OpenMP over target
particles / wave vectors).  This module only compiles it with gcc, loads it with
ctypes and picks the Ewald parameter xi and the cutoffs for a requested accuracy;
the result does not depend on xi.

Parity status of each function (pins live in ``tests/test_oracle_pins.py``):
  mobility()      pinned: xi-independence (also on sheared lattices), identity of
                  the lattices at strain gamma and gamma - 1, isolated-sphere limit, Hasimoto
                  simple-cubic drag (Sec. 6.1, Eq. dst-corr), Eq. uf-self,
                  symmetry and positive definiteness of the F,T,S block,
                  free-space limits, compressible-term special cases.
  pair_block()    pinned: free-space closed forms, finite-difference relations
                  between blocks.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "se_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libse_oracle.so")
_lib = None

NCOMP = 12
PARTS_REAL, PARTS_WAVE, PARTS_SELF, PARTS_ALL = 1, 2, 4, 7


def build(force: bool = False) -> str:
    """Compile se_oracle.c into libse_oracle.so next to it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        d, l, i = ctypes.c_double, ctypes.c_long, ctypes.c_int
        p = ctypes.c_void_p
        lib.se_oracle_mobility.argtypes = [l, d, p, p, p, p, l, p, d, d, d, i, d]
        lib.se_oracle_mobility.restype = i
        lib.se_oracle_mobility_sheared.argtypes = [l, d, d, p, p, p, p, l, p, d, d, d, i, d]
        lib.se_oracle_mobility_sheared.restype = i
        lib.se_oracle_pair_block.argtypes = [p, d, d, d, i, d, p]
        lib.se_oracle_pair_block.restype = i
        lib.se_oracle_stresslet_basis.argtypes = [p]
        lib.se_oracle_num_threads.restype = i
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads() -> int:
    return int(_load().se_oracle_num_threads())


def stresslet_basis() -> np.ndarray:
    """The orthonormal traceless-symmetric basis Y[m, a, b] used for S and E."""
    out = np.zeros(45)
    _load().se_oracle_stresslet_basis(_ptr(out))
    return out.reshape(5, 3, 3)


def cutoffs(xi: float, tol: float) -> tuple[float, float]:
    """Real-space cutoff rc and wave cutoff kc for relative truncation ~tol.

    Both series decay like exp(-(xi r)^2) and exp(-k^2/(4 xi^2)) (Eqs.
    oseen-ewald-rs/ws); a margin covers the polynomial prefactors of the
    high-order derivative terms.
    """
    c = math.sqrt(-math.log(tol)) + 1.5
    return c / xi, 2.0 * c * xi


def choose_xi(N: int, L: float, nrows: int, tol: float) -> float:
    """xi that minimises the estimated oracle cost (real ~ pairs, wave ~ k-vectors)."""
    best = None
    V = L ** 3
    for xi in np.geomspace(0.02, 5.0, 200):
        rc, kc = cutoffs(xi, tol)
        pairs = nrows * N * (4.0 / 3.0 * math.pi * rc ** 3) / V + nrows
        nk = 0.5 * 4.0 / 3.0 * math.pi * (kc * L / (2 * math.pi)) ** 3
        cost = 2.0e4 * pairs + nk * (40.0 * N + 300.0 * nrows)
        if best is None or cost < best[0]:
            best = (cost, float(xi))
    return best[1]


def mobility(pos, rad, L, x, rows=None, xi=None, tol=1e-13, parts=PARTS_ALL,
             eta=1.0, rc=None, kc=None, gamma=0.0):
    """y = M_inf . x for the listed target rows (all particles if rows is None).

    pos [N,3], rad [N], x [N,12] = [F, T, S(5 on the orthonormal basis), S_tr].
    gamma: strain of the sheared lattice a2 = (gamma L, L, 0) (0: the cubic box).
    Returns y [nrows, 12] = [U, Omega, E(5), E_tr].
    """
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    rad = np.ascontiguousarray(rad, dtype=np.float64).reshape(-1)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, NCOMP)
    N = pos.shape[0]
    if rad.shape[0] != N or x.shape[0] != N:
        raise ValueError("pos, rad and x must describe the same N particles")
    if rows is not None:
        rows = np.ascontiguousarray(rows, dtype=np.int64).reshape(-1)
        nrows = rows.shape[0]
    else:
        nrows = N
    if xi is None:
        xi = choose_xi(N, L, nrows, tol)
    rc0, kc0 = cutoffs(xi, tol)
    rc = rc0 if rc is None else rc
    kc = kc0 if kc is None else kc
    y = np.zeros((nrows, NCOMP))
    rc_ = lib.se_oracle_mobility_sheared(N, float(L), float(gamma), _ptr(pos), _ptr(rad), _ptr(x), _ptr(rows),
                                         nrows, _ptr(y), float(xi), float(rc), float(kc), int(parts),
                                         float(eta))
    if rc_ != 0:
        raise RuntimeError(f"se_oracle_mobility failed with code {rc_}")
    return y


def pair_block(x, ai, aj, xi=1.0, kind=0, eta=1.0):
    """12x12 pair block (rows: U,Omega,E(5),E_tr; columns: F,T,S(5),S_tr).

    kind 0: real-space Ewald part, 1: free space, 2: wave-space self remainder at x = 0.
    """
    lib = _load()
    xv = np.ascontiguousarray(x, dtype=np.float64).reshape(3)
    out = np.zeros(NCOMP * NCOMP)
    r = lib.se_oracle_pair_block(_ptr(xv), float(ai), float(aj), float(xi), int(kind), float(eta), _ptr(out))
    if r != 0:
        raise ValueError("invalid pair_block arguments")
    return out.reshape(NCOMP, NCOMP)


def dense_matrix(pos, rad, L, ncomp=NCOMP, **kw):
    """Dense (N*ncomp)^2 matrix of M_inf restricted to the first ncomp components."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    N = pos.shape[0]
    n = N * ncomp
    Mat = np.zeros((n, n))
    X = np.zeros((N, NCOMP))
    for col in range(n):
        X[:] = 0.0
        X[col // ncomp, col % ncomp] = 1.0
        Mat[:, col] = mobility(pos, rad, L, X, **kw)[:, :ncomp].reshape(-1)
    return Mat
