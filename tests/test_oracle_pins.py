"""Pins of the FP64 direct-Ewald oracle against what the paper and the
mathematics fix (no GPU).  Each test names the passage it relies on.

A plausible mistake anywhere in the oracle (a dropped Faxen term, a wrong sign
or index, a transposed operand, a wrong self term) fails at least one of:
  * Eq. uf-self                  closed-form wave-space self term (paper value)
  * xi-independence              real + wave - self does not depend on xi
  * Hasimoto simple-cubic array  Sec. 6.1 / Eq. dst-corr (1.76 coefficient)
  * symmetry + positive definiteness of the F,T,S block (Sec. 2.1)
  * free-space closed forms      Eq. oseen, Eq. pres-vel-disturb, Eq. pres-funda
  * derivative relations         Eqs. faxen-t, faxen-s, mul-expand (curl/sym-grad/K)
  * compressible special cases   Sec. 2.3 (one-way trace coupling)
"""
import math

import numpy as np
import pytest

from paper_1506_08481_b300 import inputs

PI = math.pi
HASIMOTO_SC = 2.8372974794806   # Hasimoto (1959) simple-cubic lattice constant


def eps():
    e = np.zeros((3, 3, 3))
    e[0, 1, 2] = e[1, 2, 0] = e[2, 0, 1] = 1
    e[0, 2, 1] = e[2, 1, 0] = e[1, 0, 2] = -1
    return e


# ---------------------------------------------------------------- self terms

@pytest.mark.parametrize("a,xi", [(1.0, 0.7), (1.3, 0.4), (0.6, 2.0)])
def test_wave_self_uf_is_eq_uf_self(oracle_mod, a, xi):
    """The self interaction removed from the wave sum, UF block, is Eq. uf-self."""
    B = oracle_mod.pair_block(np.zeros(3), a, a, xi, kind=2)
    ref = xi * (9 - 10 * a * a * xi * xi + 7 * a ** 4 * xi ** 4) / (18 * PI ** 1.5)
    np.testing.assert_allclose(np.diag(B)[:3], ref, rtol=1e-13)
    # translation-rotation and force-stresslet parts vanish at coincidence (parity)
    assert np.abs(B[:3, 3:]).max() < 1e-15 and np.abs(B[3:, :3]).max() < 1e-15


# ---------------------------------------------------------------- Ewald split

def test_xi_independence_all_components(oracle_mod):
    """Real + wave - self is independent of the splitting parameter (Eq. oseen-split):
    pins every real-space, wave-space and self term, including the trace terms."""
    rng = np.random.default_rng(1)
    N, L = 6, 8.0
    pos = rng.uniform(0, L, (N, 3))
    rad = rng.uniform(0.5, 1.2, N)
    x = rng.standard_normal((N, 12))
    ys = [oracle_mod.mobility(pos, rad, L, x, xi=xi, tol=1e-15) for xi in (0.45, 0.9, 1.8)]
    scale = np.abs(ys[0]).max(axis=0)
    for y in ys[1:]:
        assert (np.abs(y - ys[0]) / scale).max() < 1e-12


def test_xi_independence_single_particle_images(oracle_mod):
    """N=1: only periodic images; xi-independence pins the self-removal of every block."""
    x = np.random.default_rng(2).standard_normal((1, 12))
    ys = [oracle_mod.mobility(np.array([[0.3, 1.1, 2.0]]), np.array([1.4]), 6.0, x, xi=xi, tol=1e-15)
          for xi in (0.4, 0.8, 1.4)]
    for y in ys[1:]:
        np.testing.assert_allclose(y, ys[0], rtol=1e-11, atol=1e-14)


# ---------------------------------------------------------------- lattice sums

@pytest.mark.parametrize("L", [4.0, 6.0, 10.0, 25.0])
def test_hasimoto_simple_cubic_array(oracle_mod, L):
    """A simple cubic array of spheres (N=1 periodic): Hasimoto's drag correction
    6 pi eta a M^UF = 1 - 2.837297 a/L + (4 pi/3)(a/L)^3 (the a^2 Faxen terms give the
    last term); rotation 8 pi eta a^3 M^OT = 1 - phi.  Sec. 6.1 states SEASD reproduces
    the simple-cubic results and Eq. dst-corr quotes 1.76 = 2.837297 (3/(4 pi))^(1/3)."""
    a = 1.0
    phi = 4 * PI / 3 * (a / L) ** 3
    cols = []
    for c in range(12):
        X = np.zeros((1, 12))
        X[0, c] = 1.0
        cols.append(oracle_mod.mobility(np.zeros((1, 3)), np.array([a]), L, X)[0])
    M = np.array(cols).T
    np.testing.assert_allclose(6 * PI * a * np.diag(M)[:3], 1 - HASIMOTO_SC * a / L + phi, rtol=1e-12)
    np.testing.assert_allclose(8 * PI * a ** 3 * np.diag(M)[3:6], 1 - phi, rtol=1e-12)
    # inversion symmetry of the lattice: UT, US, OS (and transposes) vanish
    assert np.abs(M[:6, 6:11]).max() < 1e-13 and np.abs(M[:3, 3:6]).max() < 1e-13
    # the pressure moment couples only to itself for a single sphere
    assert abs(M[11, 11] * 16 * PI * a ** 3 / 3 - 1) < 1e-13
    assert np.abs(M[11, :11]).max() < 1e-13 and np.abs(M[:11, 11]).max() < 1e-13


def test_paper_coefficient_1p76():
    """Eq. dst-corr: 1.76 is Hasimoto's constant times (3/(4 pi))^(1/3)."""
    assert abs(HASIMOTO_SC * (3 / (4 * PI)) ** (1 / 3) - 1.76) < 5e-3


def test_isolated_sphere_limit(oracle_mod):
    """L -> infinity: the periodic self mobilities tend to the isolated-sphere values of
    Eqs. faxen-f/t/s/p, with the lattice correction shrinking like a/L (translation) and
    (a/L)^3 (rotation, strain, pressure moment)."""
    a = 0.8
    errs = []
    for L in (20.0, 40.0, 80.0):
        X = np.eye(12)
        y = np.array([oracle_mod.mobility(np.zeros((1, 3)), np.array([a]), L, X[c:c + 1])[0] for c in range(12)]).T
        d = np.diag(y)
        iso = np.r_[np.full(3, 1 / (6 * PI * a)), np.full(3, 1 / (8 * PI * a ** 3)),
                    np.full(5, 3 / (20 * PI * a ** 3)), 3 / (16 * PI * a ** 3)]
        rel = np.abs(d / iso - 1)
        errs.append(rel)
        assert rel[:3].max() < 3.0 * a / L and rel[3:].max() < 20.0 * (a / L) ** 3
    # translation correction halves, the others shrink 8x, when L doubles
    assert 1.9 < errs[0][0] / errs[1][0] < 2.1
    assert np.all((7.5 < errs[1][3:11] / errs[2][3:11]) & (errs[1][3:11] / errs[2][3:11] < 8.5))


# ---------------------------------------------------------------- SPD of F,T,S block

def test_fts_block_symmetric_positive_definite(oracle_mod):
    """The grand mobility restricted to F,T,S is symmetric positive definite
    (Sec. 2.1, Lorentz reciprocal theorem) for non-overlapping spheres."""
    rng = np.random.default_rng(3)
    rad = inputs.radii_bidisperse(8, 1.0, 1.6, 0.5, rng)
    L = inputs.box_side(rad, 0.15)
    pos = inputs.positions_rsa(rad, L, rng)
    M = oracle_mod.dense_matrix(pos, rad, L, ncomp=11, tol=1e-14)
    assert np.abs(M - M.T).max() / np.abs(M).max() < 1e-12
    np.linalg.cholesky(0.5 * (M + M.T))
    # the compressible (trace) coupling is one-way, hence non-symmetric (Sec. 2.3)
    M12 = oracle_mod.dense_matrix(pos, rad, L, ncomp=12, tol=1e-14)
    assert np.abs(M12 - M12.T).max() / np.abs(M12).max() > 1e-3


# ---------------------------------------------------------------- free space

def _free(oracle_mod, x, ai, aj):
    return oracle_mod.pair_block(np.asarray(x, float), ai, aj, kind=1)


def test_free_space_closed_forms(oracle_mod):
    """Free-space pair couplings (psi = r, phi = 1/r): polydisperse Rotne-Prager
    translation (Eq. faxen-f with Eq. mul-expand, Eq. oseen), rotlet, rotation-rotation,
    source velocity Q (Eq. pres-vel-disturb) and the pressure of a force and of a
    stresslet (Eqs. pres-funda, pres-multi-expans, faxen-p)."""
    rng = np.random.default_rng(4)
    e = eps()
    Y = np.array([[[1, 0, 0], [0, -1, 0], [0, 0, 0]],
                  [[-1, 0, 0], [0, -1, 0], [0, 0, 2]],
                  [[0, 1, 0], [1, 0, 0], [0, 0, 0]],
                  [[0, 0, 1], [0, 0, 0], [1, 0, 0]],
                  [[0, 0, 0], [0, 0, 1], [0, 1, 0]]], float)
    Y /= np.sqrt((Y * Y).sum(axis=(1, 2)))[:, None, None]
    np.testing.assert_allclose(oracle_mod.stresslet_basis(), Y, atol=1e-15)
    for _ in range(5):
        x = rng.standard_normal(3) * 3
        r = np.linalg.norm(x)
        xh = x / r
        ai, aj = rng.uniform(0.3, 1.0, 2)
        B = _free(oracle_mod, x, ai, aj)
        s = ai * ai + aj * aj
        UF = ((1 + s / (3 * r * r)) * np.eye(3) + (1 - s / (r * r)) * np.outer(xh, xh)) / (8 * PI * r)
        np.testing.assert_allclose(B[:3, :3], UF, rtol=1e-12, atol=1e-15)
        UT = np.einsum("abg,g->ab", e, x) / (8 * PI * r ** 3)          # (T x x)/r^3
        np.testing.assert_allclose(B[:3, 3:6], UT, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(B[3:6, :3], UT, rtol=1e-12, atol=1e-15)  # (F x x)/r^3
        OT = (3 * np.outer(xh, xh) - np.eye(3)) / (16 * PI * r ** 3)
        np.testing.assert_allclose(B[3:6, 3:6], OT, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(B[:3, 11], x / (16 * PI * r ** 3), rtol=1e-12)
        np.testing.assert_allclose(B[11, :3], 3 * x / (16 * PI * r ** 3), rtol=1e-12)
        xSx = np.einsum("a,mab,b->m", x, Y, x)
        np.testing.assert_allclose(B[11, 6:11], 9 * xSx / (16 * PI * r ** 5), rtol=1e-12, atol=1e-16)
        assert abs(B[11, 11]) == 0 and np.abs(B[11, 3:6]).max() == 0 and np.abs(B[3:6, 11]).max() < 1e-16
        # stresslet velocity for point particles: 3 x (x.S.x)/(8 pi r^5)
        B0 = _free(oracle_mod, x, 0.0, 0.0)
        np.testing.assert_allclose(B0[:3, 6:11], 3 * np.outer(x, xSx) / (8 * PI * r ** 5), rtol=1e-12, atol=1e-16)


def _fd_grad(f, x, h):
    """Central difference d f / d x_mu, returns [3, ...]."""
    out = []
    for mu in range(3):
        d = np.zeros(3)
        d[mu] = h
        out.append((f(x + d) - f(x - d)) / (2 * h))
    return np.array(out)


def _fd_lap(f, x, h):
    out = -6 * f(x)
    for mu in range(3):
        d = np.zeros(3)
        d[mu] = h
        out = out + f(x + d) + f(x - d)
    return out / (h * h)


@pytest.mark.parametrize("kind", [1, 0])
def test_target_rows_are_faxen_derivatives_of_velocity(oracle_mod, kind):
    """Omega = 1/2 curl v (Eq. faxen-t) and E = (1 + a^2 Lap/10) sym grad v (Eq. faxen-s),
    U = (1 + a^2 Lap/6) v (Eq. faxen-f): the Omega and E rows of every column equal
    finite-difference derivatives of the point-target U row (free space and the
    real-space Ewald part)."""
    rng = np.random.default_rng(5)
    e = eps()
    Y = oracle_mod.stresslet_basis()
    for _ in range(3):
        x = rng.standard_normal(3)
        x *= 2.5 / np.linalg.norm(x)
        ai, aj = rng.uniform(0.4, 0.9, 2)
        v = lambda p: oracle_mod.pair_block(p, 0.0, aj, 0.9, kind=kind)[:3, :]
        G = _fd_grad(v, x, 1e-4)                         # G[mu, n, col] = d_mu v_n
        B = oracle_mod.pair_block(x, 0.0, aj, 0.9, kind=kind)
        Om = 0.5 * np.einsum("amn,mnc->ac", e, G)
        np.testing.assert_allclose(B[3:6], Om, rtol=1e-6, atol=1e-9)
        E = np.einsum("kmn,mnc->kc", Y, G)
        np.testing.assert_allclose(B[6:11], E, rtol=1e-6, atol=1e-9)
        # Faxen Laplacian at the target
        Bi = oracle_mod.pair_block(x, ai, aj, 0.9, kind=kind)
        lapv = _fd_lap(v, x, 2e-3)
        np.testing.assert_allclose(Bi[:3], B[:3] + ai * ai / 6 * lapv, rtol=1e-5, atol=1e-8)
        lapE = _fd_lap(lambda p: oracle_mod.pair_block(p, 0.0, aj, 0.9, kind=kind)[6:11], x, 2e-3)
        np.testing.assert_allclose(Bi[6:11], B[6:11] + ai * ai / 10 * lapE, rtol=1e-5, atol=1e-8)


def test_source_columns_are_multipoles_of_the_stokeslet(oracle_mod):
    """Eq. mul-expand with R and K as defined after it: for a point source,
    the torque column is 1/2 curl (field point) of the Stokeslet column and the
    stresslet column is the symmetric source-point gradient of the Stokeslet column;
    the source Faxen factors are (1 + a_j^2 Lap/6) on F and (1 + a_j^2 Lap/10) on S."""
    rng = np.random.default_rng(6)
    e = eps()
    Y = oracle_mod.stresslet_basis()
    for _ in range(3):
        x = rng.standard_normal(3)
        x *= 2.2 / np.linalg.norm(x)
        aj = rng.uniform(0.4, 0.9)
        uF = lambda p: oracle_mod.pair_block(p, 0.0, 0.0, kind=1)[:3, :3]
        B = oracle_mod.pair_block(x, 0.0, 0.0, kind=1)
        G = _fd_grad(uF, x, 1e-4)                        # d_mu (field) of U<-F[n, b]
        UT = 0.5 * np.einsum("amn,mnb->ab", e, G)
        np.testing.assert_allclose(B[:3, 3:6], UT, rtol=1e-6, atol=1e-9)
        # source displacement = -field displacement
        US = -np.einsum("kbg,gab->ak", Y, G)
        np.testing.assert_allclose(B[:3, 6:11], US, rtol=1e-6, atol=1e-9)
        Bj = oracle_mod.pair_block(x, 0.0, aj, kind=1)
        lapF = _fd_lap(uF, x, 2e-3)
        np.testing.assert_allclose(Bj[:3, :3], B[:3, :3] + aj * aj / 6 * lapF, rtol=1e-5, atol=1e-8)
        lapS = _fd_lap(lambda p: oracle_mod.pair_block(p, 0.0, 0.0, kind=1)[:3, 6:11], x, 2e-3)
        np.testing.assert_allclose(Bj[:3, 6:11], B[:3, 6:11] + aj * aj / 10 * lapS, rtol=1e-5, atol=1e-8)


def test_periodic_pair_tends_to_free_space(oracle_mod):
    """Two spheres in ever larger boxes: the periodic coupling tends to the free-space
    pair coupling plus the image correction, which shrinks like 1/L."""
    x = np.array([1.7, -2.1, 2.6])
    ai, aj = 0.7, 1.1
    free = _free(oracle_mod, x, ai, aj)
    prev = None
    for L in (30.0, 60.0, 120.0):
        pos = np.array([[0, 0, 0], -x]) + L / 2
        rad = np.array([ai, aj])
        cols = []
        for c in range(12):
            X = np.zeros((2, 12))
            X[1, c] = 1.0
            cols.append(oracle_mod.mobility(pos, rad, L, X, rows=np.array([0]))[0])
        M = np.array(cols).T
        dev = np.abs(M - free).max() / np.abs(free).max()
        if prev is not None:
            assert 1.8 < prev / dev < 2.2
        prev = dev
    assert prev < 0.15


# ---------------------------------------------------------------- compressible terms

def test_compressible_one_way_coupling(oracle_mod):
    """Sec. 2.3: a pressure moment moves other spheres (U, E) but gives no rotation and
    no pressure disturbance; E_tr is driven by forces and stresslets only."""
    rng = np.random.default_rng(7)
    rad = rng.uniform(0.5, 1.0, 5)
    L = 9.0
    pos = rng.uniform(0, L, (5, 3))
    X = np.zeros((5, 12))
    X[:, 11] = rng.standard_normal(5)
    y = oracle_mod.mobility(pos, rad, L, X)
    assert np.abs(y[:, 3:6]).max() < 1e-15                       # Omega <- S_tr
    np.testing.assert_allclose(y[:, 11], 3 * X[:, 11] / (16 * PI * rad ** 3), rtol=1e-13)
    assert np.abs(y[:, :3]).max() > 1e-4 and np.abs(y[:, 6:11]).max() > 1e-4
    X = np.zeros((5, 12))
    X[:, 3:6] = rng.standard_normal((5, 3))
    y = oracle_mod.mobility(pos, rad, L, X)
    assert np.abs(y[:, 11]).max() < 1e-15                        # E_tr <- T


@pytest.mark.parametrize("gamma", [0.3, -0.5])
def test_sheared_lattice_xi_independence(oracle_mod, gamma):
    """On the sheared lattice a2 = (gamma L, L, 0) (Sec. 3.2) the split into real-space
    images and reciprocal-lattice waves leaves the sum independent of xi."""
    from paper_1506_08481_b300 import inputs
    rng = np.random.default_rng(3)
    rad = rng.uniform(0.6, 1.0, 6)
    L = 8.0
    pos = inputs.positions_rsa(rad, L, rng)
    x = rng.standard_normal((6, 12))
    ys = [oracle_mod.mobility(pos, rad, L, x, xi=xi, tol=1e-13, gamma=gamma) for xi in (0.5, 0.9, 1.4)]
    for y in ys[1:]:
        assert np.abs(y - ys[0]).max() <= 1e-12 * np.abs(ys[0]).max()


def test_sheared_lattice_periodic_in_the_strain(oracle_mod):
    """Strains gamma and gamma - 1 give the same lattice (a2 - a1), hence the same
    mobility; gamma = 0 is another lattice and another mobility; the F, T, S block stays
    symmetric positive definite."""
    from paper_1506_08481_b300 import inputs
    rng = np.random.default_rng(4)
    rad = rng.uniform(0.6, 1.0, 5)
    L = 7.5
    pos = inputs.positions_rsa(rad, L, rng)
    x = rng.standard_normal((5, 12))
    y1 = oracle_mod.mobility(pos, rad, L, x, tol=1e-13, gamma=0.2)
    y2 = oracle_mod.mobility(pos, rad, L, x, tol=1e-13, gamma=-0.8)
    y0 = oracle_mod.mobility(pos, rad, L, x, tol=1e-13, gamma=0.0)
    assert np.abs(y1 - y2).max() <= 1e-12 * np.abs(y1).max()
    assert np.abs(y1 - y0).max() > 1e-4 * np.abs(y1).max()
    A = oracle_mod.dense_matrix(pos, rad, L, ncomp=11, tol=1e-12, gamma=0.4)
    assert np.abs(A - A.T).max() <= 1e-10 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
