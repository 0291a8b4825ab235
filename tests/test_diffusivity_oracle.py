"""Pins of oracle/diffusivity.py (rigid-particle far-field mobility and the self-diffusivity
estimator of Sec. 6.1, Eq. dstr-def) against closed forms and identities: the simple
cubic array (Hasimoto's drag; no stresslet by symmetry), the Schur-complement form of mu,
positive definiteness and the Loewner bound mu <= M_FT,FT (rigidity can only reduce the
mobility), and the estimator's convergence to diag(mu)."""
import math

import numpy as np

from oracle import diffusivity


def test_simple_cubic_array(oracle_mod):
    """One sphere per cubic cell: 6 pi eta a mu^tt = 1 - 2.837297 a/L + (4 pi/3)(a/L)^3 + O((a/L)^6)
    (Hasimoto), and the translation induces no stresslet (inversion symmetry of the lattice)."""
    a, L = 1.0, 12.0
    M = oracle_mod.dense_matrix(np.array([[3.0, 4.0, 5.0]]), np.array([a]), L, ncomp=11, tol=1e-13)
    mu = diffusivity.rigid_mobility(M)
    x = a / L
    np.testing.assert_allclose(6 * math.pi * mu[0, 0], 1 - 2.837297 * x + 4 * math.pi / 3 * x ** 3, rtol=0, atol=2e-5)
    np.testing.assert_allclose(mu[:3, :3], mu[0, 0] * np.eye(3), atol=1e-12)
    uw, s = diffusivity.rigid_response(M, np.array([[1.0, -2.0, 0.5, 0.0, 0.0, 0.0]]))
    assert np.abs(s).max() < 1e-12


def test_schur_complement_and_bounds(oracle_mod):
    from paper_1506_08481_b300 import inputs
    cfg = inputs.lognormal(seed=4, n=10, phi=0.3)
    M = oracle_mod.dense_matrix(cfg.pos, cfg.rad, cfg.L, ncomp=11, tol=1e-13)
    mu = diffusivity.rigid_mobility(M)
    N = cfg.N
    ft = diffusivity._ft_index(N)
    si = diffusivity._s_index(N)
    schur = M[np.ix_(ft, ft)] - M[np.ix_(ft, si)] @ np.linalg.solve(M[np.ix_(si, si)], M[np.ix_(si, ft)])
    np.testing.assert_allclose(mu, schur, rtol=1e-9, atol=1e-12)
    assert np.linalg.eigvalsh(0.5 * (mu + mu.T)).min() > 0
    assert np.linalg.eigvalsh(M[np.ix_(ft, ft)] - mu).min() > -1e-12
    # the response: (U, Omega) and S satisfy the grand-mobility rows with E = 0
    f = np.random.default_rng(0).standard_normal((N, 6))
    uw, s = diffusivity.rigid_response(M, f)
    x = np.zeros((N, 11))
    x[:, :6], x[:, 6:] = f, s
    y = (M @ x.reshape(-1)).reshape(N, 11)
    np.testing.assert_allclose(y[:, :6], uw, rtol=1e-9, atol=1e-12)
    assert np.abs(y[:, 6:]).max() < 1e-9 * np.abs(y[:, :6]).max()


def test_estimator_converges_to_the_diagonal(oracle_mod):
    from paper_1506_08481_b300 import inputs
    cfg = inputs.lognormal(seed=6, n=6, phi=0.25)
    M = oracle_mod.dense_matrix(cfg.pos, cfg.rad, cfg.L, ncomp=11, tol=1e-12)
    mu = diffusivity.rigid_mobility(M)
    exact = diffusivity.diag_traces(mu)
    fr = np.random.default_rng(1).standard_normal((20000, cfg.N, 6))
    est = diffusivity.estimate(mu, fr)
    # each estimate is a mean of 20000 quadratic forms: standard error ~ |mu_i| sqrt(2/3) / sqrt(20000)
    scale = np.abs(mu).max()
    assert np.abs(est - exact).max() < 6 * scale * math.sqrt(2 / 3) / math.sqrt(20000)


def test_viscosity_dilute_limit_is_einstein(oracle_mod):
    """A single sphere in a large periodic cell: eta_s / eta = 1 + 5 phi / 2 + O(phi^2)
    (Einstein; the isolated rigid sphere's stresslet (20/3) pi eta a^3 E)."""
    a = 1.0
    for L in (20.0, 40.0):
        M = oracle_mod.dense_matrix(np.array([[1.0, 2.0, 3.0]]), np.array([a]), L, ncomp=11, tol=1e-13)
        phi = 4 * math.pi / 3 * a ** 3 / L ** 3
        r = diffusivity.viscosity_ratio(M, L)
        assert abs(r - 1 - 2.5 * phi) < 10 * phi ** 2, (L, r, phi)
    # the five basis strains give the same value for a cubic lattice, and the
    # rigid spheres do not move
    M = oracle_mod.dense_matrix(np.array([[1.0, 2.0, 3.0]]), np.array([a]), 20.0, ncomp=11, tol=1e-13)
    uw, s = diffusivity.rigid_response_strain(M, np.array([0.0, 0.0, 1.0, 0.0, 0.0]))
    assert np.abs(uw).max() < 1e-12
    np.testing.assert_allclose(s[0, 2], 20 * math.pi / 3 * a ** 3 * (1 + 0.0), rtol=2e-3)
