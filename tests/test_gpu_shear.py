"""Sheared periodic cells (SE_OPT_SHEAR; the cell a1 = (L, 0, 0), a2 = (gamma L, L, 0),
a3 = (0, 0, L) of Sec. 3.2, with the wave-space size approach) against the FP64 oracle on
the same lattice (oracle.mobility(..., gamma)): the product in FP64 (<= 1e-9) and FP32
(<= 1e-6), the identity of strains 1/2 and -1/2 (the same lattice), positions given in
any periodic image, and block-preconditioned, spectral and learned solves."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1506_08481_b300 import api, inputs  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def ctx_for(cfg, gamma, precision, M=64, P=24, xi=1.0, rc=5.45, size_mode=2):
    c = api.Context()
    c.set_params(xi, M, P, rc)
    c.set_option(api.SE_OPT_SIZE_MODE, size_mode)
    c.set_option(api.SE_OPT_SHEAR, gamma)
    c.set_option(api.SE_OPT_PRECISION, precision)
    c.set_config(cfg.pos, cfg.rad, cfg.L)
    return c


@pytest.fixture(scope="module")
def poly():
    """N = 37 radii 0.5..1 in L = 11, placed without overlap on every lattice used below
    (strains 0.5, -0.3, 0.2; 0.5 and -0.5 are one lattice)."""
    rng = np.random.default_rng(11)
    rad = rng.uniform(0.5, 1.0, 37)
    L = 11.0
    for _ in range(50):
        pos = inputs.positions_rsa_sheared(rad, L, 0.5, rng)
        if all(_min_gap(pos, rad, L, g) > 0 for g in (-0.3, 0.2, 0.3)):
            break
    x = rng.standard_normal((37, 12))
    return inputs.Config("small_poly", L, pos, rad), x


def _min_gap(pos, rad, L, g):
    d = pos[:, None, :] - pos[None, :, :]
    ny = np.round(d[..., 1] / L)
    d[..., 1] -= ny * L
    d[..., 0] -= ny * g * L
    d[..., 0] -= L * np.round(d[..., 0] / L)
    d[..., 2] -= L * np.round(d[..., 2] / L)
    r = np.sqrt((d ** 2).sum(-1)) - rad[:, None] - rad[None, :]
    np.fill_diagonal(r, np.inf)
    return r.min()


@pytest.mark.parametrize("size_mode", [2, 3])
@pytest.mark.parametrize("gamma", [0.5, -0.3, 0.2])
def test_sheared_product_vs_oracle(oracle_mod, poly, gamma, size_mode):
    """Both wave-space size approaches on the sheared lattice: mode 2 (the window's
    gradients along the sheared directions in the spread and gather) and mode 3 (every
    derivative in k-space with the sheared reciprocal lattice)."""
    cfg, x = poly
    ref = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x, tol=1e-15, gamma=gamma)
    y = ctx_for(cfg, gamma, 1, size_mode=size_mode).apply(torch.tensor(x, device="cuda")).cpu().numpy()
    for sl in (slice(0, 3), slice(3, 6), slice(6, 11), slice(11, 12)):
        assert rel(y[:, sl], ref[:, sl]) <= 1e-9, (gamma, sl)
    y32 = ctx_for(cfg, gamma, 0, M=48, P=16, xi=0.9, rc=5.4, size_mode=size_mode).apply(
        torch.tensor(x, device="cuda", dtype=torch.float32)).double().cpu().numpy()
    assert rel(y32, ref) <= 1e-6
    # the sheared cell changes the result (the test would pass trivially otherwise)
    ref0 = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x, tol=1e-13)
    assert rel(ref0, ref) > 1e-4


def test_half_strains_are_the_same_lattice(poly):
    """a2 = (L/2, L, 0) and (-L/2, L, 0) differ by a1: the same periodic suspension, on
    different grids of fractional coordinates."""
    cfg, x = poly
    xt = torch.tensor(x, device="cuda")
    y1 = ctx_for(cfg, 0.5, 1).apply(xt).cpu().numpy()
    y2 = ctx_for(cfg, -0.5, 1).apply(xt).cpu().numpy()
    assert rel(y1, y2) <= 1e-9


def test_positions_in_any_image(poly):
    cfg, x = poly
    g = 0.2
    shift = np.random.default_rng(2).integers(-2, 3, (cfg.N, 3))
    a = np.array([[cfg.L, 0, 0], [g * cfg.L, cfg.L, 0], [0, 0, cfg.L]])
    moved = inputs.Config("moved", cfg.L, cfg.pos + shift @ a, cfg.rad)
    xt = torch.tensor(x, device="cuda")
    y1 = ctx_for(cfg, g, 1).apply(xt).cpu().numpy()
    y2 = ctx_for(moved, g, 1).apply(xt).cpu().numpy()
    assert rel(y2, y1) <= 1e-12


def test_sheared_solve(oracle_mod):
    rng = np.random.default_rng(21)
    g = 0.4
    rad = rng.uniform(0.8, 1.2, 30)
    L = (4 / 3 * np.pi * np.sum(rad ** 3) / 0.25) ** (1 / 3)
    cfg = inputs.Config("sheared", L, inputs.positions_rsa_sheared(rad, L, g, rng), rad)
    A = oracle_mod.dense_matrix(cfg.pos, cfg.rad, cfg.L, ncomp=11, tol=1e-13, gamma=g)
    b = np.random.default_rng(5).standard_normal((cfg.N, 11))
    x_or = np.linalg.solve(A, b.reshape(-1))
    from paper_1506_08481_b300 import params
    sp = params.choose(cfg.L, cfg.N, 1e-11, M_max=64, a_eff=params.effective_radius(cfg.rad))
    c = api.Context()
    c.set_params(sp.xi, sp.M, sp.P, min(sp.rc, 0.45 * cfg.L))
    c.set_option(api.SE_OPT_SHAPE_M, sp.m)
    c.set_option(api.SE_OPT_SIZE_MODE, 2)
    c.set_option(api.SE_OPT_SHEAR, g)
    c.set_option(api.SE_OPT_PRECISION, 1)
    c.set_config(cfg.pos, cfg.rad, cfg.L)
    x, iters, relres = c.solve(torch.tensor(b, device="cuda"), rtol=1e-11, maxit=400,
                               precond=api.SE_PRECOND_BLOCK)
    assert relres <= 1e-11
    assert rel(x.cpu().numpy().reshape(-1), x_or) <= 1e-7
    print(f"sheared solve: {iters} products")


def test_sheared_spectral_and_learned_solves():
    """The long-wavelength (spectral) correction of the block preconditioner on a sheared cell:
    its plane waves are those of the sheared reciprocal lattice, k = (2 pi / L)(q1, q2 - gamma q1,
    q3), in the probes and in the coarse correction product.  At gamma = 0.3 (N = 2000, radii
    0.8-1.2, phi = 0.3, FP32 products with double-float residuals): the spectral and learned
    solves reach the tolerance with fewer products than the block one and agree with its
    solution to the conditioning of the residual tolerance."""
    import os
    from paper_1506_08481_b300 import params
    rng = np.random.default_rng(31)
    g = 0.3
    rad = rng.uniform(0.8, 1.2, 2000)
    L = inputs.box_side(rad, 0.3)
    cfg = inputs.Config("sheared_n2000", L, inputs.positions_rsa_sheared(rad, L, g, rng), rad)
    sp = params.choose(cfg.L, cfg.N, 1e-6, M_max=96, a_eff=params.effective_radius(cfg.rad), precision=0)
    c = api.Context()
    c.set_params(sp.xi, sp.M, sp.P, sp.rc)
    c.set_option(api.SE_OPT_SHAPE_M, sp.m)
    c.set_option(api.SE_OPT_SIZE_MODE, 2)
    c.set_option(api.SE_OPT_SHEAR, g)
    c.set_option(api.SE_OPT_PRECISION, 0)
    c.set_option(api.SE_OPT_RESTART, 100)
    c.set_config(cfg.pos, cfg.rad, cfg.L)
    w = os.path.join(os.path.dirname(api.__file__), "learned_pc_weights.npy")
    c.set_learned_weights(np.load(w))
    b = torch.tensor(np.random.default_rng(6).standard_normal((cfg.N, 11)), device="cuda")
    out = {}
    for pc in (api.SE_PRECOND_BLOCK, api.SE_PRECOND_SPECTRAL, api.SE_PRECOND_LEARNED):
        x, iters, relres = c.solve(b, rtol=1e-6, maxit=800, precond=pc)
        assert relres <= 1e-6
        out[pc] = (x.cpu().numpy(), iters)
    xb, ib = out[api.SE_PRECOND_BLOCK]
    print("sheared solves (block, spectral, learned):", ib, out[api.SE_PRECOND_SPECTRAL][1],
          out[api.SE_PRECOND_LEARNED][1])
    for pc in (api.SE_PRECOND_SPECTRAL, api.SE_PRECOND_LEARNED):
        x, it = out[pc]
        assert it <= 0.8 * ib
        assert rel(x, xb) <= 3e-4


def test_shear_needs_the_wave_space_approach(poly):
    cfg, _ = poly
    c = api.Context()
    c.set_params(1.0, 64, 24, 5.45)
    with pytest.raises(api.SeError):
        c.set_option(api.SE_OPT_SHEAR, 0.2)              # size approach 0 (hybrid)
    c.set_option(api.SE_OPT_SIZE_MODE, 2)
    c.set_option(api.SE_OPT_SHEAR, 0.2)
    with pytest.raises(api.SeError):
        c.set_option(api.SE_OPT_SIZE_MODE, 1)
    with pytest.raises(api.SeError):
        c.set_option(api.SE_OPT_SHEAR, 0.7)              # outside [-1/2, 1/2]
    c.set_config(cfg.pos, cfg.rad, cfg.L)
