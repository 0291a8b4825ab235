"""Rigid spheres driven by forces and torques (E = 0; se_rigid_solve) and the far-field
self-diffusivity estimator of Sec. 6.1 (Eq. dstr-def; se_far_field_diffusivity) against
the FP64 oracle (oracle/diffusivity.py on the dense oracle matrix).  FP64 products: the
GMRES tolerance and the product error (~1e-10) times the conditioning bound the
difference (1e-8); FP32 products with FP64 refinement: 1e-5."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import diffusivity  # noqa: E402
from paper_1506_08481_b300 import api, inputs, params  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make(cfg, tol, precision, fp32_tol=None):
    sp = params.choose(cfg.L, cfg.N, tol, M_max=64, a_eff=params.effective_radius(cfg.rad),
                       fp32_tol=fp32_tol if precision == 0 else None)
    ctx = api.Context()
    ctx.set_params(sp.xi, sp.M, sp.P, sp.rc)
    ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
    ctx.set_option(api.SE_OPT_PRECISION, precision)
    ctx.set_option(api.SE_OPT_RESTART, 60)
    ctx.set_config(cfg.pos, cfg.rad, cfg.L)
    return ctx


@pytest.fixture(scope="module")
def poly12(oracle_mod):
    cfg = inputs.lognormal(seed=9, n=12, phi=0.3)
    M = oracle_mod.dense_matrix(cfg.pos, cfg.rad, cfg.L, ncomp=11, tol=1e-13)
    return cfg, M, diffusivity.rigid_mobility(M)


def test_rigid_solve_fp64(poly12):
    cfg, M, mu = poly12
    ctx = make(cfg, 1e-11, precision=1)
    f = np.random.default_rng(2).standard_normal((cfg.N, 6))
    uw, s, iters, relres = ctx.rigid_solve(torch.tensor(f, device="cuda"), rtol=1e-12)
    uw_or, s_or = diffusivity.rigid_response(M, f)
    print(f"rigid solve: U {rel(uw.cpu().numpy(), uw_or):.2e}, S {rel(s.cpu().numpy(), s_or):.2e}, {iters} products")
    assert relres <= 1e-12
    assert rel(uw.cpu().numpy(), uw_or) <= 1e-8
    assert rel(s.cpu().numpy(), s_or) <= 1e-7


def test_diffusivity_estimator_fp64(poly12):
    """The estimator on given samples equals the oracle's estimator on the same samples."""
    cfg, M, mu = poly12
    ctx = make(cfg, 1e-11, precision=1)
    fr = np.random.default_rng(3).standard_normal((4, cfg.N, 6))
    d, prods = ctx.far_field_diffusivity(torch.tensor(fr, device="cuda"), rtol=1e-12)
    ref = diffusivity.estimate(mu, fr)
    print(f"estimator: {rel(d.cpu().numpy(), ref):.2e}, {prods} products")
    assert rel(d.cpu().numpy(), ref) <= 1e-8


def test_simple_cubic_array_rigid_mobility():
    """One sphere per periodic cell: the rigid mobility is Hasimoto's drag, no stresslet."""
    cfg = inputs.Config("sc", 12.0, np.array([[3.0, 4.0, 5.0]]), np.array([1.0]))
    ctx = make(cfg, 1e-11, precision=1)
    f = torch.tensor([[1.0, 0.0, 0.0, 0.0, 0.0, 0.0]], device="cuda", dtype=torch.float64)
    uw, s, _, _ = ctx.rigid_solve(f, rtol=1e-12)
    x = 1.0 / 12.0
    assert abs(6 * math.pi * float(uw[0, 0]) - (1 - 2.837297 * x + 4 * math.pi / 3 * x ** 3)) < 2e-5
    assert float(s.abs().max()) < 1e-10


def test_rigid_solve_fp32_products(oracle_mod):
    cfg = inputs.mono_dense(seed=4, n=30, phi=0.35)
    M = oracle_mod.dense_matrix(cfg.pos, cfg.rad, cfg.L, ncomp=11, tol=1e-12)
    ctx = make(cfg, 1e-8, precision=0, fp32_tol=1e-5)
    f = np.random.default_rng(4).standard_normal((cfg.N, 6))
    uw, s, iters, relres = ctx.rigid_solve(torch.tensor(f, device="cuda"), rtol=1e-8)
    uw_or, _ = diffusivity.rigid_response(M, f)
    print(f"FP32 products: U {rel(uw.cpu().numpy(), uw_or):.2e}, {iters} products")
    assert rel(uw.cpu().numpy(), uw_or) <= 1e-5


def test_imposed_strain_and_viscosity(poly12):
    """Force- and torque-free rigid spheres in an imposed strain, and the high-frequency
    viscosity eta_s / eta, against the oracle's resistance relations."""
    cfg, M, mu = poly12
    ctx = make(cfg, 1e-11, precision=1)
    e = np.array([0.3, -0.2, 1.0, 0.1, 0.5])
    uw, s, iters, relres = ctx.rigid_solve(None, einf=e, rtol=1e-12)
    uw_or, s_or = diffusivity.rigid_response_strain(M, e)
    print(f"imposed strain: U {rel(uw.cpu().numpy(), uw_or):.2e}, S {rel(s.cpu().numpy(), s_or):.2e}")
    assert rel(s.cpu().numpy(), s_or) <= 1e-8
    assert rel(uw.cpu().numpy(), uw_or) <= 1e-7
    r, prods = ctx.high_frequency_viscosity(rtol=1e-12)
    r_or = diffusivity.viscosity_ratio(M, cfg.L)
    print(f"eta_s/eta {r:.12f} vs oracle {r_or:.12f}, {prods} products")
    assert abs(r - r_or) <= 1e-9 * r_or
