"""Far-field Brownian source M^{-1/2} c by the Swan-Brady initial value problem (Sec. 4.3,
Eqs. ivp-1, ivp-forward, ivp-backward; se_brownian_ivp) against the FP64 oracle: the same
discrete scheme on the dense oracle matrix (oracle/brownian.py), and the exact
A^{-1/2} c from its eigendecomposition within the scheme's own discretisation error.

Tolerances: the GPU scheme differs from the oracle's by the SE product error and the
GMRES tolerance of its solves, amplified by the conditioning of the shifted systems
(measured in the test); FP64 products ~1e-10 -> 1e-7 bound, FP32 products with FP64
refinement -> 1e-5."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import brownian  # noqa: E402
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


def test_ivp_fts_fp64_matches_oracle_scheme(oracle_mod):
    """N = 14 log-normal spheres at phi = 0.3, F, T, S (11 components), FP64 products,
    dtau = 0.1 and 0.05."""
    cfg = inputs.lognormal(seed=8, n=14, phi=0.3)
    A = oracle_mod.dense_matrix(cfg.pos, cfg.rad, cfg.L, ncomp=11, tol=1e-13)
    c = np.random.default_rng(3).standard_normal((cfg.N, 11))
    ctx = make(cfg, 1e-11, precision=1)
    s = 6 * math.pi * float(np.mean(cfg.rad))
    exact = brownian.inv_sqrt(A, c.reshape(-1))
    for nsteps in (10, 20):
        x, prods = ctx.brownian_ivp(torch.tensor(c, device="cuda"), nsteps=nsteps, rtol=1e-12, scale=s)
        x = x.cpu().numpy().reshape(-1)
        ref = math.sqrt(s) * brownian.ivp_inv_sqrt(s * A, c.reshape(-1), nsteps)
        err, disc = rel(x, ref), rel(ref, exact)
        print(f"nsteps {nsteps}: vs oracle scheme {err:.2e}, scheme vs exact {disc:.2e}, {prods} products")
        assert err <= 1e-7
        assert rel(x, exact) <= disc + 1e-7
    # the default scale (6 pi eta <a>) is the one used above
    x2, _ = ctx.brownian_ivp(torch.tensor(c, device="cuda"), nsteps=10, rtol=1e-12)
    x1, _ = ctx.brownian_ivp(torch.tensor(c, device="cuda"), nsteps=10, rtol=1e-12, scale=s)
    assert float(torch.linalg.norm(x2 - x1) / torch.linalg.norm(x1)) <= 1e-10


def test_ivp_forces_fp32_products(oracle_mod):
    """N = 60 monodisperse spheres at phi = 0.35, forces only, FP32 products with FP64
    refinement in every solve, against the oracle scheme on the dense oracle matrix."""
    cfg = inputs.mono_dense(seed=4, n=60, phi=0.35)
    A = oracle_mod.dense_matrix(cfg.pos, cfg.rad, cfg.L, ncomp=3, tol=1e-12)
    c = np.random.default_rng(5).standard_normal((cfg.N, 3))
    ctx = make(cfg, 1e-8, precision=0, fp32_tol=1e-5)
    s = 6 * math.pi
    x, prods = ctx.brownian_ivp(torch.tensor(c, device="cuda"), nsteps=10, rtol=1e-8, scale=s)
    ref = math.sqrt(s) * brownian.ivp_inv_sqrt(s * A, c.reshape(-1), 10)
    err = rel(x.cpu().numpy().reshape(-1), ref)
    print(f"FP32 products: vs oracle scheme {err:.2e}, {prods} products")
    assert err <= 1e-5


def test_ivp_rejects_the_trace_components():
    cfg = inputs.lognormal(seed=8, n=5, phi=0.2)
    ctx = make(cfg, 1e-8, precision=1)
    with pytest.raises(api.SeError) as e:
        ctx.brownian_ivp(torch.zeros(cfg.N, 12, device="cuda", dtype=torch.float64))
    assert e.value.code == api.SE_ERR_ARG
