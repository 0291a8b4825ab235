"""GMRES with the block-diagonal far-field preconditioner (Sec. 5, the preconditioner
built from the diagonal blocks of the far-field mobility) against the FP64 oracle: the
solution of the dense oracle system, and the residual of the oracle product at sampled
rows for a system too large to assemble.

Tolerances: a converged solve with FP64 products matches the oracle's dense solution to
within cond(M) x the product error, both measured in the test (the perturbation bound of
a linear system); with FP32 products and FP64 true-residual refinement, the residual
against the oracle matrix is the solve tolerance plus the FP32 product error (~5e-7).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1506_08481_b300 import api, inputs, params  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solve_ctx(cfg, tol, precision, M_max=64, restart=60, fp32_tol=None):
    """Context for solves: tol bounds the method error (the FP64 residual products),
    fp32_tol the FP32 rounding of the Krylov products when precision is 0."""
    sp = params.choose(cfg.L, cfg.N, tol, M_max=M_max, a_eff=params.effective_radius(cfg.rad),
                       fp32_tol=fp32_tol if precision == 0 else None)
    ctx = api.Context()
    ctx.set_params(sp.xi, sp.M, sp.P, sp.rc)
    ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
    ctx.set_option(api.SE_OPT_PRECISION, precision)
    ctx.set_option(api.SE_OPT_RESTART, restart)
    ctx.set_config(cfg.pos, cfg.rad, cfg.L)
    return ctx


@pytest.fixture(scope="module")
def poly40(oracle_mod):
    """N = 40 log-normal spheres (mean 1, std 0.2) at phi = 0.3; dense F,T,S oracle system."""
    cfg = inputs.lognormal(seed=21, n=40, phi=0.3)
    A = oracle_mod.dense_matrix(cfg.pos, cfg.rad, cfg.L, ncomp=11, tol=1e-13)
    b = np.random.default_rng(5).standard_normal((cfg.N, 11))
    x = np.linalg.solve(A, b.reshape(-1)).reshape(cfg.N, 11)
    return cfg, A, b, x


def product_error(ctx, A, N, nc=11, seed=17):
    """Relative 2-norm error of the context's product against the oracle matrix."""
    v = np.random.default_rng(seed).standard_normal((N, nc))
    y = ctx.apply(torch.tensor(v, device="cuda")).cpu().numpy()
    ref = (A @ v.reshape(-1)).reshape(N, nc)
    return rel(y, ref)


def test_fp64_solve_matches_oracle_solution(poly40):
    """With FP64 products the solve converges to the solution of the perturbed system
    M_se x = b; its distance to the oracle's solution is bounded by cond(M) times the
    product error (perturbation bound for linear systems)."""
    cfg, A, b, x_or = poly40
    ctx = solve_ctx(cfg, 1e-11, precision=1)
    ep = product_error(ctx, A, cfg.N)
    assert ep <= 1e-8
    bt = torch.tensor(b, device="cuda")
    x, iters, relres = ctx.solve(bt, rtol=1e-12, maxit=400, precond=api.SE_PRECOND_BLOCK)
    x = x.cpu().numpy()
    assert relres <= 1e-12
    kappa = np.linalg.cond(A)
    assert rel(x, x_or) <= 2 * kappa * (ep + 1e-12)
    # residual of the oracle system: (M_se - A) x, bounded by the operator error times |A| |x|
    bound = 2 * ep * np.linalg.norm(A, 2) * np.linalg.norm(x) / np.linalg.norm(b) + 1e-12
    assert np.linalg.norm(b.reshape(-1) - A @ x.reshape(-1)) / np.linalg.norm(b) <= bound
    print(f"product error {ep:.2e}, cond {kappa:.1f}, solution error {rel(x, x_or):.2e}, {iters} products")


def test_fp32_products_with_fp64_refinement(poly40):
    """FP32 products inside the Krylov cycles, FP64 true residual at each restart: the
    solve stops at rtol against its own FP64 product, and against the oracle matrix
    the residual is rtol plus the product error times |A| |x| / |b|."""
    cfg, A, b, x_or = poly40
    ctx = solve_ctx(cfg, 1e-9, precision=0, fp32_tol=1e-5)
    ep32 = product_error(ctx, A, cfg.N)
    assert ep32 <= 1e-5
    ctx.set_option(api.SE_OPT_PRECISION, 1)
    ep64 = product_error(ctx, A, cfg.N)
    ctx.set_option(api.SE_OPT_PRECISION, 0)
    bt = torch.tensor(b, device="cuda")
    x, iters, relres = ctx.solve(bt, rtol=1e-6, maxit=400, precond=api.SE_PRECOND_BLOCK)
    x = x.cpu().numpy()
    assert relres <= 1e-6
    amp = np.linalg.norm(A, 2) * np.linalg.norm(x) / np.linalg.norm(b)
    assert np.linalg.norm(b.reshape(-1) - A @ x.reshape(-1)) / np.linalg.norm(b) <= 1e-6 + 2 * ep64 * amp
    assert rel(x, x_or) <= np.linalg.cond(A) * (1e-6 + 2 * ep64 * amp)
    print(f"FP32 product error {ep32:.2e}, FP64 {ep64:.2e}, {iters} products")


def test_preconditioners_reach_the_same_solution(poly40):
    """No preconditioner, the block preconditioner and the learned one without weights
    converge to one solution; the block preconditioner needs fewer products."""
    cfg, A, b, x_or = poly40
    ctx = solve_ctx(cfg, 1e-11, precision=1)
    bt = torch.tensor(b, device="cuda")
    out = {}
    for name, pc in (("none", api.SE_PRECOND_NONE), ("block", api.SE_PRECOND_BLOCK),
                     ("learned", api.SE_PRECOND_LEARNED)):
        x, iters, relres = ctx.solve(bt, rtol=1e-11, maxit=600, precond=pc)
        assert relres <= 1e-11, name
        out[name] = (x.cpu().numpy(), iters)
    bound = 2 * np.linalg.cond(A) * (product_error(ctx, A, cfg.N) + 1e-11)
    for name in out:
        assert rel(out[name][0], x_or) <= bound, name
    assert out["block"][1] < out["none"][1]
    print("products none/block/learned:", [out[k][1] for k in out])


def test_forces_only_solve(oracle_mod, poly40):
    cfg, _, b11, _ = poly40
    A = oracle_mod.dense_matrix(cfg.pos, cfg.rad, cfg.L, ncomp=3, tol=1e-13)
    b = b11[:, :3].copy()
    x_or = np.linalg.solve(A, b.reshape(-1)).reshape(cfg.N, 3)
    ctx = solve_ctx(cfg, 1e-11, precision=1)
    ep = product_error(ctx, A, cfg.N, nc=3)
    x, iters, relres = ctx.solve(torch.tensor(b, device="cuda"), rtol=1e-12, maxit=300)
    assert rel(x.cpu().numpy(), x_or) <= 2 * np.linalg.cond(A) * (ep + 1e-12)


def test_single_sphere_block_is_the_exact_inverse():
    """One sphere in the box: M_inf is its own diagonal block, which the block
    preconditioner inverts, so GMRES stops after one product."""
    cfg = inputs.Config("one", 9.0, np.array([[1.0, 2.0, 3.0]]), np.array([1.3]))
    ctx = solve_ctx(cfg, 1e-11, precision=1)
    b = torch.tensor(np.random.default_rng(9).standard_normal((1, 11)), device="cuda")
    x, iters, relres = ctx.solve(b, rtol=1e-10, maxit=50)
    assert relres <= 1e-10 and iters <= 2
    y = ctx.apply(x)
    assert rel(y.cpu().numpy(), b.cpu().numpy()) <= 1e-10


def test_lognormal_n20000_solve_rows_vs_oracle(oracle_mod):
    """Polydisperse solve at N = 20000, phi = 0.4, log-normal radii: GMRES to 1e-6 with
    the plain, the learned (trained weights if the package has them) and the spectral
    preconditioner, FP32 products with double-float true residuals.  The oracle product of
    each solution at 64 random rows gives back the right-hand side to the tolerance plus the
    product error, and the library's FP64 product of the solution equals the oracle's on
    those rows to the method error (the parameters are chosen for 1e-8)."""
    import os
    cfg = inputs.lognormal(seed=3, n=20000, phi=0.4)
    ctx = solve_ctx(cfg, 1e-8, precision=0, M_max=128, restart=100, fp32_tol=1e-5)
    rng = np.random.default_rng(13)
    b = rng.standard_normal((cfg.N, 11))
    bt = torch.tensor(b, device="cuda")
    weights = os.path.join(os.path.dirname(api.__file__), "learned_pc_weights.npy")
    if os.path.exists(weights):
        ctx.set_learned_weights(np.load(weights))
    rows = rng.choice(cfg.N, 64, replace=False)
    its = {}
    for name, pc in (("block", api.SE_PRECOND_BLOCK), ("learned", api.SE_PRECOND_LEARNED),
                     ("spectral", api.SE_PRECOND_SPECTRAL)):
        x, iters, relres = ctx.solve(bt, rtol=1e-6, maxit=1500, precond=pc)
        assert relres <= 1e-6, name
        ctx.set_option(api.SE_OPT_PRECISION, 1)
        y64 = ctx.apply(x).cpu().numpy()
        ctx.set_option(api.SE_OPT_PRECISION, 0)
        assert rel(y64, b) <= 1.05e-6, name
        x12 = np.zeros((cfg.N, 12))
        x12[:, :11] = x.cpu().numpy()
        y = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x12, rows=rows, tol=1e-10)[:, :11]
        d, r = rel(y64[rows], y), rel(y, b[rows])
        print(f"N=20000 {name}: oracle residual on 64 rows {r:.2e}, FP64 product vs oracle {d:.2e}")
        assert d <= 1e-7, name
        assert r <= 1.5e-6, name
        its[name] = iters
    print("N=20000 products block/learned/spectral:", its)
    assert its["spectral"] < its["block"]


def test_spectral_preconditioner_cuts_products():
    """Monodisperse phi = 0.45, N = 4000: the long-wavelength transverse force modes set
    the iteration count of the block-preconditioned solve; the spectral correction of
    those modes (SE_PRECOND_SPECTRAL) needs fewer products and reaches the same solution."""
    cfg = inputs.mono_dense(seed=2, n=4000, phi=0.45)
    ctx = solve_ctx(cfg, 1e-9, precision=1, M_max=96, restart=100)
    b = torch.tensor(np.random.default_rng(21).standard_normal((cfg.N, 11)), device="cuda")
    xb, ib, rb = ctx.solve(b, rtol=1e-8, maxit=1000, precond=api.SE_PRECOND_BLOCK)
    xs, is_, rs = ctx.solve(b, rtol=1e-8, maxit=1000, precond=api.SE_PRECOND_SPECTRAL)
    assert rb <= 1e-8 and rs <= 1e-8
    assert float(torch.linalg.norm(xs - xb) / torch.linalg.norm(xb)) <= 1e-6
    print("N=4000 products block/spectral:", ib, is_)
    assert is_ < ib
