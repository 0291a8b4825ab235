"""GPU parity of the Spectral Ewald grand-mobility product against the FP64
direct-Ewald oracle, element by element on the same seeded inputs.

Tolerances (relative 2-norm over all compared components):
  FP64 mode   <= 1e-9   (parameters chosen for ~1e-10 truncation error)
  FP32 mode   <= 1e-6
derived from the FP32 unit roundoff 6e-8 times the ~10x growth through the
spread / FFT / gather chain; the real-space part alone must match the oracle's
real-space part to 1e-12 (FP64), being the same sum term by term.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1506_08481_b300 import api, inputs  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_ctx(xi, M, P, rc, cfg, precision=1, size_mode=0, parts=7):
    ctx = api.Context()
    ctx.set_params(xi, M, P, rc)
    ctx.set_option(api.SE_OPT_PRECISION, precision)
    ctx.set_option(api.SE_OPT_SIZE_MODE, size_mode)
    ctx.set_option(api.SE_OPT_PARTS, parts)
    ctx.set_config(cfg.pos, cfg.rad, cfg.L)
    return ctx


def gpu_apply(ctx, x, dtype=torch.float64):
    xt = torch.tensor(np.ascontiguousarray(x), device="cuda", dtype=dtype)
    return ctx.apply(xt).double().cpu().numpy()


@pytest.fixture(scope="module")
def small_poly():
    """N = 37 polydisperse spheres (radii 0.5..1.0) at phi ~ 0.1 in a box of 11."""
    rng = np.random.default_rng(11)
    rad = rng.uniform(0.5, 1.0, 37)
    L = 11.0
    pos = inputs.positions_rsa(rad, L, rng)
    x = rng.standard_normal((37, 12))
    return inputs.Config("small_poly", L, pos, rad), x


@pytest.fixture(scope="module")
def small_poly_ref(oracle_mod, small_poly):
    cfg, x = small_poly
    return oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x, tol=1e-15)


def test_mono_n100_forces_fp64_parity(oracle_mod):
    """Monodisperse N=100, phi=0.2, forces only, FP64.  At the prescribed grid M=32 and
    support P=16 the method's own truncation + resolution error for this box is ~3e-8 at
    the best (xi, m) = (0.75, 6.5); with the grid and support the parameter chooser
    picks for 1e-10 the product matches the oracle to <= 1e-9."""
    from paper_1506_08481_b300 import params
    cfg = inputs.mono_n100(seed=0)
    x = np.zeros((cfg.N, 12))
    x[:, :3] = np.random.default_rng(1).standard_normal((cfg.N, 3))
    ref = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x, tol=1e-15)[:, :3]
    ctx = make_ctx(0.75, 32, 16, 6.35, cfg)
    ctx.set_option(api.SE_OPT_SHAPE_M, 6.5)
    assert rel(gpu_apply(ctx, x[:, :3]), ref) <= 1e-7
    sp = params.choose(cfg.L, cfg.N, 1e-11, M_max=64)
    ctx = make_ctx(sp.xi, sp.M, sp.P, sp.rc, cfg)
    ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
    assert rel(gpu_apply(ctx, x[:, :3]), ref) <= 1e-9


@pytest.mark.parametrize("size_mode", [0, 1, 2, 3])
def test_all_components_fp64(small_poly, small_poly_ref, size_mode):
    cfg, x = small_poly
    ctx = make_ctx(1.0, 64, 24, 5.45, cfg, precision=1, size_mode=size_mode)
    y = gpu_apply(ctx, x)
    for sl in (slice(0, 3), slice(3, 6), slice(6, 11), slice(11, 12)):
        assert rel(y[:, sl], small_poly_ref[:, sl]) <= 1e-9, sl


@pytest.mark.parametrize("size_mode", [0, 1, 2, 3])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_all_components_fp32(small_poly, small_poly_ref, size_mode, dtype):
    cfg, x = small_poly
    ctx = make_ctx(0.9, 48, 16, 5.4, cfg, precision=0, size_mode=size_mode)
    y = gpu_apply(ctx, x, dtype)
    assert rel(y, small_poly_ref) <= 1e-6


def test_real_space_part_term_by_term(oracle_mod, small_poly):
    """parts = real space only, FP64: the U, Omega, E rows equal the oracle's real-space
    sum (same xi and rc).  (E_tr splits the harmonic pressure Faxen term differently.)"""
    cfg, x = small_poly
    xi, rc = 0.8, 5.2
    ref = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x, xi=xi, rc=rc, kc=1.0, parts=1)
    ctx = make_ctx(xi, 32, 12, rc, cfg, precision=1, parts=1)
    y = gpu_apply(ctx, x)
    assert rel(y[:, :11], ref[:, :11]) <= 1e-12


def test_self_part(oracle_mod, small_poly):
    cfg, x = small_poly
    ref = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x, xi=0.8, rc=1.0, kc=1.0, parts=4)
    y = gpu_apply(make_ctx(0.8, 32, 12, 5.0, cfg, precision=1, parts=4), x)
    assert rel(y, ref) <= 1e-13


def test_ncomp_prefixes_agree(small_poly):
    """ncomp 3/6/11/12 use the leading components; results agree with zero-padded 12."""
    cfg, x = small_poly
    ctx = make_ctx(0.9, 48, 16, 5.4, cfg, precision=1)
    for nc in (3, 6, 11):
        xx = np.zeros_like(x)
        xx[:, :nc] = x[:, :nc]
        y12 = gpu_apply(ctx, xx)[:, :nc]
        y = gpu_apply(ctx, x[:, :nc].copy())
        assert rel(y, y12) <= 1e-13


def test_host_buffer_entry_point(small_poly):
    """se_mobility_apply_host with pageable and with page-locked host buffers, for all 12
    components and a 3-component prefix."""
    cfg, x = small_poly
    ctx = make_ctx(0.9, 48, 16, 5.4, cfg, precision=1)
    np.testing.assert_allclose(ctx.apply_host(x), gpu_apply(ctx, x), rtol=0, atol=1e-15)
    for nc in (12, 3):
        xp = torch.from_numpy(x[:, :nc].copy()).pin_memory()
        yp = torch.full_like(xp, float("nan")).pin_memory()
        out = ctx.apply_host(xp.numpy(), yp.numpy())
        np.testing.assert_allclose(out, gpu_apply(ctx, x[:, :nc].copy()), rtol=0, atol=1e-15)


@pytest.mark.parametrize("N,M", [(1, 24), (33, 72), (65, 40)])
def test_ragged_sizes_and_grids(oracle_mod, N, M):
    """N = 1, N not a multiple of the warp or block, M = 3 * 8, M = 72 and M = 40 (= 5 * 8,
    rejected) grids, particles straddling the periodic boundary."""
    rng = np.random.default_rng(N)
    rad = rng.uniform(0.6, 1.0, N)
    L = 9.0
    pos = inputs.positions_rsa(rad, L, rng)
    pos[0] = [L - 0.05, 0.02, L - 0.3]            # wraps around every face
    x = rng.standard_normal((N, 12))
    cfg = inputs.Config("ragged", L, pos, rad)
    if M == 40:
        ctx = api.Context()
        with pytest.raises(api.SeError) as e:
            ctx.set_params(1.0, M, 16, 4.0)
        assert e.value.code == api.SE_ERR_GRID
        return
    from paper_1506_08481_b300 import params
    ref = oracle_mod.mobility(pos, rad, L, x, tol=1e-14)
    tol = 1e-11 if M > 24 else 1e-5
    sp = params.choose(L, N, tol, M_max=M, M_min=M, a_eff=params.effective_radius(rad))
    ctx = make_ctx(sp.xi, M, sp.P, sp.rc, cfg, precision=1)
    ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
    y = gpu_apply(ctx, x)
    assert rel(y, ref) <= 100 * tol


def _raw_apply(ctx, ncomp, x, y, dtype):
    import ctypes
    return ctx.lib.se_mobility_apply(ctx.h, ncomp, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), dtype)


def test_error_codes():
    """The C ABI returns its documented codes and leaves the context usable."""
    ctx = api.Context()
    z = torch.zeros(8, 12, device="cuda", dtype=torch.float64)
    assert _raw_apply(ctx, 3, z, z.clone(), api.SE_F64) == api.SE_ERR_STATE   # before params/config
    ctx.set_params(1.0, 32, 12, 4.0)
    with pytest.raises(api.SeError) as e:
        ctx.set_config(np.zeros((0, 3)), np.ones(0), 10.0)                    # empty configuration
    assert e.value.code == api.SE_ERR_ARG
    with pytest.raises(api.SeError) as e:
        ctx.set_config(np.zeros((2, 3)), np.ones(2), 7.9)                     # rc >= L/2
    assert e.value.code == api.SE_ERR_CUTOFF
    pos = np.array([[1.0, 1.0, 1.0], [np.nan, 2.0, 2.0]])
    with pytest.raises(api.SeError) as e:
        ctx.set_config(pos, np.ones(2), 10.0)
    assert e.value.code == api.SE_ERR_NONFINITE
    with pytest.raises(api.SeError) as e:
        ctx.set_config(np.array([[1.0, 1.0, 1.0], [2.0, 2.0, 2.0]]), np.array([1.0, -1.0]), 10.0)
    assert e.value.code == api.SE_ERR_NONFINITE
    with pytest.raises(api.SeError) as e:
        ctx.set_params(1.0, 32, 30, 4.0)                                       # P > M - 8
    assert e.value.code == api.SE_ERR_GRID
    ctx.set_params(1.0, 32, 12, 4.0)
    ctx.set_config(np.array([[1.0, 1.0, 1.0], [4.0, 4.0, 4.0]]), np.ones(2), 10.0)
    x = torch.zeros(2, 12, device="cuda", dtype=torch.float64)
    assert _raw_apply(ctx, 5, x, x.clone(), api.SE_F64) == api.SE_ERR_ARG     # ncomp
    assert _raw_apply(ctx, 12, x, x.clone(), 7) == api.SE_ERR_ARG             # dtype
    assert ctx.lib.se_set_option(ctx.h, 99, 1.0) == api.SE_ERR_ARG
    y = ctx.apply(torch.ones(2, 12, device="cuda", dtype=torch.float64))       # still usable
    assert torch.isfinite(y).all()


def test_bidisperse_n2000_precision_ladder(oracle_mod):
    """Bidisperse N=2000 (radii 1, 2), phi=0.3, F,T,S (11 components): parameter sets
    tuned for 1e-4, 1e-6, 1e-8; FP32 meets 1e-4 and 1e-6, FP64 meets 1e-8."""
    cfg = inputs.bidisperse(seed=0)
    x = inputs.moments(cfg.N, np.random.default_rng(5), 11)
    ref = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x, tol=1e-12)[:, :11]
    from paper_1506_08481_b300 import params
    for tol, prec in ((1e-4, 0), (1e-6, 0), (1e-8, 1)):
        sp = params.choose(cfg.L, cfg.N, tol / 3, M_max=192, a_eff=params.effective_radius(cfg.rad),
                           precision=prec)
        ctx = make_ctx(sp.xi, sp.M, sp.P, sp.rc, cfg, precision=prec)
        ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
        y = gpu_apply(ctx, x[:, :11].copy())
        err = rel(y, ref)
        assert err <= tol, (tol, err)


def test_viscosity_scales_the_product(small_poly):
    """Every block of M_inf carries 1/eta (Eqs. oseen, faxen-f/t/s/p): changing the
    viscosity after the configuration is set rescales the product exactly."""
    cfg, x = small_poly
    ctx = make_ctx(0.9, 48, 16, 5.4, cfg, precision=1)
    y1 = gpu_apply(ctx, x)
    ctx.set_option(api.SE_OPT_ETA, 2.5)
    y2 = gpu_apply(ctx, x)
    assert rel(y2 * 2.5, y1) <= 1e-13
    ctx.set_option(api.SE_OPT_ETA, 1.0)
    assert rel(gpu_apply(ctx, x), y1) <= 1e-15


@pytest.mark.parametrize("size_mode", [0, 1])
def test_gather_variants_agree(small_poly, small_poly_ref, size_mode):
    """The warp-per-particle gather and the bin-staged gather (SE_OPT_GATHER 1, 2) sum
    the same terms in a different order: they agree to rounding, and both match the oracle."""
    cfg, x = small_poly
    out = {}
    for g in (1, 2):
        ctx = make_ctx(1.0, 64, 24, 5.45, cfg, precision=1, size_mode=size_mode)
        ctx.set_option(api.SE_OPT_GATHER, g)
        out[g] = gpu_apply(ctx, x)
        assert rel(out[g], small_poly_ref) <= 1e-9
    assert rel(out[2], out[1]) <= 1e-13


@pytest.mark.parametrize("precision", [0, 1])
def test_real_space_placement_identical(oracle_mod, precision):
    """The real-space sum in line or on the second stream beside the spread or the FFT
    chain runs the same kernels: the products are bitwise identical (each placement
    twice).  Inside the gather kernel (overlap 3, FP32) every target's pairs are summed in
    the same order by other compiled code, whose multiply-adds the compiler may contract
    differently: that product agrees to FP32 rounding.  All match the oracle."""
    from paper_1506_08481_b300 import params
    cfg = inputs.bidisperse(seed=3, n=3000, phi=0.3)
    x = inputs.moments(cfg.N, np.random.default_rng(4), 12)
    sp = params.choose(cfg.L, cfg.N, 2.5e-7, a_eff=params.effective_radius(cfg.rad), precision=precision,
                       fp32_tol=1e-6 if precision == 0 else None)
    ctx = make_ctx(sp.xi, sp.M, sp.P, sp.rc, cfg, precision=precision, size_mode=1)
    ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
    dt = torch.float32 if precision == 0 else torch.float64
    outs, launches = {}, {}
    for overlap in (2, 0, 1, 3, 2, 3):
        ctx.set_option(api.SE_OPT_OVERLAP, overlap)
        outs.setdefault(overlap, []).append(gpu_apply(ctx, x, dt))
        l0 = ctx.kernel_launches()
        outs[overlap].append(gpu_apply(ctx, x, dt))
        launches[overlap] = ctx.kernel_launches() - l0
    for ov in (0, 1, 2):
        for o in outs[ov]:
            assert np.array_equal(o, outs[2][0])
    for o in outs[3]:
        assert np.array_equal(o, outs[3][0])
        if precision == 0:
            assert rel(o, outs[2][0]) <= 1e-6
        else:
            assert np.array_equal(o, outs[2][0])
    # overlap 3: the FP32 product sums the real-space part inside the gather kernel (one
    # launch fewer); the FP64 and double-float products run it in line
    assert launches[3] == launches[2] - (1 if precision == 0 else 0)
    rows = np.random.default_rng(5).choice(cfg.N, 12, replace=False)
    ref = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x, rows=rows, tol=1e-12)
    for ov in (2, 3):
        assert rel(outs[ov][0][rows], ref) <= 1e-6
    with pytest.raises(api.SeError):
        ctx.set_option(api.SE_OPT_OVERLAP, 4)


def _fill_case(case):
    rng = np.random.default_rng({"poly": 21, "close": 22, "wide": 23}[case])
    if case == "poly":
        rad = rng.uniform(0.3, 1.0, 500)
        L = inputs.box_side(rad, 0.3)
        return inputs.Config(case, L, inputs.positions_rsa(rad, L, rng), rad), 0.7, min(7.0, 0.49 * L)
    if case == "close":
        # pairs at separation 0.085 (spheres of radius 0.04 nearly touching): r < 0.1
        L, n = 4.0, 150
        c = inputs.positions_rsa(np.full(n, 0.2), L, rng)
        d = rng.standard_normal((n, 3))
        d *= 0.085 / np.linalg.norm(d, axis=1, keepdims=True)
        pos = np.concatenate([c, c + d])
        return inputs.Config(case, L, pos, np.full(2 * n, 0.04)), 3.0, 1.5
    rad = np.full(200, 0.5)
    L = 12.0
    return inputs.Config(case, L, inputs.positions_rsa(rad, L, rng), rad), 2.0, 5.0      # xi rc = 10


@pytest.mark.parametrize("case", ["poly", "close", "wide"])
def test_pair_fill_double_float(oracle_mod, case):
    """The FP32 pair table's radial coefficients evaluated in double-float arithmetic
    (SE_OPT_PAIR_FILL 0, the default) and in FP64 (1) round to the same FP32 numbers but for
    rare last-bit differences: the FP32 real-space products agree to 2e-8 relative, and both
    match the oracle's real-space sum to FP32 accuracy.  'close' has pairs closer than 0.1 and
    'wide' has xi r up to 10, both beyond the double-float range (those pairs take FP64)."""
    cfg, xi, rc = _fill_case(case)
    x = inputs.moments(cfg.N, np.random.default_rng(5), 12)
    ref = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x, xi=xi, rc=rc, kc=1.0, parts=1)
    ctx = make_ctx(xi, 32, 12, rc, cfg, precision=0, parts=1)
    y_ff = gpu_apply(ctx, x, torch.float32)
    ctx.set_option(api.SE_OPT_PAIR_FILL, 1)
    y_64 = gpu_apply(ctx, x, torch.float32)
    ctx.set_option(api.SE_OPT_PAIR_FILL, 0)
    assert np.array_equal(gpu_apply(ctx, x, torch.float32), y_ff)
    assert rel(y_ff, y_64) <= 2e-8
    assert rel(y_ff[:, :11], ref[:, :11]) <= 5e-7
    assert rel(y_64[:, :11], ref[:, :11]) <= 5e-7
    with pytest.raises(api.SeError):
        ctx.set_option(api.SE_OPT_PAIR_FILL, 2)


def test_monodisperse_pair_table(oracle_mod):
    """Equal radii: the FP32 table stores 13 of the 19 coefficients and derives the others
    (c3 = c2, c9..c11 = -c6..-c8, c17 = 3 c15, c18 = -3 c16).  Against the 19-coefficient
    table of the same spheres (one radius moved by one part in 1e15, which makes the
    configuration polydisperse), the real-space and full FP32 products agree to FP32
    rounding (the derived coefficients differ from separately rounded ones by up to 1.5 ulp;
    a wrong slot or sign would differ at order one), and the real-space part matches the
    oracle."""
    rng = np.random.default_rng(41)
    rad = np.full(1200, 1.0)
    L = inputs.box_side(rad, 0.25)
    cfg = inputs.Config("mono", L, inputs.positions_rsa(rad, L, rng), rad)
    rad2 = rad.copy()
    rad2[7] *= 1 + 1e-15
    cfg2 = inputs.Config("mono_perturbed", L, cfg.pos, rad2)
    x = inputs.moments(cfg.N, np.random.default_rng(6), 12)
    xi, rc = 0.8, 5.5
    ref = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x, xi=xi, rc=rc, kc=1.0, parts=1)
    for parts, tol in ((1, 2e-7), (7, 2e-7)):
        y = gpu_apply(make_ctx(xi, 48, 16, rc, cfg, precision=0, size_mode=1, parts=parts), x, torch.float32)
        y2 = gpu_apply(make_ctx(xi, 48, 16, rc, cfg2, precision=0, size_mode=1, parts=parts), x, torch.float32)
        assert rel(y, y2) <= tol
        if parts == 1:
            assert rel(y[:, :11], ref[:, :11]) <= 5e-7


@pytest.mark.parametrize("ncomp", [3, 6, 11, 12])
@pytest.mark.parametrize("mono", [True, False])
def test_fused_gather_real_space(ncomp, mono):
    """The FP32 product with the real-space sum inside the gather kernel (SE_OPT_OVERLAP 3,
    the default) against the sum in a kernel of its own (2), for F T S (S_tr), the 13- and
    19-coefficient tables and two support sizes (P = 16: two support columns per gather
    lane; P = 14: one): each target's pairs are summed in the same order, so the products
    agree to FP32 rounding (bit for bit in the builds measured), with one kernel launch
    fewer per product.  F and F T (3, 6 components) keep the sum in line: their in-line
    sums read 2 and 6 coefficient rows."""
    rng = np.random.default_rng(43)
    rad = np.full(1500, 1.0) if mono else rng.uniform(0.6, 1.0, 1500)
    L = inputs.box_side(rad, 0.25)
    cfg = inputs.Config("fused", L, inputs.positions_rsa(rad, L, rng), rad)
    x = inputs.moments(cfg.N, np.random.default_rng(7), ncomp)[:, :ncomp].copy()
    for P in (16, 14):
        ctx = make_ctx(0.8, 48, P, 5.5, cfg, precision=0, size_mode=1)
        out, launches = {}, {}
        for ov in (2, 3):
            ctx.set_option(api.SE_OPT_OVERLAP, ov)
            gpu_apply(ctx, x, torch.float32)
            l0 = ctx.kernel_launches()
            out[ov] = gpu_apply(ctx, x, torch.float32)
            launches[ov] = ctx.kernel_launches() - l0
        assert launches[3] == launches[2] - (1 if ncomp > 6 else 0)
        assert rel(out[3], out[2]) <= 1e-6
        assert np.abs(out[3]).max() > 0 and np.isfinite(out[3]).all()


@pytest.mark.parametrize("precision", [0, 1])
def test_set_config_reuses_pair_buffers(precision):
    """set_config overwrites the previous configuration's pair table in place while it fits
    (same N, no more pairs than the buffers hold) and reallocates otherwise: a context
    taken through configurations A (phi 0.2), B (new positions), C (phi 0.35: more pairs
    than A's buffers hold), D (fewer particles) and A again gives, after each, the product
    of a fresh context on that configuration, bit for bit."""
    rng = np.random.default_rng(31)
    rad = rng.uniform(0.6, 1.0, 1500)
    def cfg(phi, n=1500, seed=0):
        r = rad[:n]
        L = inputs.box_side(r, phi)
        return inputs.Config(f"c{phi}_{n}_{seed}", L, inputs.positions_rsa(r, L, np.random.default_rng(seed)), r)
    cfgs = [cfg(0.2), cfg(0.2, seed=1), cfg(0.35), cfg(0.2, n=900), cfg(0.2)]
    dt = torch.float32 if precision == 0 else torch.float64
    xi, M, P = 0.9, 48, 16
    reused = make_ctx(xi, M, P, 5.0, cfgs[0], precision=precision, size_mode=1)
    for c in cfgs:
        x = inputs.moments(c.N, np.random.default_rng(c.N), 12)
        reused.set_config(c.pos, c.rad, c.L)
        y = gpu_apply(reused, x, dt)
        fresh = make_ctx(xi, M, P, 5.0, c, precision=precision, size_mode=1)
        assert np.array_equal(y, gpu_apply(fresh, x, dt)), c.name
        fresh.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_cutoff_boundary_pairs(oracle_mod, precision):
    """Pairs at |x| = rc (1 +- delta), delta from 1e-13 to 1e-2, along axes, diagonals and
    random directions, some across the periodic boundary, each pair further than rc from
    every other sphere: the real-space sum keeps exactly the pairs with |x| < rc (the
    FP64 decision of the oracle's image loop), including those decided in the thin band
    where FP32 separations cannot tell."""
    rng = np.random.default_rng(29)
    L, rc, xi = 40.0, 4.0, 0.5
    deltas = [s * d for d in (1e-13, 1e-9, 3e-7, 3e-6, 1e-4, 1e-2) for s in (1, -1)]
    dirs = [np.array([1.0, 0, 0]), np.array([0, -1.0, 0]), np.ones(3) / np.sqrt(3)]
    dirs += [v / np.linalg.norm(v) for v in rng.standard_normal((3, 3))]
    pos = []
    slots = [(8.0 + 10 * a, 8.0 + 10 * b, 8.0 + 10 * c) for a in range(4) for b in range(4) for c in range(4)]
    k = 0
    for d in deltas:
        for u in dirs[:4] if abs(d) > 1e-5 else dirs:
            p = np.array(slots[k])
            k += 1
            pos += [p, np.mod(p + rc * (1 + d) * u, L)]
    pos = np.array(pos)
    rad = np.full(len(pos), 0.5)
    cfg = inputs.Config("cutoff", L, pos, rad)
    x = rng.standard_normal((len(pos), 12))
    ref = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x, xi=xi, rc=rc, kc=1.0, parts=1)
    inside = np.array([d < 0 for d in deltas for _ in (dirs[:4] if abs(d) > 1e-5 else dirs)])
    # every pair inside rc is felt, every pair outside is not
    assert np.all(np.abs(ref[0::2][inside]).max(axis=1) > 1e-6)
    assert np.all(ref[0::2][~inside] == 0)
    ctx = make_ctx(xi, 32, 8, rc, cfg, precision=precision, parts=1)
    y = gpu_apply(ctx, x, dtype=torch.float64 if precision else torch.float32)
    assert np.all(y[0::2][~inside] == 0) and np.all(y[1::2][~inside] == 0)
    assert rel(y[:, :11], ref[:, :11]) <= (1e-12 if precision else 2e-6)


@pytest.mark.parametrize("M,P", [(216, 24), (72, 24), (48, 16), (48, 32), (24, 8), (24, 12)])
@pytest.mark.parametrize("ncomp", [3, 6, 11, 12])
def test_spread_variants_agree(small_poly, small_poly_ref, M, P, ncomp):
    """FP32 spreading over one-warp 8 x 4 x 16 blocks with packed FMAs (the default where the
    grid has room for it: M = 72 and 216 leave a last tile of 8 planes, M = 48 and 24 split the
    tiles' particles over partial grids, M = 24 with P = 12 falls back) and over two-warp
    8 x 8 x 16 tiles (SE_OPT_SPREAD 2) against 8^3 tiles (SE_OPT_SPREAD 1): the same terms in
    another order, so they agree to FP32 rounding."""
    cfg, x = small_poly
    x = x[:, :ncomp].copy()
    out = {}
    for s in (0, 1, 2):
        ctx = make_ctx(0.9, M, P, 5.4, cfg, precision=0)
        ctx.set_option(api.SE_OPT_SPREAD, s)
        out[s] = gpu_apply(ctx, x, dtype=torch.float32)
    # Each is an FP32 evaluation of the same sums; its rounding (2^-24) is amplified by the
    # cancellation in the real-space approach's Faxen weight 1 - a^2 kappa^2 alpha (Sec. 3.2;
    # kappa = M / L grid points per unit length, alpha = 2 pi / P at the default m = sqrt(pi P)),
    # about 100 for the largest sphere at M = 216 in this box of 11 (both are then ~3e-6 from FP64).
    amp = max(1.0, (cfg.rad.max() * M / cfg.L) ** 2 * 2 * np.pi / P)
    assert rel(out[0], out[1]) <= max(2e-6, 2.0 ** -24 * amp)
    assert rel(out[2], out[1]) <= max(2e-6, 2.0 ** -24 * amp)
    if M == 72 and ncomp == 12:
        assert rel(out[0], small_poly_ref) <= 1e-5


def test_overlap_detection():
    """se_set_config rejects overlapping spheres within rc (SE_ERR_OVERLAP), including
    across the periodic boundary and coincident centres; touching spheres are accepted;
    SE_OPT_OVERLAP_CHECK 0 turns the check off."""
    L = 10.0
    rad = np.array([1.0, 1.0, 0.5])
    cases = {
        "overlap": (np.array([[2.0, 2.0, 2.0], [3.9, 2.0, 2.0], [7.0, 7.0, 7.0]]), True),
        "periodic": (np.array([[0.5, 5.0, 5.0], [9.0, 5.0, 5.0], [5.0, 1.0, 8.0]]), True),   # 1.5 apart
        "coincident": (np.array([[4.0, 4.0, 4.0], [4.0, 4.0, 4.0], [8.0, 8.0, 8.0]]), True),
        "touching": (np.array([[2.0, 2.0, 2.0], [4.0, 2.0, 2.0], [7.0, 7.0, 7.0]]), False),
    }
    for name, (pos, bad) in cases.items():
        ctx = api.Context()
        ctx.set_params(1.0, 32, 8, 4.0)
        if bad:
            with pytest.raises(api.SeError) as e:
                ctx.set_config(pos, rad, L)
            assert e.value.code == api.SE_ERR_OVERLAP, name
        else:
            ctx.set_config(pos, rad, L)
            y = ctx.apply(torch.ones(3, 12, device="cuda", dtype=torch.float64))
            assert torch.isfinite(y).all(), name
    ctx = api.Context()
    ctx.set_params(1.0, 32, 8, 4.0)
    ctx.set_option(api.SE_OPT_OVERLAP_CHECK, 0)
    ctx.set_config(cases["overlap"][0], rad, L)
    assert torch.isfinite(ctx.apply(torch.ones(3, 12, device="cuda", dtype=torch.float64))).all()


@pytest.mark.parametrize("size_mode", [0, 1, 2, 3])
@pytest.mark.parametrize("ncomp", [3, 12])
def test_double_float_mode(small_poly, small_poly_ref, size_mode, ncomp):
    """SE_OPT_PRECISION 2 (spread and gather in double-float, the rest in FP64) gives the
    FP64 product to double-float rounding (~2^-44 per operation) and meets the FP64 parity
    bound against the oracle; FP32 and FP64 inputs and outputs."""
    cfg, x = small_poly
    xx = x[:, :ncomp].copy()
    c64 = make_ctx(1.0, 64, 24, 5.45, cfg, precision=1, size_mode=size_mode)
    y64 = gpu_apply(c64, xx)
    cff = make_ctx(1.0, 64, 24, 5.45, cfg, precision=2, size_mode=size_mode)
    yff = gpu_apply(cff, xx)
    assert rel(yff, y64) <= 1e-12
    if ncomp == 12:
        assert rel(yff, small_poly_ref) <= 1e-9
    y32io = gpu_apply(cff, xx, dtype=torch.float32)
    assert rel(y32io, y64) <= 2e-7


@pytest.mark.parametrize("ff_table", [1, 0])
@pytest.mark.parametrize("ncomp", [3, 6, 11, 12])
def test_double_float_real_space_part(oracle_mod, small_poly, ncomp, ff_table):
    """The real-space sum of SE_OPT_PRECISION 2 (the pair table contracted in double-float
    arithmetic) alone, reading the double-float copy of the pair table (SE_OPT_FF_TABLE 1)
    or converting the FP64 table as it reads it (0): equal to the FP64 real-space sum to
    double-float rounding and, in the U, Omega, E rows, to the oracle's real-space part
    (same xi, rc) to its FP64 parity bound, for every prefix.  (E_tr splits the harmonic
    pressure Faxen term differently.)"""
    cfg, x = small_poly
    xx = x[:, :ncomp].copy()
    y64 = gpu_apply(make_ctx(0.9, 48, 16, 5.4, cfg, precision=1, parts=1), xx)
    cff = make_ctx(0.9, 48, 16, 5.4, cfg, precision=2, parts=1)
    cff.set_option(api.SE_OPT_FF_TABLE, ff_table)
    yff = gpu_apply(cff, xx)
    assert rel(yff, y64) <= 1e-12
    x12 = np.zeros((cfg.N, 12))
    x12[:, :ncomp] = xx
    nr = min(ncomp, 11)
    ref = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x12, xi=0.9, rc=5.4, kc=1.0, parts=1)[:, :nr]
    assert rel(yff[:, :nr], ref) <= 1e-12


def test_double_float_mode_large_grid(oracle_mod):
    """Bidisperse N = 2000 at the parameters the error model picks for 1e-10 (FP64): the
    double-float product equals the FP64 one to 1e-12 and meets 1e-9 against the oracle."""
    cfg = inputs.bidisperse(seed=0)
    x12 = inputs.moments(cfg.N, np.random.default_rng(5), 11)          # [N, 12], S_tr = 0
    x = x12[:, :11].copy()
    from paper_1506_08481_b300 import params
    sp = params.choose(cfg.L, cfg.N, 3e-11, M_max=192, a_eff=params.effective_radius(cfg.rad), precision=1)
    out = {}
    for prec in (1, 2):
        ctx = make_ctx(sp.xi, sp.M, sp.P, sp.rc, cfg, precision=prec)
        ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
        out[prec] = gpu_apply(ctx, x)
    assert rel(out[2], out[1]) <= 1e-12
    rows = np.random.default_rng(0).choice(cfg.N, 16, replace=False)
    ref = oracle_mod.mobility(cfg.pos, cfg.rad, cfg.L, x12, rows=rows, tol=1e-13)[:, :11]
    assert rel(out[2][rows], ref) <= 1e-9



@pytest.mark.parametrize("ncomp", [3, 6, 11, 12])
def test_wave_space_approach_ncomp_and_split(small_poly, small_poly_ref, ncomp):
    """SE_OPT_SIZE_MODE 2 (source and target Faxen operators in wave space) for every
    ncomp prefix, on a grid whose spreading tiles are split over several CTAs (M = 48)
    and one that is not (M = 144): equal to the hybrid approach to their method errors,
    and to the FP64 oracle to 1e-9."""
    cfg, x = small_poly
    for M, P in ((144, 24), (48, 20)):          # tiles not split / split over CTAs
        ctx = make_ctx(1.0, M, P, 5.45, cfg, precision=1, size_mode=2)
        y = gpu_apply(ctx, x[:, :ncomp].copy())
        ctx2 = make_ctx(1.0, M, P, 5.45, cfg, precision=1, size_mode=0)
        y0 = gpu_apply(ctx2, x[:, :ncomp].copy())
        assert rel(y, y0) <= 1e-7, (M, P)
        if ncomp == 12 and M == 144:
            assert rel(y, small_poly_ref) <= 1e-9
