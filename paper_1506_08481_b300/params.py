"""Host-side choice of the Ewald / Spectral Ewald parameters (xi, M, P, rc, m).

Error model (relative 2-norm of the product, conservative by a factor 2-10 against the
FP64 oracle on the measured configurations):
  real space   pairs beyond rc dropped:        exp(-(xi rc)^2) f_r            (Eq. oseen-ewald-rs)
  truncation   Gaussian cut at |s| = P/2:       exp(-m^2/2) f_w                (Eq. theta-param)
  resolution   the grid aliases of the Gaussian, ghat(nu -+ 1)/ghat(nu) = exp(-A (1 - 2|nu|)),
               weighted by the kernel decay exp(-B nu^2) of the mode nu = q/M:
                 max_nu exp(-A (1 - 2 nu) - B nu^2) f_w,  A = pi^2 P^2/(2 m^2),  B = (pi M/(xi L))^2
               (its nu = 1/2 value exp(-B/4) is the wave-space truncation of Eq. oseen-ewald-ws)
The factors carry the derivatives that the torque, stresslet and Faxen terms put on
the kernels (Eq. mul-expand: up to two Laplacians and two gradients of J), which
multiply each truncated tail by powers of the wave number or of 1/r:
  f_r = 1 + 0.1 (a xi)^4 (xi rc)^6,    f_w = 1 + 0.25 (a xi)^8 E_w^6,   E_w = pi M/(2 xi L),
with a the effective radius <a^8>^(1/8) (fitted to the oracle's real- and wave-space
truncation errors of mono-, bi- and polydisperse suspensions, 12 components).
FP32 products add a rounding floor 3e-7 (1 + R): the wave grids carry each particle's
own wave-space self term, which the FP64 self correction cancels (Eq. uf-self and its
torque/stresslet analogues); R = (20/3) (a xi)^3 (25 - 42 (a xi)^2 + 27 (a xi)^4) / (50 pi^(1/2))
is the ratio of that stresslet self term to the isolated-sphere stresslet mobility
3/(20 pi eta a^3), so the FP32 error grows with a xi and the choice keeps a xi near 1.
The net k-space factor exp(theta q^2/(4 xi^2) - k^2/(4 xi^2)) of Eq. wave-result never
amplifies (rounding noise stays at working precision) iff P xi L <= M m.
Cost model (relative device time of this library's kernels): real-space pairs
N n (4 pi/3) rc^3, plus 0.5 M^3 log2 M for the FFT chain, plus 0.1 N P^3 for spread + gather.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# prefactor between the model and the measured relative 2-norm error
ERROR_PREFACTOR = 1.0

# The large-scale monodisperse workload: N = 200000 spheres of radius 1 at phi = 0.45
# (box side L = 123.018), all 12 components, support P = 24, real-space size approach.
# The FP32 rounding of the wave-space part grows with the sharpness of the window on
# the grid, kappa sqrt(alpha) ~ M m / (L P) (the gather's derivative weights amplify the
# grid's rounding noise; measured: E block 1.2e-6 at M = 216, m = 8.68, 6.8e-7 at M = 144,
# m = 8), so the grid is the coarsest that resolves the wave-space sum at this support:
# xi = 0.45 (the method error, FP64, ~1e-7), rc = 10 for the real-space truncation.
LARGE_MONO = dict(xi=0.45, M=144, P=24, rc=10.0, m=8.0, size_mode=1)


@dataclass
class SeParams:
    xi: float
    M: int
    P: int
    rc: float
    m: float

    @property
    def alpha(self) -> float:
        """Gaussian exp(-alpha s^2) in grid units (edge value exp(-m^2/2) at s = P/2)."""
        return 2.0 * self.m ** 2 / self.P ** 2

    def theta(self) -> float:
        """theta of Eq. theta-param."""
        return (2.0 * math.pi * self.P * self.xi / (self.M * self.m)) ** 2


def fft_sizes(lo: int = 8, hi: int = 512) -> list[int]:
    """Grid sizes supported by the FFT: 2^a 3^b, multiples of 8."""
    out = []
    for a in range(3, 10):
        for b in range(0, 6):
            v = 2 ** a * 3 ** b
            if lo <= v <= hi:
                out.append(v)
    return sorted(out)


def effective_radius(rad) -> float:
    """<a^8>^(1/8), the radius that sets the size factors of the error model."""
    r = np.asarray(rad, dtype=np.float64)
    return float(np.mean(r ** 8) ** 0.125)


def resolution_exponent(P: int, m, M: int, xi, L: float):
    """min over modes of A (1 - 2 nu) + B nu^2 (the resolution error is exp(-this))."""
    A = math.pi ** 2 * P ** 2 / (2.0 * np.asarray(m) ** 2)
    B = (math.pi * M / (np.asarray(xi) * L)) ** 2
    return np.where(A / B >= 0.5, B / 4.0, A - A * A / B)


def _f_real(a, xi, Er):
    return 1.0 + 0.1 * (a * xi) ** 4 * Er ** 6


def _f_wave(a, xi, M, L):
    Ew = math.pi * M / (2.0 * xi * L)
    return 1.0 + 0.25 * (a * xi) ** 8 * Ew ** 6


FP32_FLOOR = 3e-7


def self_ratio(axi):
    """Wave-space stresslet self term over the isolated-sphere stresslet mobility at a xi."""
    axi = np.asarray(axi, dtype=np.float64)
    return axi ** 3 * (25.0 - 42.0 * axi ** 2 + 27.0 * axi ** 4) * (20.0 / 3.0) / (50.0 * math.sqrt(math.pi))


def _e32(a, xi):
    return FP32_FLOOR * (1.0 + self_ratio(a * xi))


def error_terms(L: float, xi: float, M: int, P: int, rc: float, m: float, a_eff: float = 1.0,
                precision: int = 1) -> dict:
    """The modelled error terms (relative); precision 0 adds the FP32 rounding floor."""
    fw = _f_wave(a_eff, xi, M, L)
    t = {"real": ERROR_PREFACTOR * math.exp(-(xi * rc) ** 2) * _f_real(a_eff, xi, xi * rc),
         "truncation": ERROR_PREFACTOR * math.exp(-m * m / 2.0) * fw,
         "resolution": ERROR_PREFACTOR * float(np.exp(-resolution_exponent(P, m, M, xi, L))) * fw}
    if precision == 0:
        t["fp32"] = float(_e32(a_eff, xi))
    return t


def error_estimate(L: float, xi: float, M: int, P: int, rc: float, m: float, a_eff: float = 1.0,
                   precision: int = 1) -> float:
    """Model of the relative error of the product."""
    return max(error_terms(L, xi, M, P, rc, m, a_eff, precision).values())


def support_for(tol: float) -> int:
    """Smallest even P with exp(-P pi / 2) <= tol / C (Eq. error-scale)."""
    P = int(math.ceil(2.0 * math.log(ERROR_PREFACTOR / tol) / math.pi))
    return max(4, P + (P % 2))


def _rc_for(tol: float, a: float, xi: float) -> float:
    """Smallest rc with the real-space term <= tol (bisection on xi rc)."""
    lo, hi = 0.0, 12.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if ERROR_PREFACTOR * math.exp(-mid * mid) * _f_real(a, xi, mid) <= tol:
            hi = mid
        else:
            lo = mid
    return hi / xi


def choose(L: float, N: int, tol: float, P: int | None = None, M_max: int = 384,
           rc_max: float | None = None, M_min: int = 16, a_eff: float = 1.0,
           precision: int = 1, fp32_tol: float | None = None) -> SeParams:
    """Cheapest (xi, M, P, m, rc) whose modelled error is <= tol; a_eff is the effective
    radius of the suspension (effective_radius), precision 0 for FP32 products.  fp32_tol
    bounds the FP32 rounding floor separately (a solve whose Krylov products run in FP32
    and whose residual runs in FP64 needs tol for the method and fp32_tol for FP32)."""
    if precision == 0 and fp32_tol is None:
        fp32_tol = tol
    supports = [P] if P is not None else list(range(support_for(tol), 33, 2))
    n = N / L ** 3
    rc_lim = 0.499 * L if rc_max is None else min(rc_max, 0.499 * L)
    ms = 3.0 + 0.075 * np.arange(121)
    best = None
    for P in supports:
        for M in fft_sizes(M_min, M_max):
            if P > M - 8:
                continue
            # largest xi per m meeting the wave-space terms (all grow with xi): bisection
            lo = np.full_like(ms, 1e-3)
            hi = M * ms / (P * L)                   # no k-space amplification
            def ok(xi):
                fw = _f_wave(a_eff, xi, M, L)
                e = np.maximum(np.exp(-ms * ms / 2.0), np.exp(-resolution_exponent(P, ms, M, xi, L)))
                good = ERROR_PREFACTOR * e * fw <= tol
                if fp32_tol is not None:
                    good &= _e32(a_eff, xi) <= fp32_tol
                return good
            good_hi = ok(hi)
            for _ in range(50):
                mid = 0.5 * (lo + hi)
                g = ok(mid)
                lo = np.where(g, mid, lo)
                hi = np.where(g, hi, mid)
            xi_m = np.where(good_hi, M * ms / (P * L), lo)
            feasible = ok(xi_m)
            for xi, m, f in zip(xi_m, ms, feasible):
                if not f:
                    continue
                rc = _rc_for(tol, a_eff, float(xi))
                if rc > rc_lim:
                    continue
                cost = N * n * 4.0 / 3.0 * math.pi * rc ** 3 + 0.5 * M ** 3 * math.log2(M) + 0.1 * N * P ** 3
                if best is None or cost < best[0]:
                    best = (cost, SeParams(xi=float(xi), M=M, P=P, rc=rc, m=float(m)))
    if best is None:
        raise ValueError("no grid up to M_max meets the accuracy with rc < L/2")
    return best[1]


def candidates(L: float, N: int, tol: float, M_max: int = 384, supports=None, a_eff: float = 1.0,
               precision: int = 1) -> list[SeParams]:
    """Distinct parameter sets meeting the error model at tol: the cheapest per grid size
    for each support."""
    out, seen = [], set()
    for P in (supports or [None]):
        for M in fft_sizes(16, M_max):
            try:
                sp = choose(L, N, tol, P=P, M_max=M, M_min=M, a_eff=a_eff, precision=precision)
            except ValueError:
                continue
            key = (sp.M, sp.P)
            if key not in seen:
                seen.add(key)
                out.append(sp)
    return out


def autotune(cfg, tol: float, ncomp: int = 3, precision: int = 0, max_candidates: int = 3, reps: int = 3,
             supports=None, fp32_tol: float | None = None, spreads=(0, 1, 2), modes=(1, 0)):
    """Time the cheapest few candidate parameter sets for a configuration on the GPU, each
    with the particle-size modes `modes` and the spreading tile shapes `spreads`
    (SE_OPT_SPREAD 0: one-warp 8 x 4 x 16 blocks where the grid has room, 1: 8^3 tiles, 2: two-warp
    8 x 8 x 16 tiles), and return
    (SeParams, size_mode, ms per product, {"spread": tile option}) of the fastest.  The
    candidates meet the error model at tol (method) and fp32_tol (FP32 rounding)."""
    import torch
    from . import api
    a_eff = effective_radius(cfg.rad)
    out, seen = [], set()
    for M in fft_sizes(16, 384):
        try:
            sp = choose(cfg.L, cfg.N, tol, P=None, M_max=M, M_min=M, a_eff=a_eff, precision=precision,
                        fp32_tol=fp32_tol)
        except ValueError:
            continue
        if (sp.M, sp.P) not in seen:
            seen.add((sp.M, sp.P))
            out.append(sp)
    cands = sorted(out, key=lambda s: s.M ** 3 * math.log2(s.M) * 0.5 + 0.1 * cfg.N * s.P ** 3
                   + cfg.N ** 2 / cfg.L ** 3 * 4.19 * s.rc ** 3)[:max_candidates]
    x = torch.randn(cfg.N, ncomp, device="cuda", dtype=torch.float32 if precision == 0 else torch.float64)
    y = torch.empty_like(x)
    best = None
    for sp in cands:
        for mode in modes:
            ctx = api.Context()
            ctx.set_params(sp.xi, sp.M, sp.P, sp.rc)
            ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
            ctx.set_option(api.SE_OPT_SIZE_MODE, mode)
            ctx.set_option(api.SE_OPT_PRECISION, precision)
            ctx.set_config(cfg.pos, cfg.rad, cfg.L)
            for spread in spreads:
                ctx.set_option(api.SE_OPT_SPREAD, spread)
                ctx.apply(x, y)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                for _ in range(reps):
                    ctx.apply(x, y)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                if best is None or ms < best[2]:
                    best = (sp, mode, ms, {"spread": spread})
            ctx.close()
    return best
