"""Host-side choice of the Ewald / Spectral Ewald parameters (xi, M, P, rc, m).

Error model (relative, up to a prefactor C calibrated against the oracle):
  real space   pairs beyond rc dropped:        exp(-(xi rc)^2)                (Eq. oseen-ewald-rs)
  truncation   Gaussian cut at |s| = P/2:       exp(-m^2/2)                   (Eq. theta-param)
  resolution   the grid aliases of the Gaussian, ghat(nu -+ 1)/ghat(nu) = exp(-A (1 - 2|nu|)),
               weighted by the kernel decay exp(-B nu^2) of the mode nu = q/M:
                 max_nu exp(-A (1 - 2 nu) - B nu^2),  A = pi^2 P^2/(2 m^2),  B = (pi M/(xi L))^2
               (its nu = 1/2 value exp(-B/4) is the wave-space truncation of Eq. oseen-ewald-ws)
With m = sqrt(pi P) the truncation is exp(-P pi/2), the minimum error of Eq. error-scale.
The net k-space factor exp(theta q^2/(4 xi^2) - k^2/(4 xi^2)) of Eq. wave-result never
amplifies (rounding noise stays at working precision) iff P xi L <= M m.
Cost model (relative device time of this library's kernels): real-space pairs
N n (4 pi/3) rc^3, plus 0.5 M^3 log2 M for the FFT chain, plus 0.1 N P^3 for spread + gather.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

# prefactor between the exponential model and the measured relative 2-norm error
ERROR_PREFACTOR = 100.0


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


def resolution_exponent(P: int, m: float, M: int, xi: float, L: float) -> float:
    """min over modes of A (1 - 2 nu) + B nu^2 (the resolution error is exp(-this))."""
    A = math.pi ** 2 * P ** 2 / (2.0 * m * m)
    B = (math.pi * M / (xi * L)) ** 2
    nu = A / B
    return B / 4.0 if nu >= 0.5 else A - A * A / B


def error_estimate(L: float, xi: float, M: int, P: int, rc: float, m: float) -> float:
    """Model of the relative error of the product."""
    e = max(math.exp(-(xi * rc) ** 2), math.exp(-m * m / 2.0),
            math.exp(-resolution_exponent(P, m, M, xi, L)))
    return ERROR_PREFACTOR * e


def support_for(tol: float) -> int:
    """Smallest even P with exp(-P pi / 2) <= tol / C (Eq. error-scale)."""
    P = int(math.ceil(2.0 * math.log(ERROR_PREFACTOR / tol) / math.pi))
    return max(4, P + (P % 2))


def choose(L: float, N: int, tol: float, P: int | None = None, M_max: int = 384,
           rc_max: float | None = None, M_min: int = 16) -> SeParams:
    """Cheapest (xi, M, m, rc) whose modelled error is <= tol."""
    E = math.log(ERROR_PREFACTOR / tol)
    supports = [P] if P is not None else list(range(support_for(tol), 33, 2))
    n = N / L ** 3
    rc_lim = 0.499 * L if rc_max is None else min(rc_max, 0.499 * L)
    best = None
    for P, M, i in ((P, M, i) for P in supports for M in fft_sizes(M_min, M_max) for i in range(121)):
        if P > M - 8:
            continue
        if True:
            m = 3.0 + 0.075 * i
            if m * m / 2.0 < E:
                continue
            A = math.pi ** 2 * P ** 2 / (2.0 * m * m)
            if A <= E:
                continue
            # largest xi meeting the resolution bound (both branches of the minimum)
            xi_res = math.pi * M * math.sqrt(A - E) / (L * A)
            if A >= (math.pi * M / (xi_res * L)) ** 2 / 2.0:
                xi_res = math.pi * M / (2.0 * L * math.sqrt(E))
            xi = min(xi_res, M * m / (P * L))          # no k-space amplification
            rc = math.sqrt(E) / xi
            if rc > rc_lim or resolution_exponent(P, m, M, xi, L) < E * (1 - 1e-9):
                continue
            cost = N * n * 4.0 / 3.0 * math.pi * rc ** 3 + 0.5 * M ** 3 * math.log2(M) + 0.1 * N * P ** 3
            if best is None or cost < best[0]:
                best = (cost, SeParams(xi=xi, M=M, P=P, rc=rc, m=m))
    if best is None:
        raise ValueError("no grid up to M_max meets the accuracy with rc < L/2")
    return best[1]


def candidates(L: float, N: int, tol: float, M_max: int = 384, supports=None) -> list[SeParams]:
    """Distinct parameter sets meeting the error model at tol: the cheapest per grid size
    for each support."""
    out, seen = [], set()
    for P in (supports or [None]):
        for M in fft_sizes(16, M_max):
            try:
                sp = choose(L, N, tol, P=P, M_max=M, M_min=M)
            except ValueError:
                continue
            key = (sp.M, sp.P)
            if key not in seen:
                seen.add(key)
                out.append(sp)
    return out


def autotune(cfg, tol: float, ncomp: int = 3, precision: int = 0, max_candidates: int = 4, reps: int = 3,
             supports=None):
    """Time the cheapest few candidate parameter sets (and both particle-size modes) for a
    configuration on the GPU and return (SeParams, size_mode, ms per product) of the fastest."""
    import torch
    from . import api
    cands = sorted(candidates(cfg.L, cfg.N, tol, supports=supports),
                   key=lambda s: s.M ** 3 * math.log2(s.M) * 0.5 + 0.1 * cfg.N * s.P ** 3
                   + cfg.N ** 2 / cfg.L ** 3 * 4.19 * s.rc ** 3)[:max_candidates]
    x = torch.randn(cfg.N, ncomp, device="cuda", dtype=torch.float32 if precision == 0 else torch.float64)
    y = torch.empty_like(x)
    best = None
    for sp in cands:
        for mode in (1, 0):
            ctx = api.Context()
            ctx.set_params(sp.xi, sp.M, sp.P, sp.rc)
            ctx.set_option(api.SE_OPT_SHAPE_M, sp.m)
            ctx.set_option(api.SE_OPT_SIZE_MODE, mode)
            ctx.set_option(api.SE_OPT_PRECISION, precision)
            ctx.set_config(cfg.pos, cfg.rad, cfg.L)
            ctx.apply(x, y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                ctx.apply(x, y)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            ctx.close()
            if best is None or ms < best[2]:
                best = (sp, mode, ms)
    return best
