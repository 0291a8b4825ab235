"""Host-side tests (no GPU): the C ABI library exports every declared entry point,
the Spectral Ewald parameter logic, the normalisation facts the k-space scaling
relies on, and the input generators."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_1506_08481_b300 import api, inputs, params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "se_mobility.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char \*)\s*\*?\s*(se_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol():
    if not os.path.exists(api.LIB_PATH):
        from paper_1506_08481_b300 import build
        build.build()
    lib = ctypes.CDLL(api.LIB_PATH)
    declared = _declared_symbols()
    assert set(declared) == set(api.ABI_SYMBOLS)
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_constants_match_the_header():
    """Every option, precision, preconditioner, stage and error code the header defines has
    the same value in the binding (the binding passes them through as plain integers)."""
    src = open(os.path.join(ROOT, "include", "se_mobility.h")).read()
    defs = dict((k, int(v)) for k, v in re.findall(r"^#define\s+(SE_[A-Z0-9_]+)\s+(-?\d+)\b", src, re.M))
    assert len(defs) > 30
    missing = [k for k in defs if k.startswith("SE_OPT_") and not hasattr(api, k)]
    assert not missing, missing
    for k, v in defs.items():
        if hasattr(api, k):
            assert getattr(api, k) == v, k


def test_theta_parameterisation_edge_value():
    """Eq. theta-param: with theta = (2 pi P xi/(M m))^2 the Gaussian of Eq. shape has the
    value exp(-m^2/2) at |t| = P/(2M); in grid units exp(-alpha s^2), alpha = 2 m^2/P^2."""
    for P, M, xi, L, m in [(16, 32, 0.8, 12.8, 7.1), (24, 384, 0.5, 123.0, 8.7), (9, 64, 0.1, 23.5, 5.3)]:
        sp = params.SeParams(xi=xi, M=M, P=P, rc=1.0, m=m)
        theta = sp.theta()
        t = P / (2.0 * M)
        h_edge = math.exp(-8 * math.pi ** 2 * xi ** 2 * t ** 2 / theta)       # Eq. shape
        assert abs(h_edge - math.exp(-m * m / 2)) < 1e-12 * math.exp(-m * m / 2) + 1e-300
        assert abs(math.exp(-sp.alpha * (P / 2) ** 2) - h_edge) < 1e-12 * h_edge
        # the grid-unit Gaussian is Eq. shape's exponent with t = s / M
        s = 1.7
        assert abs(sp.alpha * s * s - 8 * math.pi ** 2 * xi ** 2 * (s / M) ** 2 / theta) < 1e-12


def test_gaussian_fourier_pair_on_the_grid():
    """Eq. shape / Eq. parseval: the sum of the P-point truncated Gaussian on the grid is,
    by Poisson summation, sum_k ghat(q/M + k) exp(-2 pi i (q/M + k) u) with
    ghat(nu) = (pi/alpha)^(1/2) exp(-pi^2 nu^2/alpha), up to the truncation error
    exp(-m^2/2) = exp(-P pi/2) at m = sqrt(pi P) (Eq. error-scale).  This fixes the
    per-dimension normalisation (alpha/pi)^(1/2) that the k-space scaling divides out
    twice; the aliases k != 0 are the resolution error, suppressed by the kernel's own
    decay near the Nyquist frequency."""
    M, P = 64, 24
    m = math.sqrt(math.pi * P)
    alpha = 2 * m * m / P ** 2
    u = 17.37
    b = math.floor(u - P / 2) + 1
    n = b + np.arange(P)
    g = np.exp(-alpha * (n - u) ** 2)
    ghat = lambda nu: math.sqrt(math.pi / alpha) * math.exp(-math.pi ** 2 * nu * nu / alpha)
    for q in range(-M // 2 + 1, M // 2):
        nu = q / M
        lhs = np.sum(g * np.exp(-2j * math.pi * nu * n))
        rhs = sum(ghat(nu + k) * np.exp(-2j * math.pi * (nu + k) * u) for k in range(-3, 4))
        assert abs(lhs - rhs) < 10 * math.exp(-P * math.pi / 2) + 1e-13   # truncation + rounding
        if abs(nu) <= 0.25:     # aliases small: exp(-pi^2 (1 - 2|nu|)/alpha) relative
            assert abs(lhs - ghat(nu) * np.exp(-2j * math.pi * nu * u)) <= 2 * math.exp(-math.pi ** 2 * (1 - 2 * abs(nu)) / alpha) * ghat(nu) + 1e-13


def test_fast_gaussian_gridding_identity():
    """Eq. fgg-exp: exp(-a (d + i D)^2) = exp(-a d^2) exp(-2 a d D)^i exp(-a D^2)^(i^2)."""
    a, D = 0.37, 1.0
    for d in (-0.5, -0.13, 0.0, 0.41):
        for i in range(-12, 13):
            lhs = math.exp(-a * (d + i * D) ** 2)
            rhs = math.exp(-a * d * d) * math.exp(-2 * a * d * D) ** i * math.exp(-a * D * D) ** (i * i)
            assert abs(lhs - rhs) <= 1e-12 * max(lhs, 1e-300)


def test_parameter_choice_respects_constraints():
    for L, N, tol in [(12.79, 100, 1e-10), (50.1, 2000, 1e-6), (123.0, 200000, 1e-6), (61.8, 20000, 1e-4)]:
        sp = params.choose(L, N, tol, M_max=384)
        assert sp.rc < L / 2
        assert sp.M in params.fft_sizes()
        assert sp.P * sp.xi * L <= sp.M * sp.m * (1 + 1e-12)           # no k-space amplification
        assert params.error_estimate(L, sp.xi, sp.M, sp.P, sp.rc, sp.m) <= tol * (1 + 1e-9)
        assert math.exp(-(math.pi * sp.M / L) ** 2 / (4 * sp.xi ** 2)) < tol   # wave-space truncation
    assert params.support_for(1e-4) <= 12 and params.support_for(1e-10) >= 16


def test_fft_sizes_are_supported_by_the_library():
    for M in params.fft_sizes():
        r = M
        while r % 2 == 0:
            r //= 2
        while r % 3 == 0:
            r //= 3
        assert r == 1 and M % 8 == 0


@pytest.mark.parametrize("maker", [inputs.mono_n100, lambda: inputs.bidisperse(n=400, phi=0.3)])
def test_generators_non_overlapping_and_volume_fraction(maker):
    c = maker()
    assert inputs.min_gap(c.pos, c.rad, c.L) >= 0
    assert np.all((c.pos >= 0) & (c.pos < c.L))


def test_dense_generator_at_phi_045():
    c = inputs.mono_dense(n=4000, phi=0.45)
    assert abs(c.phi - 0.45) < 1e-9
    assert inputs.min_gap(c.pos, c.rad, c.L) >= 0


def test_lognormal_radii_moments():
    r = inputs.radii_lognormal(200000, 1.0, 0.2, np.random.default_rng(0))
    assert abs(r.mean() - 1.0) < 3e-3 and abs(r.std() - 0.2) < 3e-3
