"""Host-side choice of the Ewald / Spectral Ewald parameters (xi, M, P, rc, m).

Error model (Sec. 5.1):
  real space   truncated beyond rc:            ~ exp(-(xi rc)^2)
  wave space   truncated at |k| = pi M / L:     ~ exp(-(pi M / L)^2 / (4 xi^2))
  SE support   Gaussian resolution/truncation:  ~ exp(-P pi / 2) at m = sqrt(pi P) (Eq. error-scale)
The net k-space factor exp(theta q^2/(4 xi^2) - k^2/(4 xi^2)) of Eq. wave-result
never amplifies (rounding noise stays at working precision) iff P xi L <= M m.
Cost model: real-space pairs ~ N n (4 pi/3) rc^3, grid ~ M^3 log M, support ~ N P^3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass


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


def support_for(tol: float) -> int:
    """Smallest even P with exp(-P pi / 2) <= tol (Eq. error-scale)."""
    P = int(math.ceil(2.0 * math.log(1.0 / tol) / math.pi))
    return max(4, P + (P % 2))


def choose(L: float, N: int, tol: float, P: int | None = None, M_max: int = 384,
           rc_max: float | None = None) -> SeParams:
    """Cheapest (xi, M, rc) meeting the error model at relative accuracy tol."""
    c = math.sqrt(math.log(1.0 / tol)) + 0.5
    if P is None:
        P = support_for(tol)
    m = math.sqrt(math.pi * P)
    n = N / L ** 3
    rc_lim = 0.5 * L * 0.999 if rc_max is None else min(rc_max, 0.5 * L * 0.999)
    best = None
    for M in fft_sizes(16, M_max):
        if P > M - 8:
            continue
        # largest xi the grid resolves, and the non-amplification bound
        xi = min(math.pi * M / L / (2.0 * c), M * m / (P * L))
        rc = c / xi
        if rc > rc_lim:
            continue
        cost = 2.0e2 * N * n * 4.0 / 3.0 * math.pi * rc ** 3 + 60.0 * M ** 3 * math.log2(M) + 40.0 * N * P ** 3
        if best is None or cost < best[0]:
            best = (cost, SeParams(xi=xi, M=M, P=P, rc=rc, m=m))
    if best is None:
        raise ValueError("no grid up to M_max meets the accuracy with rc < L/2")
    return best[1]
