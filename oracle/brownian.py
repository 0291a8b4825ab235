"""FP64 reference of the far-field Brownian source M^{-1/2} c (test infrastructure).

Sec. 4.3 of the paper obtains the far-field Brownian force from A^{-1/2} Psi (Eq. br-f-ff)
as the value at tau = 1 of the initial value problem (Eq. ivp-1)

    dx/dtau = -1/2 [tau I + (1 - tau) A]^{-1} (A - I) x,   x(0) = c,

marched in steps of dtau, each an explicit Euler half-step (Eq. ivp-forward) followed by
an implicit Euler half-step (Eq. ivp-backward).  ``ivp_inv_sqrt`` takes those steps in
that order on a dense matrix with numpy's dense solver; ``inv_sqrt`` is the definition
of A^{-1/2} c through the eigendecomposition of the symmetric positive definite A.  Plain
numpy, written from the equations; shares no code with the CUDA path.  Pinned in
tests/test_brownian_oracle.py: A = I, the scalar recurrence in closed form, second-order
convergence to inv_sqrt as dtau -> 0, and the similarity invariance of the scheme.
"""
import numpy as np


def inv_sqrt(A, c):
    """A^{-1/2} c for symmetric positive definite A (eigendecomposition)."""
    A = np.asarray(A, dtype=np.float64)
    lam, V = np.linalg.eigh(0.5 * (A + A.T))
    if lam.min() <= 0:
        raise ValueError("A is not positive definite")
    return V @ ((V.T @ np.asarray(c, dtype=np.float64)) / np.sqrt(lam))


def ivp_inv_sqrt(A, c, nsteps):
    """x(1) of Eq. ivp-1 by nsteps steps of Eqs. ivp-forward and ivp-backward."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    eye = np.eye(n)
    x = np.array(c, dtype=np.float64)
    dtau = 1.0 / nsteps
    for i in range(nsteps):
        tau_i, tau_next = i * dtau, (i + 1) * dtau
        # Eq. ivp-forward: (x_{i+1/2} - x_i) / (dtau/2) = -1/2 B(tau_i)^{-1} (A - I) x_i
        B = tau_i * eye + (1 - tau_i) * A
        x_half = x - 0.25 * dtau * np.linalg.solve(B, (A - eye) @ x)
        # Eq. ivp-backward: (x_{i+1} - x_{i+1/2}) / (dtau/2) = -1/2 B(tau_{i+1})^{-1} (A - I) x_{i+1},
        # i.e. [B(tau_{i+1}) + (dtau/4)(A - I)] x_{i+1} = B(tau_{i+1}) x_{i+1/2}
        B = tau_next * eye + (1 - tau_next) * A
        x = np.linalg.solve(B + 0.25 * dtau * (A - eye), B @ x_half)
    return x
