"""Pins of oracle/brownian.py (the Swan-Brady initial value problem for A^{-1/2} c,
Sec. 4.3, Eqs. ivp-1, ivp-forward, ivp-backward) against the mathematics: the exact
solution of the scalar problem, A^{-1/2} from the eigendecomposition, second-order
convergence in dtau, and the invariance of the scheme under orthogonal similarity."""
import numpy as np
import pytest

from oracle import brownian


def test_identity_is_exact():
    c = np.random.default_rng(0).standard_normal(7)
    for n in (1, 3, 10):
        np.testing.assert_allclose(brownian.ivp_inv_sqrt(np.eye(7), c, n), c, rtol=0, atol=1e-15)


@pytest.mark.parametrize("lam", [0.04, 0.5, 3.0, 25.0])
def test_scalar_converges_to_the_exact_solution(lam):
    """For A = lam the IVP has the closed-form solution x(tau) = c sqrt((lam + tau (1 - lam))/lam),
    so x(1) = lam^{-1/2} c; the half-step pair is second order in dtau."""
    exact = lam ** -0.5
    errs = [abs(brownian.ivp_inv_sqrt(np.array([[lam]]), np.array([1.0]), n)[0] - exact) for n in (20, 40, 80, 160)]
    assert errs[-1] < 1e-3 * exact
    for e0, e1 in zip(errs, errs[1:]):
        assert 3.0 < e0 / e1 < 4.3, errs
    assert 3.7 < errs[-2] / errs[-1] < 4.3, errs        # asymptotically second order


def test_dense_spd_converges_to_the_inverse_square_root():
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((9, 9)))
    lam = np.geomspace(0.05, 20.0, 9)
    A = Q @ np.diag(lam) @ Q.T
    c = rng.standard_normal(9)
    ref = Q @ ((Q.T @ c) / np.sqrt(lam))
    np.testing.assert_allclose(brownian.inv_sqrt(A, c), ref, rtol=1e-12, atol=1e-12)
    errs = [np.linalg.norm(brownian.ivp_inv_sqrt(A, c, n) - ref) / np.linalg.norm(ref) for n in (20, 40, 80)]
    assert errs[-1] < 2e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_orthogonal_similarity_invariance():
    """The scheme uses only rational functions of A: ivp(Q D Q^T, c) = Q ivp(D, Q^T c)."""
    rng = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    D = np.diag(np.geomspace(0.1, 8.0, 6))
    c = rng.standard_normal(6)
    a = brownian.ivp_inv_sqrt(Q @ D @ Q.T, c, 10)
    b = Q @ brownian.ivp_inv_sqrt(D, Q.T @ c, 10)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)
    # and for diagonal A every component follows its own scalar problem
    for k in range(6):
        e = np.zeros(6)
        e[k] = c[k]
        np.testing.assert_allclose(brownian.ivp_inv_sqrt(D, e, 10)[k],
                                   brownian.ivp_inv_sqrt(D[k:k + 1, k:k + 1], c[k:k + 1], 10)[0], rtol=1e-14)
