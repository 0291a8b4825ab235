"""FP64 reference of the rigid-particle far-field mobility and the self-diffusivity
estimator (test infrastructure).

Sec. 6.1 defines the short-time self-diffusivities through the diagonal blocks mu_ii of
R_FU^{-1} (Eq. dstr-def); with far-field interactions only the grand resistance is the
inverse of the F, T, S grand mobility M, and the rigid spheres' (U, Omega) follow from
(F, T) with the strain rate E = 0.  The estimator of the paper (after Sierou & Brady)
averages (U^R, Omega^R)(F^R, T^R) over random (F^R, T^R) of unit covariance, which tends to
diag(mu).  Everything here is dense numpy on the oracle's matrix (oracle.dense_matrix with
ncomp = 11), written from those definitions; it shares no code with the CUDA path.
The high-frequency shear viscosity (the eta_s of Eq. dst-corr) follows from the same
resistance with forces and torques zero and a strain imposed.  Pinned in
tests/test_diffusivity_oracle.py.
"""
import numpy as np

NC = 11


def _ft_index(N):
    return np.array([11 * i + c for i in range(N) for c in range(6)])


def _s_index(N):
    return np.array([11 * i + 6 + c for i in range(N) for c in range(5)])


def rigid_mobility(M11):
    """mu = (R_FU)^{-1} with R = M11^{-1}, on the (F, T) components: [6N, 6N]."""
    M11 = np.asarray(M11, dtype=np.float64)
    N = M11.shape[0] // NC
    R = np.linalg.inv(M11)
    ft = _ft_index(N)
    return np.linalg.inv(R[np.ix_(ft, ft)])


def rigid_response(M11, ft_vec):
    """(U, Omega) [N, 6] and S [N, 5] for forces and torques ft_vec [N, 6], E = 0:
    (U, Omega) = mu (F, T), and S from the resistance relation S = R_SU (U, Omega)."""
    M11 = np.asarray(M11, dtype=np.float64)
    N = M11.shape[0] // NC
    R = np.linalg.inv(M11)
    ft, si = _ft_index(N), _s_index(N)
    uw = np.linalg.solve(R[np.ix_(ft, ft)], np.asarray(ft_vec, dtype=np.float64).reshape(-1))
    s = R[np.ix_(si, ft)] @ uw
    return uw.reshape(N, 6), s.reshape(N, 5)


def rigid_response_strain(M11, e):
    """(U, Omega) [N, 6] and S [N, 5] of force- and torque-free rigid spheres in the
    imposed strain rate e (5 numbers on the orthonormal basis): with R = M11^{-1},
    [F; S] = R [U; E] and F = 0 give R_FU U = -R_FE E, then S = R_SU U + R_SE E."""
    M11 = np.asarray(M11, dtype=np.float64)
    N = M11.shape[0] // NC
    R = np.linalg.inv(M11)
    ft, si = _ft_index(N), _s_index(N)
    E = np.tile(np.asarray(e, dtype=np.float64), N)
    uw = np.linalg.solve(R[np.ix_(ft, ft)], -R[np.ix_(ft, si)] @ E)
    s = R[np.ix_(si, ft)] @ uw + R[np.ix_(si, si)] @ E
    return uw.reshape(N, 6), s.reshape(N, 5)


def viscosity_ratio(M11, L, eta=1.0):
    """eta_s / eta: particle stress n <S> of force- and torque-free rigid spheres in each
    orthonormal basis strain e_k, (sum_i S_i . e_k) / (2 eta V), averaged over k."""
    acc = 0.0
    for k in range(5):
        e = np.zeros(5)
        e[k] = 1.0
        _, s = rigid_response_strain(M11, e)
        acc += s[:, k].sum() / (2 * eta * L ** 3)
    return 1.0 + acc / 5


def diag_traces(mu):
    """Per particle (tr mu_ii^tt / 3, tr mu_ii^rr / 3): [N, 2]."""
    N = mu.shape[0] // 6
    out = np.zeros((N, 2))
    for i in range(N):
        b = mu[6 * i:6 * i + 6, 6 * i:6 * i + 6]
        out[i] = (np.trace(b[:3, :3]) / 3, np.trace(b[3:, 3:]) / 3)
    return out


def estimate(mu, fr):
    """The estimator on the given samples fr [nsamples, N, 6]: per particle the sample
    mean of (U . F)/3 and (Omega . T)/3 with (U, Omega) = mu (F, T)."""
    fr = np.asarray(fr, dtype=np.float64)
    ns, N = fr.shape[0], fr.shape[1]
    acc = np.zeros((N, 2))
    for k in range(ns):
        uw = (mu @ fr[k].reshape(-1)).reshape(N, 6)
        acc[:, 0] += np.sum(uw[:, :3] * fr[k, :, :3], axis=1) / 3
        acc[:, 1] += np.sum(uw[:, 3:] * fr[k, :, 3:], axis=1) / 3
    return acc / ns
