// Real-space part of the grand-mobility product (Sec. 3.3): for each particle i,
// every neighbour j in the 27 surrounding cells with |x| < rc, x = r_i - r_j
// (minimum image; rc < L/2 so each pair has at most one image in range).
//
// The couplings are the Faxen laws (Eqs. faxen-f/t/s/p) applied to the multipole
// velocity field (Eq. mul-expand, Eq. compress-vel-disturb) with the real-space
// Ewald generators psi_R(r) = r erfc(xi r) - exp(-xi^2 r^2)/(xi sqrt pi)
// (Eq. oseen-ewald-rs) and phi_R(r) = erfc(xi r)/r (Eq. source-split).
// With D = (1/r) d/dr, every derivative of a radial function is a contraction of
// x and delta with D^k of it; D psi_R = B_0, D^k psi_R = (-1)^{k-1} B_{k-1},
// D^k phi_R = (-1)^k B_k, where
//   B_0 = erfc(xi r)/r,  B_n = [(2n-1) B_{n-1} + (2 xi^2)^n exp(-xi^2 r^2)/(xi sqrt pi)]/r^2
// (W. Smith's multipole-Ewald recurrence), and D^k Lap g = (2k+3) D^{k+1} g + r^2 D^{k+2} g.
// For a Faxen-weighted generator G = (1 + c1 Lap + c2 Lap^2) psi, G_k = D^k G, and
//   U  <- F : [(2 G1 + r^2 G2) F - x (x.F) G2] / (8 pi eta)        G = f6_i f6_j psi
//   U  <- T : (LG)_1 (x x T) / (16 pi eta)                           G = f6_i psi
//   U  <- S : [-(3 G2 + r^2 G3) S.x + x (x.S.x) G3] / (8 pi eta)      G = f6_i f10_j psi
//   U  <- Str: -x Phi_1 Str / (16 pi eta)                            Phi = f6_i phi
//   Om <- F : (LG)_1 (x x F) / (16 pi eta)                           G = f6_j psi
//   Om <- T : [x (x.T) (Lpsi)_2 - T (2 (Lpsi)_1 + r^2 (Lpsi)_2)] / (32 pi eta)
//   Om <- S : -(LG)_2 x x (S.x) / (16 pi eta)                        G = f10_j psi
//   E  <- F : [(3 G2 + r^2 G3) sym(x F) - G3 (x.F) x x] / (8 pi eta)  G = f10_i f6_j psi
//   E  <- T : (LG)_2 sym(x (x x T)) / (16 pi eta)                    G = f10_i psi
//   E  <- S : -[(3 G2 + r^2 G3) S + (3 G3 + r^2 G4) sym(x S.x) - G4 (x.S.x) x x] / (8 pi eta)
//                                                                      G = f10_i f10_j psi
//   E  <- Str: -Phi_2 x x Str / (16 pi eta)                          Phi = f10_i phi
//   Etr <- F: -3 (x.F) Phi_1 / (16 pi eta),  Phi = f6_j phi;  Etr <- S: 3 (x.S.x) Phi_2 / (16 pi eta),  Phi = f10_j phi
// with f6 = 1 + a^2 Lap/6, f10 = 1 + a^2 Lap/10 and (LG)_1 = 5 G2 + r^2 G3, (LG)_2 = 7 G3 + r^2 G4.
// (The pressure source factors f6_j, f10_j act on a harmonic function and leave the
// total unchanged; they make the real part consistent with the spread force density.)
// E rows are accumulated as a symmetric tensor and projected on the orthonormal
// traceless basis at the end.
#include "se_internal.cuh"

namespace se {

namespace {

template <typename T>
__device__ __forceinline__ T erfc_t(T x);
template <>
__device__ __forceinline__ float erfc_t<float>(float x) { return erfcf(x); }
template <>
__device__ __forceinline__ double erfc_t<double>(double x) { return erfc(x); }

template <typename T, int NCOMP>
__global__ void __launch_bounds__(128) real_kernel(int N, double L, double rc, SeParams p, int nc,
                                                   const int *cell_start, const double *pos,
                                                   const double *rad, const T *xs, T *yreal)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double pxi = pos[3 * i], pyi = pos[3 * i + 1], pzi = pos[3 * i + 2];
    const T ai = (T)rad[i], ai2 = ai * ai;
    const T xi = (T)p.xi, x2 = xi * xi;
    const T exn = (T)(1.0 / (p.xi * sqrt(kPi)));
    const T c8 = (T)(1.0 / (8 * kPi * p.eta)), c16 = (T)(1.0 / (16 * kPi * p.eta)),
            c32 = (T)(1.0 / (32 * kPi * p.eta));
    const double rc2 = rc * rc;
    const double cellw = L / nc;
    T U0 = 0, U1 = 0, U2 = 0, O0 = 0, O1 = 0, O2 = 0, Et = 0;
    T Axx = 0, Ayy = 0, Azz = 0, Axy = 0, Axz = 0, Ayz = 0;
    const int cx = min(nc - 1, (int)(pxi / cellw)), cy = min(nc - 1, (int)(pyi / cellw)),
              cz = min(nc - 1, (int)(pzi / cellw));
    const int span = nc >= 3 ? 1 : 0;
    for (int dz = -span; dz <= span; ++dz)
        for (int dy = -span; dy <= span; ++dy)
            for (int dx = -span; dx <= span; ++dx) {
                const int ccx = (cx + dx + nc) % nc, ccy = (cy + dy + nc) % nc, ccz = (cz + dz + nc) % nc;
                const int cell = (ccz * nc + ccy) * nc + ccx;
                const int js = cell_start[cell], je = cell_start[cell + 1];
                for (int j = js; j < je; ++j) {
                    if (j == i) continue;
                    double ddx = pxi - pos[3 * j], ddy = pyi - pos[3 * j + 1], ddz = pzi - pos[3 * j + 2];
                    ddx -= L * rint(ddx / L);
                    ddy -= L * rint(ddy / L);
                    ddz -= L * rint(ddz / L);
                    const double rr2 = ddx * ddx + ddy * ddy + ddz * ddz;
                    if (rr2 >= rc2) continue;
                    const T x0 = (T)ddx, x1 = (T)ddy, x2_ = (T)ddz, r2 = (T)rr2;
                    const T r = sqrt(r2), ir2 = 1 / r2;
                    const T aj = (T)rad[j], aj2 = aj * aj;
                    // B_0 .. B_7
                    T B[8];
                    const T ex = exp(-x2 * r2) * exn;
                    B[0] = erfc_t(xi * r) / r;
                    T pw = 1;
#pragma unroll
                    for (int n = 1; n < 8; ++n) {
                        pw *= 2 * x2;
                        B[n] = ((2 * n - 1) * B[n - 1] + pw * ex) * ir2;
                    }
                    // D^k psi (s), D^k Lap psi (l), D^k Lap^2 psi (m)
                    const T s2 = -B[1], s3 = B[2], s4 = -B[3], s5 = B[4], s6 = -B[5], s7 = B[6], s8 = -B[7];
                    const T s1 = B[0];
                    const T l1 = 5 * s2 + r2 * s3, l2 = 7 * s3 + r2 * s4, l3 = 9 * s4 + r2 * s5,
                            l4 = 11 * s5 + r2 * s6, l5 = 13 * s6 + r2 * s7, l6 = 15 * s7 + r2 * s8;
                    const T m1 = 5 * l2 + r2 * l3, m2 = 7 * l3 + r2 * l4, m3 = 9 * l4 + r2 * l5,
                            m4 = 11 * l5 + r2 * l6;
                    const T *xj = xs + (size_t)j * kNC;
                    const T F0 = xj[0], F1 = xj[1], F2 = xj[2];
                    const T xF = x0 * F0 + x1 * F1 + x2_ * F2;
                    {   // U <- F
                        const T c1 = (ai2 + aj2) * (T)(1.0 / 6), cc = ai2 * aj2 * (T)(1.0 / 36);
                        const T G1 = s1 + c1 * l1 + cc * m1, G2 = s2 + c1 * l2 + cc * m2;
                        const T a = c8 * (2 * G1 + r2 * G2), bb = c8 * xF * G2;
                        U0 += a * F0 - bb * x0;
                        U1 += a * F1 - bb * x1;
                        U2 += a * F2 - bb * x2_;
                    }
                    if constexpr (NCOMP >= 6) {
                        const T T0 = xj[3], T1 = xj[4], T2 = xj[5];
                        const T xT0 = x1 * T2 - x2_ * T1, xT1 = x2_ * T0 - x0 * T2, xT2 = x0 * T1 - x1 * T0;
                        const T xF0 = x1 * F2 - x2_ * F1, xF1 = x2_ * F0 - x0 * F2, xF2 = x0 * F1 - x1 * F0;
                        {   // U <- T
                            const T LG1 = c16 * (l1 + ai2 * (T)(1.0 / 6) * m1);
                            U0 += LG1 * xT0;
                            U1 += LG1 * xT1;
                            U2 += LG1 * xT2;
                        }
                        {   // Om <- F
                            const T LG1 = c16 * (l1 + aj2 * (T)(1.0 / 6) * m1);
                            O0 += LG1 * xF0;
                            O1 += LG1 * xF1;
                            O2 += LG1 * xF2;
                        }
                        {   // Om <- T
                            const T xTd = x0 * T0 + x1 * T1 + x2_ * T2;
                            const T a = c32 * xTd * l2, bb = c32 * (2 * l1 + r2 * l2);
                            O0 += a * x0 - bb * T0;
                            O1 += a * x1 - bb * T1;
                            O2 += a * x2_ - bb * T2;
                        }
                        if constexpr (NCOMP >= 11) {
                            // S tensor of j and its contractions
                            const T r2h = (T)0.70710678118654752440, r6 = (T)0.40824829046386301637;
                            const T Sxx = r2h * xj[6] - r6 * xj[7], Syy = -r2h * xj[6] - r6 * xj[7],
                                    Szz = 2 * r6 * xj[7], Sxy = r2h * xj[8], Sxz = r2h * xj[9],
                                    Syz = r2h * xj[10];
                            const T Sx0 = Sxx * x0 + Sxy * x1 + Sxz * x2_;
                            const T Sx1 = Sxy * x0 + Syy * x1 + Syz * x2_;
                            const T Sx2 = Sxz * x0 + Syz * x1 + Szz * x2_;
                            const T xSx = x0 * Sx0 + x1 * Sx1 + x2_ * Sx2;
                            {   // U <- S
                                const T c1 = ai2 * (T)(1.0 / 6) + aj2 * (T)0.1, cc = ai2 * aj2 * (T)(1.0 / 60);
                                const T G2 = s2 + c1 * l2 + cc * m2, G3 = s3 + c1 * l3 + cc * m3;
                                const T a = -c8 * (3 * G2 + r2 * G3), bb = c8 * xSx * G3;
                                U0 += a * Sx0 + bb * x0;
                                U1 += a * Sx1 + bb * x1;
                                U2 += a * Sx2 + bb * x2_;
                            }
                            {   // Om <- S
                                const T LG2 = -c16 * (l2 + aj2 * (T)0.1 * m2);
                                O0 += LG2 * (x1 * Sx2 - x2_ * Sx1);
                                O1 += LG2 * (x2_ * Sx0 - x0 * Sx2);
                                O2 += LG2 * (x0 * Sx1 - x1 * Sx0);
                            }
                            {   // E <- F
                                const T c1 = ai2 * (T)0.1 + aj2 * (T)(1.0 / 6), cc = ai2 * aj2 * (T)(1.0 / 60);
                                const T G2 = s2 + c1 * l2 + cc * m2, G3 = s3 + c1 * l3 + cc * m3;
                                const T a = c8 * (3 * G2 + r2 * G3), bb = -c8 * G3 * xF;
                                Axx += a * x0 * F0 + bb * x0 * x0;
                                Ayy += a * x1 * F1 + bb * x1 * x1;
                                Azz += a * x2_ * F2 + bb * x2_ * x2_;
                                Axy += a * (T)0.5 * (x0 * F1 + x1 * F0) + bb * x0 * x1;
                                Axz += a * (T)0.5 * (x0 * F2 + x2_ * F0) + bb * x0 * x2_;
                                Ayz += a * (T)0.5 * (x1 * F2 + x2_ * F1) + bb * x1 * x2_;
                            }
                            {   // E <- T
                                const T a = c16 * (l2 + ai2 * (T)0.1 * m2);
                                Axx += a * x0 * xT0;
                                Ayy += a * x1 * xT1;
                                Azz += a * x2_ * xT2;
                                Axy += a * (T)0.5 * (x0 * xT1 + x1 * xT0);
                                Axz += a * (T)0.5 * (x0 * xT2 + x2_ * xT0);
                                Ayz += a * (T)0.5 * (x1 * xT2 + x2_ * xT1);
                            }
                            {   // E <- S
                                const T c1 = (ai2 + aj2) * (T)0.1, cc = ai2 * aj2 * (T)0.01;
                                const T G2 = s2 + c1 * l2 + cc * m2, G3 = s3 + c1 * l3 + cc * m3,
                                        G4 = s4 + c1 * l4 + cc * m4;
                                const T a = -c8 * (3 * G2 + r2 * G3), bb = -c8 * (3 * G3 + r2 * G4),
                                        cq = c8 * G4 * xSx;
                                Axx += a * Sxx + bb * x0 * Sx0 + cq * x0 * x0;
                                Ayy += a * Syy + bb * x1 * Sx1 + cq * x1 * x1;
                                Azz += a * Szz + bb * x2_ * Sx2 + cq * x2_ * x2_;
                                Axy += a * Sxy + bb * (T)0.5 * (x0 * Sx1 + x1 * Sx0) + cq * x0 * x1;
                                Axz += a * Sxz + bb * (T)0.5 * (x0 * Sx2 + x2_ * Sx0) + cq * x0 * x2_;
                                Ayz += a * Syz + bb * (T)0.5 * (x1 * Sx2 + x2_ * Sx1) + cq * x1 * x2_;
                            }
                            if constexpr (NCOMP >= 12) {
                                // phi: p_k = (-1)^k B_k ; Lap phi: q_k = (2k+3) p_{k+1} + r^2 p_{k+2}
                                const T p1 = -B[1], p2 = B[2], p3 = -B[3], p4 = B[4];
                                const T q1 = 5 * p2 + r2 * p3, q2 = 7 * p3 + r2 * p4;
                                const T Str = xj[11];
                                {   // U <- Str
                                    const T a = -c16 * (p1 + ai2 * (T)(1.0 / 6) * q1) * Str;
                                    U0 += a * x0;
                                    U1 += a * x1;
                                    U2 += a * x2_;
                                }
                                {   // E <- Str
                                    const T a = -c16 * (p2 + ai2 * (T)0.1 * q2) * Str;
                                    Axx += a * x0 * x0;
                                    Ayy += a * x1 * x1;
                                    Azz += a * x2_ * x2_;
                                    Axy += a * x0 * x1;
                                    Axz += a * x0 * x2_;
                                    Ayz += a * x1 * x2_;
                                }
                                // Etr <- F, S
                                Et += -3 * c16 * xF * (p1 + aj2 * (T)(1.0 / 6) * q1) +
                                      3 * c16 * xSx * (p2 + aj2 * (T)0.1 * q2);
                            }
                        }
                    }
                }
            }
    T *yo = yreal + (size_t)i * kNC;
    yo[0] = U0;
    yo[1] = U1;
    yo[2] = U2;
    yo[3] = O0;
    yo[4] = O1;
    yo[5] = O2;
    const T r2h = (T)0.70710678118654752440, r6 = (T)0.40824829046386301637, sq2 = (T)1.41421356237309504880;
    yo[6] = r2h * (Axx - Ayy);
    yo[7] = r6 * (2 * Azz - Axx - Ayy);
    yo[8] = sq2 * Axy;
    yo[9] = sq2 * Axz;
    yo[10] = sq2 * Ayz;
    yo[11] = Et;
}

}  // namespace

template <typename T>
void launch_real(se_ctx *c, const T *xs, T *yreal, cudaStream_t s, int ncomp)
{
    const SeParams p = make_params(c);
    const int N = (int)c->N;
    const int tpb = 128;
    auto go = [&](auto kern) {
        kern<<<(N + tpb - 1) / tpb, tpb, 0, s>>>(N, c->L, c->rc, p, c->nc, c->b.cell_start, c->b.pos,
                                                  c->b.rad, xs, yreal);
    };
    if (ncomp <= 3) go(real_kernel<T, 3>);
    else if (ncomp <= 6) go(real_kernel<T, 6>);
    else if (ncomp <= 11) go(real_kernel<T, 11>);
    else go(real_kernel<T, 12>);
    c->launches++;
}

template void launch_real<float>(se_ctx *, const float *, float *, cudaStream_t, int);
template void launch_real<double>(se_ctx *, const double *, double *, cudaStream_t, int);

}  // namespace se
