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
#include <cmath>
#include <type_traits>
#include <vector>
#include <algorithm>

#include "se_internal.cuh"
#include "se_real_table.cuh"

namespace se {

namespace {

template <typename T>
__device__ __forceinline__ T erfc_t(T x);
template <>
__device__ __forceinline__ float erfc_t<float>(float x) { return erfcf(x); }
template <>
__device__ __forceinline__ double erfc_t<double>(double x) { return erfc(x); }

// Adds the couplings of source j (moments xj, radius^2 aj2) to target i (radius^2 ai2)
// at separation x = r_i - r_j, |x|^2 = r2 < rc^2.
template <typename T, int NCOMP>
__device__ __forceinline__ void pair_accumulate(const T x0, const T x1, const T x2_, const T r2, const T ai2,
                                                const T aj2, const T *xj, const T xi, const T x2,
                                                const T exn, const T c8, const T c16, const T c32, T &U0,
                                                T &U1, T &U2, T &O0, T &O1, T &O2, T &Et, T &Axx, T &Ayy,
                                                T &Azz, T &Axy, T &Axz, T &Ayz)
{
    const T r = sqrt(r2), ir2 = 1 / r2;
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
    const T s1 = B[0], s2 = -B[1], s3 = B[2], s4 = -B[3], s5 = B[4], s6 = -B[5], s7 = B[6], s8 = -B[7];
    const T l1 = 5 * s2 + r2 * s3, l2 = 7 * s3 + r2 * s4, l3 = 9 * s4 + r2 * s5, l4 = 11 * s5 + r2 * s6,
            l5 = 13 * s6 + r2 * s7, l6 = 15 * s7 + r2 * s8;
    const T m1 = 5 * l2 + r2 * l3, m2 = 7 * l3 + r2 * l4, m3 = 9 * l4 + r2 * l5, m4 = 11 * l5 + r2 * l6;
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

// One CTA per cell of side >= rc: its particles are the targets (one per thread);
// the particles of the 27 neighbouring cells are staged in shared memory and every
// staged source serves all targets of the cell.  Positions are offsets from the
// own cell's origin, so x = off_i - (d * cellw + off_j) for the neighbour cell at
// displacement d, accurate in FP32; with a single cell the minimum image is taken.
template <typename T, int NCOMP>
__global__ void __launch_bounds__(64) real_kernel(double L, double rc, SeParams p, int nc,
                                                  const int *cell_start, const T *rel, const T *xs,
                                                  T *yreal)
{
    constexpr int CH = 64;
    constexpr int NM = NCOMP;
    __shared__ T sj[CH][4];
    __shared__ T smx[CH][NM];
    const int cell = blockIdx.x;
    const int cx = cell % nc, cy = (cell / nc) % nc, cz = cell / (nc * nc);
    const int ts = cell_start[cell], te = cell_start[cell + 1];
    const T cellw = (T)(L / nc), Lt = (T)L;
    const T rc2 = (T)(rc * rc);
    const T xi = (T)p.xi, x2 = xi * xi;
    const T exn = (T)(1.0 / (p.xi * sqrt(kPi)));
    const T c8 = (T)(1.0 / (8 * kPi * p.eta)), c16 = (T)(1.0 / (16 * kPi * p.eta)),
            c32 = (T)(1.0 / (32 * kPi * p.eta));
    const int span = nc >= 3 ? 1 : 0;
    for (int tb = ts; tb < te; tb += CH) {
        const int i = tb + threadIdx.x;
        const bool active = i < te;
        T oi0 = 0, oi1 = 0, oi2 = 0, ai2 = 0;
        if (active) {
            oi0 = rel[4 * i];
            oi1 = rel[4 * i + 1];
            oi2 = rel[4 * i + 2];
            ai2 = rel[4 * i + 3] * rel[4 * i + 3];
        }
        T U0 = 0, U1 = 0, U2 = 0, O0 = 0, O1 = 0, O2 = 0, Et = 0;
        T Axx = 0, Ayy = 0, Azz = 0, Axy = 0, Axz = 0, Ayz = 0;
        for (int dz = -span; dz <= span; ++dz)
            for (int dy = -span; dy <= span; ++dy)
                for (int dx = -span; dx <= span; ++dx) {
                    const int nb = (((cz + dz + nc) % nc) * nc + (cy + dy + nc) % nc) * nc + (cx + dx + nc) % nc;
                    const int js = cell_start[nb], je = cell_start[nb + 1];
                    const T sh0 = dx * cellw, sh1 = dy * cellw, sh2 = dz * cellw;
                    for (int jb = js; jb < je; jb += CH) {
                        const int cnt = min(CH, je - jb);
                        __syncthreads();
                        for (int e = threadIdx.x; e < cnt * 4; e += blockDim.x) sj[e >> 2][e & 3] = rel[4 * jb + e];
                        for (int e = threadIdx.x; e < cnt * NM; e += blockDim.x)
                            smx[e / NM][e % NM] = xs[(size_t)(jb + e / NM) * kNC + e % NM];
                        __syncthreads();
                        if (!active) continue;
                        for (int k = 0; k < cnt; ++k) {
                            if (jb + k == i) continue;
                            T x0 = oi0 - (sh0 + sj[k][0]), x1 = oi1 - (sh1 + sj[k][1]), x2_ = oi2 - (sh2 + sj[k][2]);
                            if (span == 0) {
                                x0 -= Lt * rint(x0 / Lt);
                                x1 -= Lt * rint(x1 / Lt);
                                x2_ -= Lt * rint(x2_ / Lt);
                            }
                            const T r2 = x0 * x0 + x1 * x1 + x2_ * x2_;
                            if (r2 >= rc2) continue;
                            T xj[kNC];
#pragma unroll
                            for (int c = 0; c < kNC; ++c) xj[c] = c < NM ? smx[k][c < NM ? c : 0] : (T)0;
                            pair_accumulate<T, NCOMP>(x0, x1, x2_, r2, ai2, sj[k][3] * sj[k][3], xj, xi, x2, exn,
                                                      c8, c16, c32, U0, U1, U2, O0, O1, O2, Et, Axx, Ayy, Azz,
                                                      Axy, Axz, Ayz);
                        }
                    }
                }
        if (active) {
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
    }
}

// Offsets of every particle from the origin of its cell, and its radius.
template <typename T>
__global__ void rel_kernel(int N, double L, int nc, const double *pos, const double *rad, T *rel)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double w = L / nc;
    for (int d = 0; d < 3; ++d) {
        const double v = pos[3 * i + d];
        int c = (int)(v / w);
        c = c >= nc ? nc - 1 : c;
        rel[4 * i + d] = (T)(v - c * w);
    }
    rel[4 * i + 3] = (T)rad[i];
}

}  // namespace

namespace {

// ---------------------------------------------------------------- stored pair table
//
// The real-space operator depends only on the configuration, so (as in Sec. 3.3,
// where it is stored as a sparse matrix per configuration) its pairs are built once:
// for every target i (cell order) the neighbours j with |x| < rc, the separation x
// and 19 radial coefficients, each the combination of B_n, Faxen radii and 1/(8 pi eta)
// that multiplies one tensor structure of the couplings listed at the top of this file:
//   0 aF  = (2 G1 + r^2 G2)/(8 pi eta)      1 bF = G2/(8 pi eta)                 (U <- F)
//   2 uT  = (LG)_1/(16 pi eta) [f6_i]       3 oF = (LG)_1/(16 pi eta) [f6_j]     (U <- T, Om <- F)
//   4 oTa = (Lpsi)_2/(32 pi eta)            5 oTb = (2 (Lpsi)_1 + r^2 (Lpsi)_2)/(32 pi eta)
//   6 uSa = -(3 G2 + r^2 G3)/(8 pi eta)     7 uSb = G3/(8 pi eta)                (U <- S)
//   8 oS  = -(LG)_2/(16 pi eta) [f10_j]                                          (Om <- S)
//   9 eFa = (3 G2 + r^2 G3)/(8 pi eta)     10 eFb = -G3/(8 pi eta)               (E <- F)
//  11 eT  = (LG)_2/(16 pi eta) [f10_i]                                           (E <- T)
//  12 eSa = -(3 G2 + r^2 G3)/(8 pi eta)    13 eSb = -(3 G3 + r^2 G4)/(8 pi eta)
//  14 eSc = G4/(8 pi eta)                                                        (E <- S)
//  15 uQ  = -Phi_1/(16 pi eta) [f6_i]      16 eQ = -Phi_2/(16 pi eta) [f10_i]    (U, E <- Str)
//  17 tF  = -3 Phi_1/(16 pi eta) [f6_j]    18 tS = 3 Phi_2/(16 pi eta) [f10_j]   (Etr <- F, S)
// The coefficients are evaluated in FP64 and stored at the compute precision.
constexpr int kNPC = 19;

// constants of pair_coefficients (per configuration): xi, xi^2, 1/(xi sqrt(pi)), 1/(8 pi eta)
struct PairConst {
    double xi, x2, exn, c8;
};

// The 19 coefficients from B_0 = erfc(xi r)/r and ex = exp(-xi^2 r^2)/(xi sqrt(pi)) by the
// recurrence above, in arithmetic R (FP64, or double-float for the FP32 table): the Laplacians
// of psi cancel (a float64 evaluation loses up to 14 bits against a 50-digit one), so R carries
// more than the stored precision.  tx2 = 2 xi^2; i6, i10 = 1/6, 1/10; c8 = 1/(8 pi eta).
template <typename R>
__device__ __forceinline__ void pair_coefficients_B(const R r2, const R ir2, const R B0, const R ex, const R ai2,
                                                    const R aj2, const R tx2, const R c8, const R i6, const R i10,
                                                    R *cf)
{
    R B[8];
    B[0] = B0;
    R pw = tx2;
#pragma unroll
    for (int n = 1; n < 8; ++n) {
        B[n] = ((2 * n - 1) * B[n - 1] + pw * ex) * ir2;
        pw = pw * tx2;
    }
    const R s1 = B[0], s2 = -B[1], s3 = B[2], s4 = -B[3], s5 = B[4], s6 = -B[5], s7 = B[6], s8 = -B[7];
    const R l1 = 5 * s2 + r2 * s3, l2 = 7 * s3 + r2 * s4, l3 = 9 * s4 + r2 * s5, l4 = 11 * s5 + r2 * s6,
            l5 = 13 * s6 + r2 * s7, l6 = 15 * s7 + r2 * s8;
    const R m1 = 5 * l2 + r2 * l3, m2 = 7 * l3 + r2 * l4, m3 = 9 * l4 + r2 * l5, m4 = 11 * l5 + r2 * l6;
    const R p1 = -B[1], p2 = B[2], p3 = -B[3], p4 = B[4];
    const R q1 = 5 * p2 + r2 * p3, q2 = 7 * p3 + r2 * p4;
    const R c16 = c8 * R(0.5f), c32 = c8 * R(0.25f);
    const R ai6 = ai2 * i6, aj6 = aj2 * i6, ai10 = ai2 * i10, aj10 = aj2 * i10;
    {
        const R c1 = ai6 + aj6, cc = ai6 * aj6;                      // (a_i^2 + a_j^2)/6, a_i^2 a_j^2/36
        const R G1 = s1 + c1 * l1 + cc * m1, G2 = s2 + c1 * l2 + cc * m2;
        cf[0] = c8 * (2 * G1 + r2 * G2);
        cf[1] = c8 * G2;
    }
    cf[2] = c16 * (l1 + ai6 * m1);
    cf[3] = c16 * (l1 + aj6 * m1);
    cf[4] = c32 * l2;
    cf[5] = c32 * (2 * l1 + r2 * l2);
    {
        const R c1 = ai6 + aj10, cc = ai6 * aj10;                    // a_i^2/6 + a_j^2/10, a_i^2 a_j^2/60
        const R G2 = s2 + c1 * l2 + cc * m2, G3 = s3 + c1 * l3 + cc * m3;
        cf[6] = -c8 * (3 * G2 + r2 * G3);
        cf[7] = c8 * G3;
    }
    cf[8] = -c16 * (l2 + aj10 * m2);
    {
        const R c1 = ai10 + aj6, cc = ai10 * aj6;
        const R G2 = s2 + c1 * l2 + cc * m2, G3 = s3 + c1 * l3 + cc * m3;
        cf[9] = c8 * (3 * G2 + r2 * G3);
        cf[10] = -c8 * G3;
    }
    cf[11] = c16 * (l2 + ai10 * m2);
    {
        const R c1 = ai10 + aj10, cc = ai10 * aj10;                  // (a_i^2 + a_j^2)/10, a_i^2 a_j^2/100
        const R G2 = s2 + c1 * l2 + cc * m2, G3 = s3 + c1 * l3 + cc * m3, G4 = s4 + c1 * l4 + cc * m4;
        cf[12] = -c8 * (3 * G2 + r2 * G3);
        cf[13] = -c8 * (3 * G3 + r2 * G4);
        cf[14] = c8 * G4;
    }
    cf[15] = -c16 * (p1 + ai6 * q1);
    cf[16] = -c16 * (p2 + ai10 * q2);
    cf[17] = -3 * c16 * (p1 + aj6 * q1);
    cf[18] = 3 * c16 * (p2 + aj10 * q2);
}

// FP64 evaluation: one FP64 division (1/r^2), a square root and the two special functions.
__device__ __forceinline__ void pair_coefficients(double r2, double ai2, double aj2, const PairConst &k, double *cf)
{
    const double r = sqrt(r2), ir2 = 1.0 / r2;
    const double ex = exp(-k.x2 * r2) * k.exn;
    const double B0 = erfc(k.xi * r) * (r * ir2);
    pair_coefficients_B<double>(r2, ir2, B0, ex, ai2, aj2, 2 * k.x2, k.c8, 1.0 / 6, 0.1, cf);
}

// ---- double-float evaluation for the FP32 table (B300's FP32 pipe issues tens of times the
// operations of its FP64 pipe).  erfc(x) = erfcx(x) exp(-x^2), with the scaled complementary error
// function erfcx from a table of Chebyshev interpolants (kErfcxDeg + 1 points per interval of width
// 1/4 on [0, xi rc], built on the host from the C library's long-double erfc and exp and stored as
// double-float coefficients of the monomials in t = 8 x - (2 j + 1) in [-1, 1]; interpolation error
// below 1e-14 relative) and exp(-x^2) from ff_exp.  Pairs outside the range where the double-float
// values stay normal FP32 numbers (r < 0.1, where B_7 ~ r^-15 grows large; xi r > kFfXmax, where
// exp(-x^2) approaches the FP32 underflow) take the FP64 evaluation.
constexpr int kErfcxDeg = 9;
constexpr double kFfXmax = 8.5, kFfR2min = 0.01;

struct PairConstFF {
    ff xi, x2, exn, tx2, c8, i6, i10;
};

__device__ __forceinline__ ff erfcx_ff(ff x, const float2 *tab, int nint)
{
    const int j = max(0, min(nint - 1, (int)(x.hi * 4.0f)));
    const ff t = ff(8.0f * x.hi, 8.0f * x.lo) - ff((float)(2 * j + 1), 0.f);
    const float2 *c = tab + j * (kErfcxDeg + 1);
    ff q(c[kErfcxDeg].x, c[kErfcxDeg].y);
#pragma unroll
    for (int m = kErfcxDeg - 1; m >= 0; --m) q = q * t + ff(c[m].x, c[m].y);
    return q;
}

__device__ __forceinline__ void pair_coefficients_ff(double r2d, double ai2d, double aj2d, const PairConstFF &k,
                                                     const float2 *tab, int nint, float *cf)
{
    const ff r2 = ff(r2d), r = ff_sqrt(r2), ir2 = ff(1) / r2;
    const ff e2 = ff_exp(-(k.x2 * r2));                 // exp(-xi^2 r^2)
    const ff B0 = erfcx_ff(k.xi * r, tab, nint) * e2 * (r * ir2);
    ff c[kNPC];
    pair_coefficients_B<ff>(r2, ir2, B0, e2 * k.exn, ff(ai2d), ff(aj2d), k.tx2, k.c8, k.i6, k.i10, c);
#pragma unroll
    for (int q = 0; q < kNPC; ++q) cf[q] = c[q].hi + c[q].lo;
}

// Neighbour search for target i (cell order): calls f(j) for every j != i with
// |x_ij| < rc (minimum image), in a fixed order (cells dz, dy, dx, then cell order).
// The decision is the FP64 one, |x|^2 < rc^2 with x = p_i - p_j wrapped by +-L; it is
// taken in FP32 where that is safe: with positions in [0, L) rounded to FP32, each
// component of the FP32 separation is within 5 * 2^-24 L of the exact one and the FP32
// |x|^2 within 2^-22 |x|^2 of its value, so |x_f32| differs from |x| by less than
// mrg = 2^-20 (L (1 + 2 |gamma|) + rc) (the sheared cell adds the rounding of the
// gamma L shift).  Below (rc - mrg)^2 the pair is surely inside, at or above
// (rc + mrg)^2 surely outside; only the thin band between repeats the FP64 test.
// Minimum image on the cell a1 = (L, 0, 0), a2 = (g L, L, 0), a3 = (0, 0, L) (|g| <= 1/2):
// the separation (positions in the wrapped cell, so each component is below (1 + |g|) L)
// is shifted by a2 until |y| <= L/2, then by a1 (at most twice) and a3.  For g = 0 it is the
// per-component wrap of the cube.
template <typename R>
__device__ __forceinline__ void min_image3(R &x, R &y, R &z, R L, R g)
{
    const R h = (R)0.5 * L;
    if (y > h) { y -= L; x -= g * L; } else if (y < -h) { y += L; x += g * L; }
    x = x > h ? x - L : (x < -h ? x + L : x);
    x = x > h ? x - L : (x < -h ? x + L : x);
    z = z > h ? z - L : (z < -h ? z + L : z);
}

struct PairSearch {
    double L, rc2, gamma;
    float Lf, gf, lo, hi;      // FP32 box and strain, and the band (rc -+ mrg)^2
    int nc;
};

template <typename F>
__device__ __forceinline__ void for_neighbours(int i, const PairSearch &ps, const int *cell_start,
                                               const double *pos, const float4 *pf, F f)
{
    const int nc = ps.nc;
    const double w = ps.L / nc;
    const double px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
    // cells of the fractional coordinates L t = (x - gamma y, y, z)
    const int cx = max(0, min(nc - 1, (int)((px - ps.gamma * py) / w))), cy = min(nc - 1, (int)(py / w)),
              cz = min(nc - 1, (int)(pz / w));
    const float4 pi = pf[i];
    const int span = nc >= 3 ? 1 : 0;
    for (int dz = -span; dz <= span; ++dz)
        for (int dy = -span; dy <= span; ++dy)
            for (int dx = -span; dx <= span; ++dx) {
                const int nb = (((cz + dz + nc) % nc) * nc + (cy + dy + nc) % nc) * nc + (cx + dx + nc) % nc;
                for (int j = cell_start[nb]; j < cell_start[nb + 1]; ++j) {
                    const float4 pj = pf[j];
                    float x0 = pi.x - pj.x, x1 = pi.y - pj.y, x2 = pi.z - pj.z;
                    min_image3(x0, x1, x2, ps.Lf, ps.gf);
                    const float r2f = x0 * x0 + x1 * x1 + x2 * x2;
                    if (r2f >= ps.hi || j == i) continue;
                    if (r2f >= ps.lo) {
                        double y0 = px - pos[3 * j], y1 = py - pos[3 * j + 1], y2 = pz - pos[3 * j + 2];
                        min_image3(y0, y1, y2, ps.L, ps.gamma);
                        if (!(y0 * y0 + y1 * y1 + y2 * y2 < ps.rc2)) continue;
                    }
                    f(j, r2f, pj.w);
                }
            }
}

__global__ void pos_f32_kernel(int N, const double *pos, const double *rad, float4 *pf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) pf[i] = make_float4((float)pos[3 * i], (float)pos[3 * i + 1], (float)pos[3 * i + 2], (float)rad[i]);
}

// Counts the pairs of target i; with `overlap` set, also flags a pair inside rc whose
// spheres overlap, |x| < (a_i + a_j)(1 - 1e-12) in FP64 (an FP32 prefilter with a 1e-4
// margin picks the candidates; touching spheres are allowed).
__global__ void pair_count_kernel(int N, PairSearch ps, const int *cell_start, const double *pos, const double *rad,
                                  const float4 *pf, int *count, int *overlap)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int n = 0;
    const float ai = pf[i].w;
    for_neighbours(i, ps, cell_start, pos, pf, [&](int j, float r2f, float aj) {
        ++n;
        const float sa = ai + aj;
        if (overlap && r2f < sa * sa * 1.0001f) {
            double y0 = pos[3 * i] - pos[3 * j], y1 = pos[3 * i + 1] - pos[3 * j + 1], y2 = pos[3 * i + 2] - pos[3 * j + 2];
            min_image3(y0, y1, y2, ps.L, ps.gamma);
            const double s = (rad[i] + rad[j]) * (1.0 - 1e-12);
            if (y0 * y0 + y1 * y1 + y2 * y2 < s * s) atomicExch(overlap, 1);
        }
    });
    count[i] = n;
}

__global__ void pair_list_kernel(int N, PairSearch ps, const int *cell_start, const double *pos, const float4 *pf,
                                 const int *off, int *pj)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int k = off[i];
    for_neighbours(i, ps, cell_start, pos, pf, [&](int j, float, float) { pj[k++] = j; });
}

// the coefficients of pair k in the SoA table: all 19, or the 13 stored slots of a monodisperse
// table (mono_slot)
template <typename T, typename C>
__device__ __forceinline__ void store_coefficients(T *pc, size_t np, int k, const C *cf, int mono)
{
    if (mono) {
#pragma unroll
        for (int q = 0; q < kNPC; ++q)
            if (mono_slot(q) >= 0) pc[(size_t)mono_slot(q) * np + k] = (T)cf[q];
    } else {
#pragma unroll
        for (int q = 0; q < kNPC; ++q) pc[(size_t)q * np + k] = (T)cf[q];
    }
}

// One warp per target: the lanes take the target's pairs in turn, form the FP64
// separation and the radial coefficients and store them (coalesced SoA rows).
template <typename T>
__global__ void __launch_bounds__(256) pair_fill_kernel(int N, double L, double gamma, PairConst pk,
                                                        const double *pos,
                                                        const double *rad, const int *off, size_t np, const int *pj,
                                                        T *px, T *pc, int mono)
{
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= N) return;
    const double p0 = pos[3 * i], p1 = pos[3 * i + 1], p2 = pos[3 * i + 2], ai2 = rad[i] * rad[i];
    const int ke = off[i + 1];
    for (int k = off[i] + lane; k < ke; k += 32) {
        const int j = pj[k];
        double x0 = p0 - pos[3 * j], x1 = p1 - pos[3 * j + 1], x2 = p2 - pos[3 * j + 2];
        min_image3(x0, x1, x2, L, gamma);
        double cf[kNPC];
        pair_coefficients(x0 * x0 + x1 * x1 + x2 * x2, ai2, rad[j] * rad[j], pk, cf);
        px[k] = (T)x0;
        px[np + k] = (T)x1;
        px[2 * np + k] = (T)x2;
        store_coefficients(pc, np, k, cf, mono);
    }
}

// The FP32 table with the coefficients in double-float arithmetic where its range allows
// (pair_coefficients_ff), in FP64 elsewhere; the separation is formed in FP64 as above.
__global__ void __launch_bounds__(256) pair_fill_ff_kernel(int N, double L, double gamma, PairConst pk,
                                                           PairConstFF pkf, const float2 *etab, int nint,
                                                           double r2_ff_max, const double *pos, const double *rad,
                                                           const int *off, size_t np, const int *pj, float *px,
                                                           float *pc, int mono)
{
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= N) return;
    const double p0 = pos[3 * i], p1 = pos[3 * i + 1], p2 = pos[3 * i + 2], ai2 = rad[i] * rad[i];
    const int ke = off[i + 1];
    for (int k = off[i] + lane; k < ke; k += 32) {
        const int j = pj[k];
        double x0 = p0 - pos[3 * j], x1 = p1 - pos[3 * j + 1], x2 = p2 - pos[3 * j + 2];
        min_image3(x0, x1, x2, L, gamma);
        const double r2 = x0 * x0 + x1 * x1 + x2 * x2, aj2 = rad[j] * rad[j];
        float cf[kNPC];
        if (r2 >= kFfR2min && r2 <= r2_ff_max) {
            pair_coefficients_ff(r2, ai2, aj2, pkf, etab, nint, cf);
        } else {
            double cd[kNPC];
            pair_coefficients(r2, ai2, aj2, pk, cd);
#pragma unroll
            for (int q = 0; q < kNPC; ++q) cf[q] = (float)cd[q];
        }
        px[k] = (float)x0;
        px[np + k] = (float)x1;
        px[2 * np + k] = (float)x2;
        store_coefficients(pc, np, k, cf, mono);
    }
}

// One warp per target (real_table_body).
template <typename T, int NCOMP, typename TL = T, bool MONO = false>
__global__ void __launch_bounds__(256) real_table_kernel(int N, const int *off, size_t np, const int *pj,
                                                         const TL *px, const TL *pc, const T *xs, T *yreal)
{
    real_table_body<T, NCOMP, TL, MONO>(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), threadIdx.x & 31, N, off,
                                        np, pj, px, pc, xs, yreal);
}

}  // namespace

// Chebyshev interpolants of erfcx(x) = erfc(x) exp(x^2) on the intervals [j/4, (j+1)/4] covering
// [0, xmax]: values at the kErfcxDeg + 1 Chebyshev points of each interval from the C library's
// long-double erfc and exp, Chebyshev coefficients by the discrete cosine sums, converted to the
// monomial basis of t in [-1, 1] (T_{m+1} = 2 t T_m - T_{m-1}) and stored as double-floats.
static std::vector<float2> erfcx_table(double xmax, int &nint)
{
    constexpr int n = kErfcxDeg + 1;
    nint = std::max(1, (int)std::ceil(xmax * 4));
    std::vector<float2> tab((size_t)nint * n);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int j = 0; j < nint; ++j) {
        long double f[n], cheb[n], mono[n] = {}, Tprev[n] = {}, Tcur[n] = {}, Tnext[n];
        for (int k = 0; k < n; ++k) {
            const long double th = pi * (k + 0.5L) / n;
            const long double x = (j + (std::cos(th) + 1) / 2) / 4.0L;
            f[k] = std::erfc(x) * std::exp(x * x);
        }
        for (int m = 0; m < n; ++m) {
            long double acc = 0;
            for (int k = 0; k < n; ++k) acc += f[k] * std::cos(m * pi * (k + 0.5L) / n);
            cheb[m] = 2 * acc / n;
        }
        cheb[0] /= 2;
        Tprev[0] = 1;                                   // T_0
        Tcur[1] = 1;                                    // T_1
        mono[0] = cheb[0];
        for (int m = 1; m < n; ++m) {
            for (int d = 0; d < n; ++d) mono[d] += cheb[m] * Tcur[d];
            for (int d = 0; d < n; ++d) Tnext[d] = (d > 0 ? 2 * Tcur[d - 1] : 0) - Tprev[d];
            for (int d = 0; d < n; ++d) {
                Tprev[d] = Tcur[d];
                Tcur[d] = Tnext[d];
            }
        }
        for (int d = 0; d < n; ++d) {
            const float hi = (float)mono[d];
            tab[(size_t)j * n + d] = make_float2(hi, (float)(mono[d] - (long double)hi));
        }
    }
    return tab;
}

static PairConstFF ff_constants(const PairConst &k)
{
    auto split = [](double d) { const float h = (float)d; return ff(h, (float)(d - (double)h)); };
    return PairConstFF{split(k.xi), split(k.x2), split(k.exn), split(2 * k.x2), split(k.c8), split(1.0 / 6),
                       split(0.1)};
}

// neighbour lists (precision independent) and coefficients at precision T
template <typename T>
int build_pair_table(se_ctx *c)
{
    cudaStream_t s = c->stream;
    const int N = (int)c->N;
    if (!c->lists_ok) {
        int *count = nullptr;
        float4 *pf = nullptr;
        auto release = [&]() {
            if (count) cudaFree(count);
            if (pf) cudaFree(pf);
        };
        auto drop_lists = [&]() {          // leave no half-built list behind
            if (c->b.pair_off) cudaFree(c->b.pair_off);
            if (c->b.pair_j) cudaFree(c->b.pair_j);
            c->b.pair_off = nullptr;
            c->b.pair_j = nullptr;
            c->pair_off_n = 0;
            c->pairj_cap = 0;
        };
        auto fail = [&]() {
            cudaGetLastError();
            release();
            drop_lists();
            c->err = "pair table allocation failed";
            return SE_ERR_NOMEM;
        };
        auto sync = [&]() {
            const cudaError_t e = cudaStreamSynchronize(s);
            if (e == cudaSuccess) return SE_OK;
            release();
            drop_lists();
            c->err = std::string("pair table build: ") + cudaGetErrorString(e);
            return SE_ERR_CUDA;
        };
        // the previous configuration's buffers are overwritten in place when they fit
        if (c->b.pair_off && c->pair_off_n != N) {
            cudaFree(c->b.pair_off);
            c->b.pair_off = nullptr;
            c->pair_off_n = 0;
        }
        if (!c->b.pair_off) {
            if (cudaMalloc(&c->b.pair_off, (N + 1) * sizeof(int)) != cudaSuccess) return fail();
            c->pair_off_n = N;
        }
        if (cudaMalloc(&count, (N + 1) * sizeof(int)) != cudaSuccess || cudaMalloc(&pf, N * sizeof(float4)) != cudaSuccess)
            return fail();
        PairSearch ps;
        ps.L = c->L;
        ps.rc2 = c->rc * c->rc;
        ps.gamma = c->shear;
        ps.nc = c->nc;
        ps.Lf = (float)c->L;
        ps.gf = (float)c->shear;
        // FP32 separations: within 5 2^-24 L of the exact ones per component, plus the
        // rounding of the shear shift gamma L
        const double mrg = std::ldexp(c->L * (1 + 2 * std::fabs(c->shear)) + c->rc, -20);
        ps.lo = (float)((c->rc - mrg) * (c->rc - mrg));
        ps.hi = (float)((c->rc + mrg) * (c->rc + mrg));
        int *ovl = c->overlap_check ? count + N : nullptr;    // the flag after the counts
        if (ovl) cudaMemsetAsync(ovl, 0, sizeof(int), s);
        pos_f32_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, c->b.pos, c->b.rad, pf);
        pair_count_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, ps, c->b.cell_start, c->b.pos, c->b.rad, pf, count, ovl);
        c->launches += 2;
        launch_scan(c, N, count, c->b.pair_off, s);
        int np = 0, hov = 0;
        cudaMemcpyAsync(&np, c->b.pair_off + N, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (ovl) cudaMemcpyAsync(&hov, ovl, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (int rc = sync()) return rc;
        if (hov) {
            release();
            drop_lists();
            c->err = "two spheres overlap (|x_ij| < a_i + a_j) within the real-space cutoff";
            return SE_ERR_OVERLAP;
        }
        c->npairs = (size_t)np;
        if (c->npairs + 1 > c->pairj_cap) {
            if (c->b.pair_j) cudaFree(c->b.pair_j);
            c->b.pair_j = nullptr;
            c->pairj_cap = 0;
            const size_t cap = c->npairs + 1 + c->npairs / 16;      // room for the next configurations
            if (cudaMalloc(&c->b.pair_j, cap * sizeof(int)) != cudaSuccess) return fail();
            c->pairj_cap = cap;
        }
        pair_list_kernel<<<(N + 127) / 128, 128, 0, s>>>(N, ps, c->b.cell_start, c->b.pos, pf, c->b.pair_off,
                                                         c->b.pair_j);
        c->launches++;
        if (int rc = sync()) return rc;
        release();
        c->lists_ok = true;
    }
    const int q = pix<T>();
    const size_t np = c->npairs;
    if (c->pair_cap[q] < np) {
        if (c->b.pair_x[q]) cudaFree(c->b.pair_x[q]);
        if (c->b.pair_c[q]) cudaFree(c->b.pair_c[q]);
        c->b.pair_x[q] = c->b.pair_c[q] = nullptr;
        c->pair_cap[q] = 0;
        const size_t cap = np + np / 16;                           // room for the next configurations
        if (cudaMalloc(&c->b.pair_x[q], (3 * cap + 1) * sizeof(T)) != cudaSuccess ||
            cudaMalloc(&c->b.pair_c[q], ((size_t)kNPC * cap + 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            if (c->b.pair_x[q]) cudaFree(c->b.pair_x[q]);
            if (c->b.pair_c[q]) cudaFree(c->b.pair_c[q]);
            c->b.pair_x[q] = c->b.pair_c[q] = nullptr;
            c->err = "pair table allocation failed";
            return SE_ERR_NOMEM;
        }
        c->pair_cap[q] = cap;
    }
    const PairConst pk{c->xi, c->xi * c->xi, 1.0 / (c->xi * std::sqrt(kPi)), 1.0 / (8 * kPi * c->eta)};
    // monodisperse FP32 tables store 13 of the 19 coefficients (mono_slot)
    const int mono = std::is_same<T, float>::value && c->mono ? 1 : 0;
    float2 *etab = nullptr;
    int nint = 0;
    if (std::is_same<T, float>::value && !c->pair_fill_fp64) {
        // erfcx table on [0, min(xi rc, kFfXmax)] (the pairs beyond take the FP64 evaluation)
        const double xmax = std::min(c->xi * c->rc * (1 + 1e-6), kFfXmax);
        const std::vector<float2> h = erfcx_table(xmax, nint);
        if (cudaMalloc(&etab, h.size() * sizeof(float2)) != cudaSuccess) {
            cudaGetLastError();
            etab = nullptr;           // the FP64 evaluation below
        } else if (cudaMemcpyAsync(etab, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice, s) !=
                   cudaSuccess) {
            cudaGetLastError();
            cudaFree(etab);
            etab = nullptr;
        }
    }
    if (etab) {
        const double xm = nint * 0.25 < kFfXmax ? nint * 0.25 : kFfXmax;    // table end
        const double r2max = (xm / c->xi) * (xm / c->xi);
        const PairConstFF pkf = ff_constants(pk);
        pair_fill_ff_kernel<<<(N + 7) / 8, 256, 0, s>>>(N, c->L, c->shear, pk, pkf, etab, nint, r2max, c->b.pos,
                                                         c->b.rad, c->b.pair_off, np, c->b.pair_j,
                                                         (float *)c->b.pair_x[q], (float *)c->b.pair_c[q], mono);
    } else {
        pair_fill_kernel<T><<<(N + 7) / 8, 256, 0, s>>>(N, c->L, c->shear, pk, c->b.pos, c->b.rad,
                                                        c->b.pair_off, np, c->b.pair_j, (T *)c->b.pair_x[q],
                                                        (T *)c->b.pair_c[q], mono);
    }
    c->launches++;
    const cudaError_t e = cudaStreamSynchronize(s);
    if (etab) cudaFree(etab);
    SE_CUDA_CHECK(c, e);
    c->pair_mono[q] = mono != 0;
    c->pairs_ok[q] = true;
    return SE_OK;
}

template int build_pair_table<float>(se_ctx *);
template int build_pair_table<double>(se_ctx *);

template <typename T>
void setup_rel(se_ctx *c, cudaStream_t s)
{
    const int N = (int)c->N;
    rel_kernel<T><<<(N + 127) / 128, 128, 0, s>>>(N, c->L, c->nc, c->b.pos, c->b.rad, (T *)c->b.rel[pix<T>()]);
    c->launches++;
}

template <typename T>
void launch_real(se_ctx *c, const T *xs, T *yreal, cudaStream_t s, int ncomp)
{
    const SeParams p = make_params(c);
    const int q = pix<T>();
    if (c->pairs_ok[q]) {
        const int N = (int)c->N, wpb = 8;
        auto go = [&](auto kern) {
            kern<<<(N + wpb - 1) / wpb, wpb * 32, 0, s>>>(N, c->b.pair_off, c->npairs, c->b.pair_j,
                                                          (const T *)c->b.pair_x[q], (const T *)c->b.pair_c[q],
                                                          xs, yreal);
        };
        if (c->pair_mono[q]) {
            if (ncomp <= 3) go(real_table_kernel<T, 3, T, true>);
            else if (ncomp <= 6) go(real_table_kernel<T, 6, T, true>);
            else if (ncomp <= 11) go(real_table_kernel<T, 11, T, true>);
            else go(real_table_kernel<T, 12, T, true>);
        } else {
            if (ncomp <= 3) go(real_table_kernel<T, 3>);
            else if (ncomp <= 6) go(real_table_kernel<T, 6>);
            else if (ncomp <= 11) go(real_table_kernel<T, 11>);
            else go(real_table_kernel<T, 12>);
        }
        c->launches++;
        return;
    }
    const int ncell = c->nc * c->nc * c->nc;
    auto go = [&](auto kern) {
        kern<<<ncell, 64, 0, s>>>(c->L, c->rc, p, c->nc, c->b.cell_start, (const T *)c->b.rel[pix<T>()], xs, yreal);
    };
    if (ncomp <= 3) go(real_kernel<T, 3>);
    else if (ncomp <= 6) go(real_kernel<T, 6>);
    else if (ncomp <= 11) go(real_kernel<T, 11>);
    else go(real_kernel<T, 12>);
    c->launches++;
}

namespace {
__global__ void d2ff_kernel(size_t n, const double *in, ff *out)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        out[k] = ff(in[k]);
}
}  // namespace

// The FP64 pair table as double-floats (once per configuration, beside the FP64 one), so
// that the double-float real-space sum reads no FP64 values.  Without memory for it, or
// with SE_OPT_FF_TABLE 0, the sum converts the FP64 table as it reads it.
int build_pair_table_ff(se_ctx *c)
{
    if (!c->pairs_ok[1] || c->pairs_ok[2] || !c->ff_table) return SE_OK;
    const size_t np = c->npairs, nx = 3 * np + 1, nc = (size_t)kNPC * np + 1;
    for (int q = 0; q < 2; ++q) {
        void *&p = q ? c->b.pair_c[2] : c->b.pair_x[2];
        if (p) cudaFree(p);
        p = nullptr;
    }
    if (cudaMalloc(&c->b.pair_x[2], nx * sizeof(ff)) != cudaSuccess ||
        cudaMalloc(&c->b.pair_c[2], nc * sizeof(ff)) != cudaSuccess) {
        cudaGetLastError();
        if (c->b.pair_x[2]) cudaFree(c->b.pair_x[2]);
        c->b.pair_x[2] = c->b.pair_c[2] = nullptr;
        return SE_OK;
    }
    cudaStream_t s = c->stream;
    d2ff_kernel<<<4 * c->sms, 256, 0, s>>>(nx, (const double *)c->b.pair_x[1], (ff *)c->b.pair_x[2]);
    d2ff_kernel<<<4 * c->sms, 256, 0, s>>>(nc, (const double *)c->b.pair_c[1], (ff *)c->b.pair_c[2]);
    c->launches += 2;
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        // no half-built copy survives: the sum falls back to the FP64 table
        cudaFree(c->b.pair_x[2]);
        cudaFree(c->b.pair_c[2]);
        c->b.pair_x[2] = c->b.pair_c[2] = nullptr;
        c->err = std::string("double-float pair table: ") + cudaGetErrorString(e);
        return SE_ERR_CUDA;
    }
    c->pairs_ok[2] = true;
    return SE_OK;
}

// The FP64-equivalent product's real-space sum: the pair table contracted in double-float
// arithmetic (B300's FP32 pipe issues many times the FMAs of its FP64 pipe), from the
// double-float table, else from the FP64 one.  Returns false, launching nothing, when
// there is neither (the caller then runs the FP64 cell-list kernel).
bool launch_real_ff(se_ctx *c, const ff *xs, ff *yreal, cudaStream_t s, int ncomp)
{
    if (!c->pairs_ok[1] && !c->pairs_ok[2]) return false;
    const int N = (int)c->N, wpb = 8;
    auto go = [&](auto kern, const auto *px, const auto *pc) {
        kern<<<(N + wpb - 1) / wpb, wpb * 32, 0, s>>>(N, c->b.pair_off, c->npairs, c->b.pair_j, px, pc, xs, yreal);
    };
    auto pick = [&](const auto *px, const auto *pc) {
        using TL = std::remove_cv_t<std::remove_pointer_t<decltype(px)>>;
        if (ncomp <= 3) go(real_table_kernel<ff, 3, TL>, px, pc);
        else if (ncomp <= 6) go(real_table_kernel<ff, 6, TL>, px, pc);
        else if (ncomp <= 11) go(real_table_kernel<ff, 11, TL>, px, pc);
        else go(real_table_kernel<ff, 12, TL>, px, pc);
    };
    if (c->pairs_ok[2]) pick((const ff *)c->b.pair_x[2], (const ff *)c->b.pair_c[2]);
    else pick((const double *)c->b.pair_x[1], (const double *)c->b.pair_c[1]);
    c->launches++;
    return true;
}

template void setup_rel<float>(se_ctx *, cudaStream_t);
template void setup_rel<double>(se_ctx *, cudaStream_t);
template void launch_real<float>(se_ctx *, const float *, float *, cudaStream_t, int);
template void launch_real<double>(se_ctx *, const double *, double *, cudaStream_t, int);

}  // namespace se

// ---------------------------------------------------------------- allocation-free variant
//
// se_real_space_apply_noalloc: the real-space pair sum of the product (the cell-list
// kernel above, in FP64) for callers that cannot allocate device memory -- for
// instance an application whose own allocator reserves the device memory up front,
// or a latency-critical caller that cannot accept the device-wide synchronisation of
// cudaMalloc / cudaFree.  Its scratch (cell keys, counts, cell starts, the particle
// order, sorted offsets and moments, the sorted result) lives in one file-scope
// device array sized for SE_NOALLOC_MAX_N particles and SE_NOALLOC_MAX_CELLS cells.
// Every GPU that loads the library holds that array (about 2 MB) until the process
// exits.  All calls share it: calls that overlap on the GPU (several host threads or
// streams at once) race on it and must be serialised by the caller.
namespace se {
namespace {

constexpr int kNaMaxN = SE_NOALLOC_MAX_N, kNaMaxCells = SE_NOALLOC_MAX_CELLS;
constexpr size_t kNaInts = 2 * (size_t)kNaMaxN + 2 * ((size_t)kNaMaxCells + 1) + 64;
constexpr size_t kNaBytes = kNaInts * sizeof(int) + (size_t)kNaMaxN * (4 + 2 * kNC) * sizeof(double);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

struct NaLayout {
    int *key, *count, *start, *perm, *flag;
    double *rel, *xs, *yr;
};

NaLayout na_layout(unsigned char *base)
{
    NaLayout l;
    int *ip = reinterpret_cast<int *>(base);
    l.key = ip;
    l.perm = ip + kNaMaxN;
    l.count = ip + 2 * kNaMaxN;
    l.start = l.count + (kNaMaxCells + 1);
    l.flag = l.start + (kNaMaxCells + 1);
    double *dp = reinterpret_cast<double *>(base + kNaInts * sizeof(int));
    l.rel = dp;
    l.xs = dp + 4 * (size_t)kNaMaxN;
    l.yr = l.xs + (size_t)kNC * kNaMaxN;
    return l;
}

__global__ void na_clear_kernel(int ncell, int *count, int *flag)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= ncell; e += gridDim.x * blockDim.x) count[e] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) flag[0] = 0;
}

__global__ void na_key_kernel(int N, double L, int nc, const double *pos, const double *rad, int *key, int *count,
                              int *flag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    bool ok = isfinite(rad[i]) && rad[i] > 0;
    int k[3];
    for (int d = 0; d < 3; ++d) {
        double v = pos[3 * i + d];
        ok = ok && isfinite(v);
        v = ok ? v - L * floor(v / L) : 0.0;
        int c = (int)(v / (L / nc));
        k[d] = c >= nc ? nc - 1 : (c < 0 ? 0 : c);
    }
    key[i] = (k[2] * nc + k[1]) * nc + k[0];
    atomicAdd(&count[key[i]], 1);
    if (!ok) atomicExch(flag, 1);
}

// exclusive scan of count[0..n) into start[0..n] (one CTA), then count is reused as a cursor
__global__ void na_scan_kernel(int n, int *count, int *start)
{
    __shared__ int part[1024];
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(n, b + per);
    int s = 0;
    for (int q = b; q < e; ++q) s += count[q];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int v = part[t];
            part[t] = acc;
            acc += v;
        }
        start[n] = acc;
    }
    __syncthreads();
    int acc = part[threadIdx.x];
    for (int q = b; q < e; ++q) {
        start[q] = acc;
        acc += count[q];
        count[q] = 0;
    }
}

__global__ void na_scatter_kernel(int N, const int *key, const int *start, int *cursor, int *perm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int k = key[i];
    perm[start[k] + atomicAdd(&cursor[k], 1)] = i;
}

// order each cell by caller index (deterministic layout), then gather offsets and moments
__global__ void na_order_kernel(int ncell, const int *start, int *perm)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= ncell) return;
    for (int i = start[b] + 1; i < start[b + 1]; ++i) {
        const int v = perm[i];
        int j = i - 1;
        while (j >= start[b] && perm[j] > v) {
            perm[j + 1] = perm[j];
            --j;
        }
        perm[j + 1] = v;
    }
}

__global__ void na_gather_kernel(int N, double L, int nc, int ncomp, const int *perm, const double *pos,
                                 const double *rad, const double *x, double *rel, double *xs)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int i = perm[k];
    const double w = L / nc;
    for (int d = 0; d < 3; ++d) {
        double v = pos[3 * i + d];
        v -= L * floor(v / L);
        int c = (int)(v / w);
        c = c >= nc ? nc - 1 : c;
        rel[4 * k + d] = v - c * w;
    }
    rel[4 * k + 3] = rad[i];
    for (int c = 0; c < kNC; ++c) xs[(size_t)k * kNC + c] = c < ncomp ? x[(size_t)i * ncomp + c] : 0.0;
}

__global__ void na_scatter_out_kernel(int N, int ncomp, const int *perm, const double *yr, double *y)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    for (int c = 0; c < ncomp; ++c) y[(size_t)perm[k] * ncomp + c] = yr[(size_t)k * kNC + c];
}

constexpr int kNaMaxDevices = 64;
unsigned char *g_noalloc_ptr[kNaMaxDevices] = {};

}  // namespace

}  // namespace se

extern "C" int se_real_space_apply_noalloc(int device, void *stream, int64_t N, double L, double xi, double rc,
                                           double eta, const double *pos, const double *radius, int ncomp,
                                           const double *x, double *y)
{
    using namespace se;
    if (!pos || !radius || !x || !y || N < 1) return SE_ERR_ARG;
    if (ncomp != 3 && ncomp != 6 && ncomp != 11 && ncomp != 12) return SE_ERR_ARG;
    if (!(L > 0) || !(xi > 0) || !(eta > 0) || !std::isfinite(L)) return SE_ERR_ARG;
    if (N > kNaMaxN) return SE_ERR_TOO_LARGE;
    if (!(rc > 0) || rc >= 0.5 * L) return SE_ERR_CUTOFF;
    if (device < 0 || device >= kNaMaxDevices) return SE_ERR_ARG;
    // the caller's current device is restored before every return
    int prev_device = -1;
    if (cudaGetDevice(&prev_device) != cudaSuccess) return SE_ERR_CUDA;
    struct Restore {
        int dev;
        ~Restore() { cudaSetDevice(dev); }
    } restore{prev_device};
    if (cudaSetDevice(device) != cudaSuccess) return SE_ERR_CUDA;
    cudaGetLastError();   // an earlier, unrelated launch error is not this call's
    // once per device: the device address of the scratch array (its host-side name is
    // only a stand-in and must not be passed to a kernel)
    if (!g_noalloc_ptr[device]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return SE_ERR_CUDA;
        }
        g_noalloc_ptr[device] = static_cast<unsigned char *>(ptr);
    }
    int nc = (int)std::floor(L / rc);
    if (nc < 3) nc = 1;
    while (nc > 1 && nc * nc * nc > kNaMaxCells) --nc;   // larger cells stay correct
    if (nc < 3) nc = 1;
    const int n = (int)N, ncell = nc * nc * nc;
    const NaLayout l = na_layout(g_noalloc_ptr[device]);
    cudaStream_t s = (cudaStream_t)stream;
    na_clear_kernel<<<(ncell + 256) / 256, 256, 0, s>>>(ncell, l.count, l.flag);
    na_key_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, L, nc, pos, radius, l.key, l.count, l.flag);
    na_scan_kernel<<<1, 1024, 0, s>>>(ncell, l.count, l.start);
    na_scatter_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, l.key, l.start, l.count, l.perm);
    na_order_kernel<<<(ncell + 127) / 128, 128, 0, s>>>(ncell, l.start, l.perm);
    na_gather_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, L, nc, ncomp, l.perm, pos, radius, x, l.rel, l.xs);
    SeParams p{};
    p.L = L;
    p.xi = xi;
    p.rc = rc;
    p.eta = eta;
    auto go = [&](auto kern) { kern<<<ncell, 64, 0, s>>>(L, rc, p, nc, l.start, l.rel, l.xs, l.yr); };
    if (ncomp <= 3) go(real_kernel<double, 3>);
    else if (ncomp <= 6) go(real_kernel<double, 6>);
    else if (ncomp <= 11) go(real_kernel<double, 11>);
    else go(real_kernel<double, 12>);
    na_scatter_out_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, ncomp, l.perm, l.yr, y);
    if (cudaGetLastError() != cudaSuccess) return SE_ERR_CUDA;   // a launch of this call failed
    int flag = 0;
    if (cudaMemcpyAsync(&flag, l.flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SE_ERR_CUDA;
    return flag ? SE_ERR_NONFINITE : SE_OK;
}
