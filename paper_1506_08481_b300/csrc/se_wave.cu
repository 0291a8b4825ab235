// Wave-space part of the grand-mobility product by the Spectral Ewald method
// (Sec. 3.1-3.2): Gaussian spreading (Eq. grid-space), forward 3D FFT, k-space
// scaling (Eq. wave-result) fused into the last forward stage together with the
// first inverse stage, inverse 3D FFT, and the trapezoid-rule gather
// (Eq. parseval-sum, Eq. parseval-sum-2).
//
// Grid units: u = x M / L, so grid points are integers; the Gaussian of Eq. shape
// is g(s) = exp(-alpha |s|^2) with alpha = 2 m^2 / P^2 (Eq. theta-param: the edge
// value at |s| = P/2 is exp(-m^2/2)); d/dx = kappa d/ds with kappa = M / L.
//
// Per particle j the spread grid holds the force density of its multipoles
//   H = F (1 + a^2 Lap/6) g + 1/2 grad g x T - S . grad (1 + a^2 Lap/10) g,   H_src = S_tr g
// (Eq. grid-space extended to torques and stresslets via Eq. mul-expand).
// With Hhat the forward DFT and q the integer wave vector, k = 2 pi q / L:
//   Ghat = c exp(-k^2/(4 xi^2) + 2 pi^2 q^2/(alpha M^2)) [ Phi (I - k k/k^2) Hhat
//          + i k/(4 k^2) Hhat_src ],  Phi = (1 + k^2/(4 xi^2))/k^2,  c = (alpha/pi)^3/(eta V)
// (Eq. wave-result: the two exp(-theta q^2/(8 xi^2)) factors of Eq. rp-wave-tq are
// the transforms of the spread and gather Gaussians, exp(theta q^2/(4 xi^2)) undoes
// them; the source term is the wave part of Eq. source-split with Q = -grad phi/(16 pi eta)),
// and the pressure (Eq. pres-multi-expans, wave part) scaled by 3/(4 eta) (Eq. faxen-p):
//   Ghat_p = (3/4) c exp(...) i k.Hhat / k^2.
// Hybrid approach (Sec. 3.2): the target Faxen Laplacian is applied in wave space,
// Ghat'' = -k^2 Ghat, and gathered with weight a_i^2/6 (U) or a_i^2/10 (E).
// Real-space approach: the target Laplacian acts on the gather weights instead.
// Nyquist planes and q = 0 are set to zero.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "se_fft.cuh"
#include "se_internal.cuh"
#include "se_real_table.cuh"

namespace se {

namespace {


template <typename T> struct V4;
template <> struct V4<float> { using t = float4; };
template <> struct V4<double> { using t = double4_32a; };
template <> struct V4<ff> { using t = ff4; };

// CTAs of 256 threads per SM the gather is compiled for (register budget) and the
// unrolling of its z-loop (loads in flight per lane)
#ifndef SE_GATHER_MINB
#define SE_GATHER_MINB 2
#endif
#ifndef SE_GATHER_NCL
#define SE_GATHER_NCL 2         // columns per lane of the FP32 4-component gather
#endif
#ifndef SE_GATHER_UNROLL
#define SE_GATHER_UNROLL 12
#endif
constexpr int kGatherUnroll = SE_GATHER_UNROLL;

__device__ __forceinline__ int wrapi(int i, int M) { return i >= M ? i - M : (i < 0 ? i + M : i); }

// S tensor (xx, yy, zz, xy, xz, yz) from coordinates on the orthonormal basis
template <typename T>
__device__ __forceinline__ void stresslet_tensor(const T *s, T S[6])
{
    const T r2 = (T)0.70710678118654752440, r6 = (T)0.40824829046386301637;
    S[0] = r2 * s[0] - r6 * s[1];
    S[1] = -r2 * s[0] - r6 * s[1];
    S[2] = 2 * r6 * s[1];
    S[3] = r2 * s[2];
    S[4] = r2 * s[3];
    S[5] = r2 * s[4];
}

// ---------------------------------------------------------------- support setup

// Per particle (cell order): first support point b (wrapped), offset s0 = b - u of
// that point from the particle, and the 1D Gaussian weights g(s0 + i), i < P, by
// fast Gaussian gridding (Eq. fgg-exp) centred on the nearest grid point:
//   g(delta + j) = exp(-alpha delta^2) exp(-2 alpha delta)^j exp(-alpha j^2).
template <typename T>
__global__ void support_kernel(int N, SeParams p, const double *pos, const double *e3 /*[2P+1], j=-P..P*/,
                               int *base, T *s0out, T *w)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int M = p.M, P = p.P;
    for (int d = 0; d < 3; ++d) {
        // grid units of the fractional coordinate: u = M t, L t = (x - gamma y, y, z)
        double u = (pos[3 * i + d] - (d == 0 ? p.gamma * pos[3 * i + 1] : 0.0)) * p.kappa;
        int b = (int)floor(u - 0.5 * P) + 1;
        double s0 = b - u;                       // in (-P/2, -P/2 + 1]
        int ic = (int)floor(-s0 + 0.5);          // index of the point nearest the particle
        double delta = s0 + ic;                  // in [-1/2, 1/2]
        double e1 = exp(-p.alpha * delta * delta), e2 = exp(-2.0 * p.alpha * delta);
        double pw = 1.0;
        for (int j = 0; ic + j < P; ++j) {       // points at and above the centre
            w[((size_t)i * 3 + d) * P + ic + j] = (T)(e1 * pw * e3[P + j]);
            pw *= e2;
        }
        pw = 1.0;
        for (int j = 1; ic - j >= 0; ++j) {      // points below the centre
            pw /= e2;
            w[((size_t)i * 3 + d) * P + ic - j] = (T)(e1 * pw * e3[P - j]);
        }
        b %= M;
        if (b < 0) b += M;
        base[3 * i + d] = b;
        s0out[3 * i + d] = (T)s0;
    }
}

// ---------------------------------------------------------------- spreading

// One CTA per kTile^3 tile of the grid; each of its 64 threads owns one (x, y)
// column of 8 grid points and accumulates their values in registers (no atomics
// anywhere).  The candidate particles (those in the bins whose support start lies
// within P - 1 points before the tile) are listed by a prefix sum over the bin counts
// and staged in shared memory 64 at a time, one particle per thread: the x and y
// Gaussian weights in the tile window, the table W_z = g_z (1, s_z, s_z^2, s_z^3) of the
// 8 tile planes, the offsets of the tile origin, the Faxen coefficients and moments.
// Along a column the force density is a cubic polynomial in s_z times g_z
// (Eq. grid-space with the torque and stresslet terms):
//   H = g [ (A0 + A1 s^2) F - alpha kappa (s x T) + (B0 + B1 s^2) S.s ],  H_src = g S_tr,
// so a thread forms 13 column coefficients per particle and spends 13 FMAs per point.
// Shared staging of spread_body (rows are XOR-swizzled by the particle slot so that the
// staging writes, one particle per thread, spread over all banks; reads broadcast one
// particle's row; per particle sp holds (sx0 sy0 A0 A1) (B0 B1 halves Str)
// (F0 F1 F2 T0) (T1 T2 Sxx Syy) (Szz Sxy Sxz Syz) as broadcast vectors)
template <typename T> struct Spread8Smem {
    T sxy[64][2 * kTile];                  // window weights x(8) y(8), entry e at e ^ ((k >> 1) & 15)
    typename V4<T>::t swz[64][kTile];      // g_z (1, s_z, s_z^2, s_z^3) of plane t at t ^ (k & 7)
    typename V4<T>::t sp[64][5];
    int bin_beg[125], bin_off[126];
};

// The tile's work for 64 threads (tid 0..63, sync() a barrier of those 64 threads).
// WS: the wave-space approach to the particle sizes (SE_OPT_SIZE_MODE 2): no Faxen
// Laplacian in the spread; instead 8 grid components per point, H0 (3) = g [F - alpha
// kappa (s x T) + 2 alpha kappa S.s], Ha (3) = g [(a^2/6) F + (a^2 alpha kappa / 5) S.s]
// (whose transform enters with -k^2: the source Faxen operators (1 + a^2 Lap/6) and
// (1 + a^2 Lap/10) in wave space), the source g S_tr and a zero; 13 FMAs per point.
template <typename T, int NCOMP, bool SPLIT, typename Sync, bool WS = false>
__device__ __forceinline__ void spread_body(int tile, int part, int tid, Sync sync, Spread8Smem<T> &sm, SeParams p,
                                            const int *tile_start, const int *tile_perm, const int *base,
                                            const T *s0g, const T *wg, const double *rad, const T *xs, T *grid,
                                            int nsplit)
{
    constexpr int TT = kTile, CH = 64;
    using T4 = typename V4<T>::t;
    auto &sxy = sm.sxy;
    auto &swz = sm.swz;
    auto &sp = sm.sp;
    auto &bin_beg = sm.bin_beg;
    auto &bin_off = sm.bin_off;
    const int M = p.M, P = p.P, nt = p.ntile;
    const int bx0 = tile % nt, by0 = (tile / nt) % nt, bz0 = tile / (nt * nt);
    const int t0[3] = {bx0 * TT, by0 * TT, bz0 * TT};
    const int tx = tid & 7, ty = tid >> 3;
    const int nbin = (P - 1 + TT - 1) / TT + 1, nb3 = nbin * nbin * nbin;
    const T alpha = (T)p.alpha, kap = (T)p.kappa, akap = alpha * kap;
    constexpr int NA = WS ? 7 : (NCOMP >= 12 ? 4 : 3);
    constexpr int GC = WS ? 8 : 4;                // grid components per point
    T acc[TT][NA];
#pragma unroll
    for (int z = 0; z < TT; ++z)
#pragma unroll
        for (int c = 0; c < NA; ++c) acc[z][c] = 0;

    // candidate list: bins (tile - b) for b in [0, nbin)^3, concatenated
    for (int bb = tid; bb < nb3; bb += CH) {
        const int bx = bb % nbin, by = (bb / nbin) % nbin, bz = bb / (nbin * nbin);
        const int bin = (wrapi(bz0 - bz, nt) * nt + wrapi(by0 - by, nt)) * nt + wrapi(bx0 - bx, nt);
        bin_beg[bb] = tile_start[bin];
        bin_off[bb + 1] = tile_start[bin + 1] - tile_start[bin];
    }
    sync();
    if (tid == 0) {
        bin_off[0] = 0;
        for (int bb = 0; bb < nb3; ++bb) bin_off[bb + 1] += bin_off[bb];
    }
    sync();
    const int total = bin_off[nb3];

    // SPLIT: part `part` of nsplit takes every nsplit-th chunk of the candidates
    // and writes the partial grid part
    int cbeg = 0, cstep = CH;
    if constexpr (SPLIT) {
        grid += (size_t)part * M * M * M * GC;
        cbeg = part * CH;
        cstep = nsplit * CH;
    }
    for (int c0 = cbeg; c0 < total; c0 += cstep) {
        const int cnt = min(CH, total - c0);
        sync();
        if ((int)tid < cnt) {
            const int k = tid, idx = c0 + k;
            int lo = 0, hi = nb3;                       // bin_off[lo] <= idx < bin_off[lo + 1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (bin_off[mid] <= idx) lo = mid; else hi = mid;
            }
            const int i = tile_perm[bin_beg[lo] + idx - bin_off[lo]];
            bool ok = true;
            int od[3];
            for (int d = 0; d < 3; ++d) {
                int o = wrapi(t0[d] - base[3 * i + d], M);   // support index of the tile origin
                if (o >= P) o -= M;
                ok &= (o < P) && (o > -TT);
                od[d] = o;
            }
            const T *w = wg + (size_t)i * 3 * P;
            const int sw_xy = (k >> 1) & 15, sw_z = k & 7;
#pragma unroll
            for (int t = 0; t < TT; ++t) {
                const int ix = od[0] + t, iy = od[1] + t, iz = od[2] + t;
                sxy[k][t ^ sw_xy] = (ix >= 0 && ix < P) ? w[ix] : (T)0;
                sxy[k][(TT + t) ^ sw_xy] = (iy >= 0 && iy < P) ? w[P + iy] : (T)0;
                const T g = (iz >= 0 && iz < P) ? w[2 * P + iz] : (T)0;
                const T sz = s0g[3 * i + 2] + (T)iz;
                swz[k][t ^ sw_z] = T4{g, g * sz, g * sz * sz, g * sz * sz * sz};
            }
            const T a = (T)rad[i], a2k2 = a * a * kap * kap;
            const T *xi = xs + (size_t)i * kNC;
            T S[6] = {0, 0, 0, 0, 0, 0}, Tq[3] = {0, 0, 0};
            if constexpr (NCOMP >= 6) { Tq[0] = xi[3]; Tq[1] = xi[4]; Tq[2] = xi[5]; }
            if constexpr (NCOMP >= 11) stresslet_tensor(xi + 6, S);
            // which halves of the tile's 8 planes the support reaches (planes t with
            // 0 <= od_z + t < P); bit 0: planes 0-3, bit 1: planes 4-7
            const int zlo = max(0, -od[2]), zhi = min(TT, P - od[2]);
            const int halves = (zlo < TT / 2 && zhi > 0 ? 1 : 0) | (zhi > TT / 2 && zlo < TT ? 2 : 0);
            // offsets of the tile origin, Faxen coefficients, moments
            if constexpr (WS) {
                const T a2 = a * a;
                sp[k][0] = T4{s0g[3 * i] + (T)od[0], s0g[3 * i + 1] + (T)od[1], a2 / 6, (T)0.2 * a2 * alpha * kap};
                sp[k][1] = T4{2 * kap * alpha, (T)0, ok ? (T)halves : (T)0, NCOMP >= 12 ? xi[11] : (T)0};
            } else {
                sp[k][0] = T4{s0g[3 * i] + (T)od[0], s0g[3 * i + 1] + (T)od[1], 1 - a2k2 * alpha,
                              (T)(2.0 / 3.0) * a2k2 * alpha * alpha};
                sp[k][1] = T4{2 * kap * alpha * (1 - a2k2 * alpha), (T)0.8 * kap * a2k2 * alpha * alpha * alpha,
                              ok ? (T)halves : (T)0, NCOMP >= 12 ? xi[11] : (T)0};
            }
            sp[k][2] = T4{xi[0], xi[1], xi[2], Tq[0]};
            sp[k][3] = T4{Tq[1], Tq[2], S[0], S[1]};
            sp[k][4] = T4{S[2], S[3], S[4], S[5]};
        }
        sync();
        for (int k = 0; k < cnt; ++k) {
            const int sw_xy = (k >> 1) & 15, sw_z = k & 7;
            const T gxy = sxy[k][tx ^ sw_xy] * sxy[k][(TT + ty) ^ sw_xy];
            const T4 v1 = sp[k][1];
            const int halves = (int)v1.z;
            if (gxy == (T)0 || halves == 0) continue;
            const T4 v0 = sp[k][0], v2 = sp[k][2];
            const T sx = v0.x + tx, sy0 = v0.y + ty;
            // the physical gradient of the window is -2 alpha kappa (sx, sy - gamma sx, sz) g in
            // the sheared cell (grid units of the fractional coordinates); gamma = 0 otherwise
            const T sy = WS ? sy0 - (T)p.gamma * sx : sy0;
            if constexpr (WS) {
                // h0[q][p], ha[q][p]: coefficients of s_z^p (p = 0, 1) of H0 and Ha (times g_xy)
                T h0[3][2], ha[3][2];
                const T F[3] = {v2.x, v2.y, v2.z};
                const T c6 = v0.z, c5 = v0.w, ak2 = v1.x;     // a^2/6, a^2 alpha kappa/5, 2 alpha kappa
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    h0[q][0] = F[q];
                    h0[q][1] = 0;
                    ha[q][0] = c6 * F[q];
                    ha[q][1] = 0;
                }
                if constexpr (NCOMP >= 6) {
                    const T4 v3 = sp[k][3];
                    const T T0 = v2.w, T1 = v3.x, T2 = v3.y;
                    h0[0][0] -= akap * sy * T2;
                    h0[1][0] += akap * sx * T2;
                    h0[2][0] -= akap * (sx * T1 - sy * T0);
                    h0[0][1] += akap * T1;
                    h0[1][1] -= akap * T0;
                    if constexpr (NCOMP >= 11) {
                        const T4 v4 = sp[k][4];
                        const T S[6] = {v3.z, v3.w, v4.x, v4.y, v4.z, v4.w};
                        const T d0[3] = {S[0] * sx + S[3] * sy, S[3] * sx + S[1] * sy, S[4] * sx + S[5] * sy};
                        const T d1[3] = {S[4], S[5], S[2]};
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            h0[q][0] += ak2 * d0[q];
                            h0[q][1] += ak2 * d1[q];
                            ha[q][0] += c5 * d0[q];
                            ha[q][1] = c5 * d1[q];
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 3; ++q)
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        h0[q][e] *= gxy;
                        ha[q][e] *= gxy;
                    }
                const T cs = NCOMP >= 12 ? gxy * v1.w : (T)0;
                auto planes = [&](auto z0c) {
                    constexpr int z0 = decltype(z0c)::value;
#pragma unroll
                    for (int z = z0; z < z0 + TT / 2; ++z) {
                        const T4 W = swz[k][z ^ sw_z];
#pragma unroll
                        for (int q = 0; q < 3; ++q) {
                            acc[z][q] += h0[q][0] * W.x + h0[q][1] * W.y;
                            acc[z][3 + q] += ha[q][0] * W.x + ha[q][1] * W.y;
                        }
                        if constexpr (NCOMP >= 12) acc[z][6] += cs * W.x;
                    }
                };
                if (halves & 1) planes(std::integral_constant<int, 0>{});
                if (halves & 2) planes(std::integral_constant<int, TT / 2>{});
                continue;
            }
            const T sxy2 = sx * sx + sy * sy;
            const T A1 = v0.w, a0 = v0.z + A1 * sxy2;
            // column coefficients c[alpha][p] of s_z^p (times g_xy)
            T c[3][4];
            const T F[3] = {v2.x, v2.y, v2.z};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                c[q][0] = a0 * F[q];
                c[q][1] = 0;
                c[q][2] = A1 * F[q];
                c[q][3] = 0;
            }
            if constexpr (NCOMP >= 6) {
                // -alpha kappa (s x T), s x T = c0 + s_z c1
                const T4 v3 = sp[k][3];
                const T T0 = v2.w, T1 = v3.x, T2 = v3.y;
                c[0][0] -= akap * sy * T2;
                c[1][0] += akap * sx * T2;
                c[2][0] -= akap * (sx * T1 - sy * T0);
                c[0][1] += akap * T1;
                c[1][1] -= akap * T0;
                if constexpr (NCOMP >= 11) {
                    // (B0 + B1 s^2) S.s with S.s = d0 + s_z d1
                    const T4 v4 = sp[k][4];
                    const T S[6] = {v3.z, v3.w, v4.x, v4.y, v4.z, v4.w};
                    const T B1 = v1.y, b0 = v1.x + B1 * sxy2;
                    const T d00 = S[0] * sx + S[3] * sy, d01 = S[3] * sx + S[1] * sy, d02 = S[4] * sx + S[5] * sy;
                    const T d10 = S[4], d11 = S[5], d12 = S[2];
                    c[0][0] += b0 * d00; c[1][0] += b0 * d01; c[2][0] += b0 * d02;
                    c[0][1] += b0 * d10; c[1][1] += b0 * d11; c[2][1] += b0 * d12;
                    c[0][2] += B1 * d00; c[1][2] += B1 * d01; c[2][2] += B1 * d02;
                    c[0][3] = B1 * d10; c[1][3] = B1 * d11; c[2][3] = B1 * d12;
                }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int e = 0; e < 4; ++e) c[q][e] *= gxy;
            const T cs = NCOMP >= 12 ? gxy * v1.w : (T)0;
            auto planes = [&](auto z0c) {
                constexpr int z0 = decltype(z0c)::value;
#pragma unroll
                for (int z = z0; z < z0 + TT / 2; ++z) {
                    const T4 W = swz[k][z ^ sw_z];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        if constexpr (std::is_same<T, ff>::value) {
                            // double-floats: the column's terms into the plane's sum with one normalisation
                            lazy_madd(acc[z][q], c[q][0], W.x);
                            if constexpr (NCOMP >= 6) lazy_madd(acc[z][q], c[q][1], W.y);
                            lazy_madd(acc[z][q], c[q][2], W.z);
                            if constexpr (NCOMP >= 11) lazy_madd(acc[z][q], c[q][3], W.w);
                            lazy_finish(acc[z][q]);
                        } else if constexpr (NCOMP >= 11)
                            acc[z][q] += c[q][0] * W.x + c[q][1] * W.y + c[q][2] * W.z + c[q][3] * W.w;
                        else if constexpr (NCOMP >= 6)
                            acc[z][q] += c[q][0] * W.x + c[q][1] * W.y + c[q][2] * W.z;
                        else
                            acc[z][q] += c[q][0] * W.x + c[q][2] * W.z;
                    }
                    if constexpr (NCOMP >= 12) acc[z][NA - 1] += cs * W.x;
                }
            };
            // planes outside the support carry zero weight: skip a half the support misses
            if (halves & 1) planes(std::integral_constant<int, 0>{});
            if (halves & 2) planes(std::integral_constant<int, TT / 2>{});
        }
    }
#pragma unroll
    for (int z = 0; z < TT; ++z) {
        const size_t gi = (((size_t)(t0[2] + z) * M + (t0[1] + ty)) * M + (t0[0] + tx)) * GC;
        T4 v;
        v.x = acc[z][0];
        v.y = acc[z][1];
        v.z = acc[z][2];
        if constexpr (WS) {
            v.w = acc[z][3];
            *reinterpret_cast<T4 *>(grid + gi) = v;
            v.x = acc[z][4];
            v.y = acc[z][5];
            v.z = NCOMP >= 12 ? acc[z][6] : (T)0;
            v.w = (T)0;
            *reinterpret_cast<T4 *>(grid + gi + 4) = v;
        } else {
            v.w = NCOMP >= 12 ? acc[z][NA - 1] : (T)0;
            *reinterpret_cast<T4 *>(grid + gi) = v;
        }
    }
}

template <typename T, int NCOMP, bool SPLIT, bool WS = false>
__global__ void __launch_bounds__(64, sizeof(T) == 4 ? 11 : 6) spread_kernel(SeParams p, const int *tile_start,
                                                    const int *tile_perm, const int *base,
                                                    const T *s0g, const T *wg, const double *rad,
                                                    const T *xs, T *grid, int nsplit)
{
    __shared__ Spread8Smem<T> sm;
    auto sync = [] { __syncthreads(); };
    spread_body<T, NCOMP, SPLIT, decltype(sync), WS>(blockIdx.x, blockIdx.y, threadIdx.x, sync, sm, p, tile_start,
                                                     tile_perm, base, s0g, wg, rad, xs, grid, nsplit);
}

// ---- FP32 spreading over 8 x 8 x 16 tiles with packed FMAs
//
// The same column scheme as spread_kernel with tiles of 16 planes: a thread's column
// coefficients (the per-particle overhead) serve 16 planes instead of 8, and the
// plane updates pair planes (2 zp, 2 zp + 1) in packed FP32 FMAs (fma.rn.f32x2: two
// lanes' worth of FMAs per issue slot), acc2[zp][q] = (value at plane 2 zp, value at
// plane 2 zp + 1) of component q.  The staged table holds, per particle and plane pair,
// (W_2zp.e, W_2zp+1.e) for e = 0..3 (W = g_z (1, s_z, s_z^2, s_z^3)).  Quarters of the
// tile (4 planes) that the support misses are skipped.  The grid's last tile is only 8
// planes deep when M / 8 is odd; its planes beyond M are computed and not written.
using u64 = unsigned long long;
__device__ __forceinline__ u64 pack2(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(u64 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c)
{
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

constexpr int kTz = 16;    // planes per tile of spread16_kernel

// particles staged per chunk (the CTA's 64 threads stage up to CH of them at a time)
#ifndef SE_SPREAD16_CH
#define SE_SPREAD16_CH 60
#endif

template <int CH = SE_SPREAD16_CH> struct Spread16SmemT {
    float sxy[CH][2 * kTile];   // window weights x(8) y(8), entry e at e ^ ((k >> 1) & 15)
    float4 swz[CH][kTz];        // unit 2 zp + h: (W_2zp, W_2zp+1) of e = 2h, 2h + 1; at unit ^ (k & 7)
    float4 sp[CH][7];           // per-particle coefficients of the column polynomials (below)
    int bin_beg[6 * 6 * 7], bin_off[6 * 6 * 7 + 1];
};
using Spread16Smem = Spread16SmemT<>;

// The update of one particle's 16-plane column at lane column (tx, ty): the 13 column
// coefficients (gxy: the column's x-y weight; v0: the particle's first staged row), then the
// plane pairs of the quarters the support reaches, in packed FMAs.  Shared by the two-warp and
// the one-warp spreading blocks.
template <int NCOMP, typename SP, typename SWZ>
__device__ __forceinline__ void spread16_column(int k, int sw_z, float gxy, float4 v0, int tx, int ty, SP &sp,
                                                SWZ &swz, u64 (&acc2)[kTz / 2][4])
{
    const int quarters = (int)v0.z;
    const float sx = v0.x + tx, sy = v0.y + ty;
    const float r2 = sx * sx + sy * sy;
    const float4 v1 = sp[k][1], v2 = sp[k][2], v5 = sp[k][5];
    const float a0 = v1.x + v1.y * r2;
    const float F[3] = {v2.x, v2.y, v2.z};
    float c[3][4];
    if constexpr (NCOMP >= 6) {
        const float4 v3 = sp[k][3];
        const float kT0 = v2.w, kT1 = v3.x, kT2 = v3.y;
        // k (s x T)-terms of the velocity coefficients and k T-terms of the first moments
        const float t[3] = {-kT2 * sy, kT2 * sx, kT0 * sy - kT1 * sx};
        const float nk[3] = {kT1, -kT0, 0.f};
        if constexpr (NCOMP >= 11) {
            const float4 v4 = sp[k][4], v6 = sp[k][6];
            const float b0 = v1.z + v1.w * r2;
            const float S0 = v3.z, S1 = v3.w, S2 = v4.x, S3 = v4.y, S4 = v4.z, S5 = v4.w;
            const float d[3] = {S0 * sx + S3 * sy, S3 * sx + S1 * sy, S4 * sx + S5 * sy};
            const float Sp[3] = {S4, S5, S2}, B1Sp[3] = {v5.w, v6.x, v6.y};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                c[q][0] = a0 * F[q] + (b0 * d[q] + t[q]);
                c[q][1] = nk[q] + b0 * Sp[q];
                c[q][3] = B1Sp[q];
            }
            c[0][2] = v5.x + v1.w * d[0];
            c[1][2] = v5.y + v1.w * d[1];
            c[2][2] = v5.z + v1.w * d[2];
        } else {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                c[q][0] = a0 * F[q] + t[q];
                c[q][1] = nk[q];
                c[q][3] = 0;
            }
            c[0][2] = v5.x;
            c[1][2] = v5.y;
            c[2][2] = v5.z;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            c[q][0] = a0 * F[q];
            c[q][1] = 0;
            c[q][3] = 0;
        }
        c[0][2] = v5.x;
        c[1][2] = v5.y;
        c[2][2] = v5.z;
    }
    constexpr int NE = NCOMP >= 11 ? 4 : (NCOMP >= 6 ? 3 : 2);
    constexpr int ES[4] = {0, 2, 1, 3};       // the terms present: 0, 2 (F); 1 (T); 3 (S)
    u64 cc[3][4];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float v = c[q][e] * gxy;
            cc[q][e] = pack2(v, v);
        }
    const float csv = NCOMP >= 12 ? gxy * v0.w : 0.f;
    const u64 cs = pack2(csv, csv);
    auto quarter = [&](auto q0c) {
        constexpr int zq = decltype(q0c)::value;
#pragma unroll
        for (int zp = 2 * zq; zp < 2 * zq + 2; ++zp) {
            const ulonglong2 wa = *reinterpret_cast<const ulonglong2 *>(&swz[k][(2 * zp) ^ sw_z]);
            const ulonglong2 wb = *reinterpret_cast<const ulonglong2 *>(&swz[k][(2 * zp + 1) ^ sw_z]);
            const u64 Wp[4] = {wa.x, wa.y, wb.x, wb.y};
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int j = 0; j < NE; ++j) acc2[zp][q] = ffma2(cc[q][ES[j]], Wp[ES[j]], acc2[zp][q]);
            if constexpr (NCOMP >= 12) acc2[zp][3] = ffma2(cs, Wp[0], acc2[zp][3]);
        }
    };
    if (quarters & 1) quarter(std::integral_constant<int, 0>{});
    if (quarters & 2) quarter(std::integral_constant<int, 1>{});
    if (quarters & 4) quarter(std::integral_constant<int, 2>{});
    if (quarters & 8) quarter(std::integral_constant<int, 3>{});
}

template <int NCOMP, bool SPLIT, typename Sync, int CH = SE_SPREAD16_CH>
__device__ __forceinline__ void spread16_body(int tile, int part, int tid, Sync sync, Spread16SmemT<CH> &sm, SeParams p,
                                              const int *tile_start, const int *tile_perm, const int *base,
                                              const float *s0g, const float *wg, const double *rad, const float *xs,
                                              float *grid, int nsplit)
{
    constexpr int TT = kTile, TZ = kTz, NT = 64;      // threads
    auto &sxy = sm.sxy;
    auto &swz = sm.swz;
    auto &sp = sm.sp;
    auto &bin_beg = sm.bin_beg;
    auto &bin_off = sm.bin_off;
    const int M = p.M, P = p.P, nt = p.ntile;
    const int bx0 = tile % nt, by0 = (tile / nt) % nt, bzp = tile / (nt * nt);
    const int t0[3] = {bx0 * TT, by0 * TT, bzp * TZ};
    const int tz_planes = min(TZ, M - t0[2]);           // 16, or 8 for the last tile of an odd nt
    const int tx = tid & 7, ty = tid >> 3;
    const int nbin = (P - 1 + TT - 1) / TT + 1;
    const int nbz = nbin + (tz_planes > TT ? 1 : 0);    // z-bins: the top bin of the tile and nbz - 1 below
    const int bztop = 2 * bzp + (tz_planes > TT ? 1 : 0);
    const int nb3 = nbin * nbin * nbz;
    const float alpha = (float)p.alpha, kap = (float)p.kappa, akap = alpha * kap;
    u64 acc2[TZ / 2][4];
#pragma unroll
    for (int z = 0; z < TZ / 2; ++z)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc2[z][c] = 0ull;

    for (int bb = tid; bb < nb3; bb += NT) {
        const int bx = bb % nbin, by = (bb / nbin) % nbin, bz = bb / (nbin * nbin);
        const int bin = (wrapi(bztop - bz, nt) * nt + wrapi(by0 - by, nt)) * nt + wrapi(bx0 - bx, nt);
        bin_beg[bb] = tile_start[bin];
        bin_off[bb + 1] = tile_start[bin + 1] - tile_start[bin];
    }
    sync();
    if (tid == 0) {
        bin_off[0] = 0;
        for (int bb = 0; bb < nb3; ++bb) bin_off[bb + 1] += bin_off[bb];
    }
    sync();
    const int total = bin_off[nb3];

    int cbeg = 0, cstep = CH;
    if constexpr (SPLIT) {
        grid += (size_t)part * M * M * M * 4;
        cbeg = part * CH;
        cstep = nsplit * CH;
    }
    for (int c0 = cbeg; c0 < total; c0 += cstep) {
        const int cnt = min(CH, total - c0);
        sync();
        if ((int)tid < cnt) {
            const int k = tid, idx = c0 + k;
            int lo = 0, hi = nb3;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (bin_off[mid] <= idx) lo = mid; else hi = mid;
            }
            const int i = tile_perm[bin_beg[lo] + idx - bin_off[lo]];
            bool ok = true;
            int od[3];
            for (int d = 0; d < 3; ++d) {
                int o = wrapi(t0[d] - base[3 * i + d], M);
                if (o >= P) o -= M;
                ok &= (o < P) && (o > -(d == 2 ? TZ : TT));
                od[d] = o;
            }
            const float *w = wg + (size_t)i * 3 * P;
            const int sw_xy = (k >> 1) & 15, sw_z = k & 7;
#pragma unroll
            for (int t = 0; t < TT; ++t) {
                const int ix = od[0] + t, iy = od[1] + t;
                sxy[k][t ^ sw_xy] = (ix >= 0 && ix < P) ? w[ix] : 0.f;
                sxy[k][(TT + t) ^ sw_xy] = (iy >= 0 && iy < P) ? w[P + iy] : 0.f;
            }
            const float s0z = s0g[3 * i + 2];
#pragma unroll
            for (int zp = 0; zp < TZ / 2; ++zp) {
                float4 W[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int iz = od[2] + 2 * zp + h;
                    const float g = (iz >= 0 && iz < P) ? w[2 * P + iz] : 0.f;
                    const float sz = s0z + (float)iz;
                    W[h] = make_float4(g, g * sz, g * sz * sz, g * sz * sz * sz);
                }
                swz[k][(2 * zp) ^ sw_z] = make_float4(W[0].x, W[1].x, W[0].y, W[1].y);
                swz[k][(2 * zp + 1) ^ sw_z] = make_float4(W[0].z, W[1].z, W[0].w, W[1].w);
            }
            const float a = (float)rad[i], a2k2 = a * a * kap * kap;
            const float *xi = xs + (size_t)i * kNC;
            float S[6] = {0, 0, 0, 0, 0, 0}, Tq[3] = {0, 0, 0};
            if constexpr (NCOMP >= 6) { Tq[0] = xi[3]; Tq[1] = xi[4]; Tq[2] = xi[5]; }
            if constexpr (NCOMP >= 11) stresslet_tensor(xi + 6, S);
            // quarters (4 planes each) of the tile that the support reaches
            const int zlo = max(0, -od[2]), zhi = min(tz_planes, P - od[2]);
            int quarters = 0;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq)
                if (zlo < 4 * qq + 4 && zhi > 4 * qq) quarters |= 1 << qq;
            // Column coefficients of the real-space approach (s = (sx, sy) the column's
            // offset, r2 = sx^2 + sy^2, k = alpha kappa):
            //   c_q0 = a0 F_q + b0 (S s)_q + k (s x T)-term,  c_q1 = k T-term + b0 (S_xz, S_yz, S_zz)_q,
            //   c_q2 = A1 F_q + B1 (S s)_q,  c_q3 = B1 (S_xz, S_yz, S_zz)_q,
            // a0 = A0 + A1 r2, b0 = B0 + B1 r2 (the Faxen weights of the force and stresslet
            // terms, which cancel near r2 = -A0/A1 and -B0/B1: formed per column as scalars
            // before they multiply the moments).  Products of particle constants that do
            // not cancel (k T, A1 F, B1 S) are formed here once.
            const float A0 = 1 - a2k2 * alpha, A1 = (2.0f / 3.0f) * a2k2 * alpha * alpha;
            const float B0 = 2 * kap * alpha * (1 - a2k2 * alpha), B1 = 0.8f * kap * a2k2 * alpha * alpha * alpha;
            sp[k][0] = make_float4(s0g[3 * i] + (float)od[0], s0g[3 * i + 1] + (float)od[1],
                                   ok ? (float)quarters : 0.f, NCOMP >= 12 ? xi[11] : 0.f);
            sp[k][1] = make_float4(A0, A1, B0, B1);
            sp[k][2] = make_float4(xi[0], xi[1], xi[2], akap * Tq[0]);
            sp[k][3] = make_float4(akap * Tq[1], akap * Tq[2], S[0], S[1]);
            sp[k][4] = make_float4(S[2], S[3], S[4], S[5]);
            sp[k][5] = make_float4(A1 * xi[0], A1 * xi[1], A1 * xi[2], B1 * S[4]);
            sp[k][6] = make_float4(B1 * S[5], B1 * S[2], 0.f, 0.f);
        }
        sync();
        for (int k = 0; k < cnt; ++k) {
            const int sw_xy = (k >> 1) & 15, sw_z = k & 7;
            const float gxy = sxy[k][tx ^ sw_xy] * sxy[k][(TT + ty) ^ sw_xy];
            const float4 v0 = sp[k][0];
            const int quarters = (int)v0.z;
            if (gxy == 0.f || quarters == 0) continue;
            spread16_column<NCOMP>(k, sw_z, gxy, v0, tx, ty, sp, swz, acc2);
        }
    }
#pragma unroll
    for (int zp = 0; zp < TZ / 2; ++zp) {
        float lo[4], hi[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) unpack2(acc2[zp][q], lo[q], hi[q]);
        const int z = 2 * zp;
        if (z < tz_planes) {
            const size_t gi = (((size_t)(t0[2] + z) * M + (t0[1] + ty)) * M + (t0[0] + tx)) * 4;
            *reinterpret_cast<float4 *>(grid + gi) = make_float4(lo[0], lo[1], lo[2], NCOMP >= 12 ? lo[3] : 0.f);
            *reinterpret_cast<float4 *>(grid + gi + (size_t)M * M * 4) =
                make_float4(hi[0], hi[1], hi[2], NCOMP >= 12 ? hi[3] : 0.f);
        }
    }
}

#ifndef SE_SPREAD16_MINB
#define SE_SPREAD16_MINB 8
#endif

template <int NCOMP, bool SPLIT>
__global__ void __launch_bounds__(64, SE_SPREAD16_MINB) spread16_kernel(SeParams p, const int *tile_start, const int *tile_perm,
                                                         const int *base, const float *s0g, const float *wg,
                                                         const double *rad, const float *xs, float *grid, int nsplit)
{
    __shared__ Spread16Smem sm;
    spread16_body<NCOMP, SPLIT>(blockIdx.x, blockIdx.y, threadIdx.x, [] { __syncthreads(); }, sm, p, tile_start,
                                tile_perm, base, s0g, wg, rad, xs, grid, nsplit);
}

#include "se_spread16w.cuh"

// Self coefficients of particle i (FP64, once per configuration): the isolated sphere
// (Eqs. faxen-f/t/s/p: 1/(6 pi eta a), 1/(8 pi eta a^3), 3/(20 pi eta a^3),
// 3/(16 pi eta a^3)) minus the self term that the wave-space sum contains (Eq. uf-self
// for U and its torque and stresslet analogues; the source-pressure coupling has none).
template <typename T>
__global__ void self_coef_kernel(int N, double xi, double eta, const double *rad, T *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double a = rad[i], a2 = a * a, x2 = xi * xi, pi32 = kPi * sqrt(kPi);
    out[4 * i] = (T)(1.0 / (6 * kPi * eta * a) - xi * (9 - 10 * a2 * x2 + 7 * a2 * a2 * x2 * x2) / (18 * pi32 * eta));
    out[4 * i + 1] = (T)(1.0 / (8 * kPi * eta * a * a2) - 5 * xi * x2 / (12 * pi32 * eta));
    out[4 * i + 2] = (T)(3.0 / (20 * kPi * eta * a * a2) -
                         xi * x2 * (25 - 42 * a2 * x2 + 27 * a2 * a2 * x2 * x2) / (50 * pi32 * eta));
    out[4 * i + 3] = (T)(3.0 / (16 * kPi * eta * a * a2));
}

// grid = sum over the nsplit partial grids, in part order
template <typename T>
__global__ void sum_parts_kernel(size_t n4, int nsplit, const T *parts, T *grid)
{
    using T4 = typename V4<T>::t;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n4) return;
    const T4 *p = reinterpret_cast<const T4 *>(parts) + e;
    T4 s = p[0];
    for (int q = 1; q < nsplit; ++q) {
        const T4 v = p[(size_t)q * n4];
        s.x += v.x;
        s.y += v.y;
        s.z += v.z;
        s.w += v.w;
    }
    reinterpret_cast<T4 *>(grid)[e] = s;
}

// ---------------------------------------------------------------- FFT passes
//
// Each pass moves a chunk of lines into shared memory with 16-byte asynchronous
// copies (the whole chunk in flight at once), transforms it there (se_fft.cuh) and
// writes it back with coalesced stores; four CTAs of 256 threads per SM at the usual
// grid sizes, so the copies of one CTA overlap the arithmetic of the others.  The
// shared buffers hold NL element-major lines of up to M + 2 elements.

template <typename T> constexpr int fft_nl() { return sizeof(T) == 4 ? 16 : 8; }
constexpr int kFftThreads = 256;

// shared layout of a pass: twiddles [M], two line buffers [NLB (M + 2)]
template <typename T2>
__device__ __forceinline__ void fft_smem(unsigned char *sm, int M, int NLB, T2 *&tw, T2 *&A, T2 *&B)
{
    tw = reinterpret_cast<T2 *>(sm);
    A = tw + ((M + 1) & ~1);
    B = A + (size_t)NLB * (M + 2);
}

// The passes below are device functions of (CTA index, shared buffer) so that the
// persistent batched kernel runs the same code; each __global__ wrapper passes its
// blockIdx and dynamic shared memory.

// x pass, forward: each grid row (y, z) carries CF real series (4, or 8 in the
// wave-space approach) packed as CF/2 complex lines (H0 + i H1, H2 + i H3, ...); after
// the transform the half spectra q = 0..M/2 are separated using Z(-q) = conj(Z(q)) of
// real data.
template <typename T, int CF = 4>
__device__ __forceinline__ void fft_x_fwd_body(int bx, unsigned char *sm, const FftPlan &plan,
                                               const typename C2<T>::t *twg, const T *grid, typename C2<T>::t *spec)
{
    using T2 = typename C2<T>::t;
    constexpr int NL = fft_nl<T>(), NCL = CF / 2, NR = NL / NCL;   // complex lines, per row, grid rows
    constexpr int CPE = sizeof(T) == 4 ? 2 : 1, NCH = NCL / CPE;     // complex per 16-byte copy, copies per point
    const int M = plan.M, Mh = M / 2 + 1;
    T2 *tw, *A, *B;
    fft_smem(sm, M, NL, tw, A, B);
    for (int e = threadIdx.x; e < M; e += blockDim.x) tw[e] = twg[e];
    const size_t row0 = (size_t)bx * NR;
    // copy h of row r at x (CPE complex lines) -> lines NCL r + CPE h .. at element x
    for (int e = threadIdx.x; e < NCH * NR * M; e += blockDim.x) {
        const int h = e % NCH, r = (e / NCH) % NR, x = e / NCH / NR;
        cp_async16(A + x * NL + NCL * r + CPE * h, grid + ((row0 + r) * M + x) * CF + 2 * CPE * h);
    }
    cp_async_wait_all();
    __syncthreads();
    const T2 *Z = fft_run_dir<NL, false>(A, B, plan, tw);
    for (int e = threadIdx.x; e < NR * Mh * NCL; e += blockDim.x) {
        const int h = e % NCL, r = (e / NCL) % NR, q = (e / NCL) / NR;
        const T2 z = Z[q * NL + NCL * r + h];
        const T2 zm = Z[(q == 0 ? 0 : M - q) * NL + NCL * r + h];
        T2 *o = spec + ((row0 + r) * Mh + q) * CF + 2 * h;
        o[0] = T2{(T)0.5 * (z.x + zm.x), (T)0.5 * (z.y - zm.y)};
        o[1] = T2{(T)0.5 * (z.y + zm.y), (T)-0.5 * (z.x - zm.x)};
    }
}

template <typename T, int CF = 4>
__global__ void __launch_bounds__(kFftThreads, 4) fft_x_fwd(FftPlan plan, const typename C2<T>::t *twg,
                                                            const T *grid, typename C2<T>::t *spec)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    fft_x_fwd_body<T, CF>(blockIdx.x, smraw, plan, twg, grid, spec);
}

// y pass (forward or inverse) in place on half spectra [z][y][q][C]: a CTA takes the
// NL / C wave numbers q0.. of one z plane, all C components, lines along y.
template <typename T, int C, bool INV>
__device__ __forceinline__ void fft_y_body(int bx, int by, unsigned char *sm, const FftPlan &plan,
                                           const typename C2<T>::t *twg, typename C2<T>::t *data)
{
    using T2 = typename C2<T>::t;
    constexpr int NL = fft_nl<T>(), LB = NL / C, CPE = sizeof(T) == 4 ? 2 : 1;   // complex per copy
    const int M = plan.M, Mh = M / 2 + 1;
    T2 *tw, *A, *B;
    fft_smem(sm, M, NL, tw, A, B);
    for (int e = threadIdx.x; e < M; e += blockDim.x) tw[e] = twg[e];
    const int q0 = bx * LB, nv = min(LB, Mh - q0) * C;     // valid lines
    const size_t base = ((size_t)by * M * Mh + q0) * C, es = (size_t)Mh * C;
    for (int e = threadIdx.x; e < (NL / CPE) * M; e += blockDim.x) {
        const int k = e % (NL / CPE), y = e / (NL / CPE);
        T2 *d = A + y * NL + k * CPE;
        if (k * CPE < nv) cp_async16(d, data + base + y * es + k * CPE);
        else
            for (int u = 0; u < CPE; ++u) d[u] = T2{0, 0};
    }
    cp_async_wait_all();
    __syncthreads();
    const T2 *Z = fft_run_dir<NL, INV>(A, B, plan, tw);
    for (int e = threadIdx.x; e < NL * M; e += blockDim.x) {
        const int l = e % NL, y = e / NL;
        if (l < nv) data[base + y * es + l] = Z[y * NL + l];
    }
}

template <typename T, int C, bool INV>
__global__ void __launch_bounds__(kFftThreads, 4) fft_y(FftPlan plan, const typename C2<T>::t *twg,
                                                        typename C2<T>::t *data)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    fft_y_body<T, C, INV>(blockIdx.x, blockIdx.y, smraw, plan, twg, data);
}

// z pass: forward transform of the 4 spectra, k-space scaling (see the file
// header), inverse transform of the CO output spectra.  A CTA takes LB wave numbers
// q0.. of one y row (LB = 4 for FP32 and 2 for FP64 while the buffers fit in shared
// memory); input lines q * 4 + c, output lines q * CO + c (the component order of the
// arrays in HBM).
// CI = 8 (the wave-space approach): the input spectra are H0 (3), Ha (3), H_src, 0 and
// the force density is H = H0 - k^2 Ha (the source Faxen operators in wave space).
template <typename T, int CO, int LB, int CI = 4>
__device__ __forceinline__ void fft_z_scale_body(int bx, int by, unsigned char *sm, const FftPlan &plan,
                                                 const typename C2<T>::t *twg, const typename C2<T>::t *specf,
                                                 typename C2<T>::t *speco, T cnorm, T twopiL, T i4x2, T ecoef,
                                                 T gam = (T)0)
{
    using T2 = typename C2<T>::t;
    constexpr int NLI = CI * LB, NLO = LB * CO, CPE = sizeof(T) == 4 ? 2 : 1;
    static_assert(NLI <= NLO, "the output line buffers hold the input lines");
    const int M = plan.M, Mh = M / 2 + 1;
    T2 *tw, *A, *B;
    fft_smem(sm, M, NLO, tw, A, B);
    for (int e = threadIdx.x; e < M; e += blockDim.x) tw[e] = twg[e];
    const int y = by;
    const int q0 = bx * LB, nq = min(LB, Mh - q0);
    const size_t zs = (size_t)M * Mh;                      // z stride in q units
    for (int e = threadIdx.x; e < (NLI / CPE) * M; e += blockDim.x) {
        const int k = e % (NLI / CPE), z = e / (NLI / CPE);
        T2 *d = A + z * NLI + k * CPE;
        if (k * CPE < nq * CI) cp_async16(d, specf + ((size_t)z * zs + (size_t)y * Mh + q0) * CI + k * CPE);
        else
            for (int u = 0; u < CPE; ++u) d[u] = T2{0, 0};
    }
    cp_async_wait_all();
    __syncthreads();
    T2 *X = fft_run_dir<NLI, false>(A, B, plan, tw);
    T2 *Y = X == A ? B : A;

    const int ys = y <= M / 2 ? y : y - M;
    for (int e = threadIdx.x; e < LB * M; e += blockDim.x) {
        const int q = e % LB, z = e / LB;
        const int qx = q0 + q, zsn = z <= M / 2 ? z : z - M;
        T2 o[CO];
#pragma unroll
        for (int c = 0; c < CO; ++c) o[c] = T2{0, 0};
        const bool zero = q >= nq || (qx == 0 && ys == 0 && zsn == 0) || 2 * qx == M || 2 * ys == M ||
                          2 * zsn == M;
        if (!zero) {
            // k = (2 pi / L)(q1, q2 - gamma q1, q3): the reciprocal lattice of the sheared cell
            const T kx = twopiL * qx, ky = twopiL * ((T)ys - gam * (T)qx), kz = twopiL * zsn;
            const T k2 = kx * kx + ky * ky + kz * kz;
            const T q2 = (T)(qx * qx + ys * ys + zsn * zsn);
            const T ex = -k2 * i4x2 + ecoef * q2;
            T E;
            if constexpr (sizeof(T) == 4) E = expf(ex) * cnorm;
            else E = exp(ex) * cnorm;
            const T ik2 = 1 / k2;
            const T Phi = E * (1 + k2 * i4x2) * ik2;
            const T2 *h = X + z * NLI + q * CI;
            T2 H0 = h[0], H1 = h[1], H2 = h[2], Hs = h[3];
            if constexpr (CI == 8) {
                H0 = T2{h[0].x - k2 * h[3].x, h[0].y - k2 * h[3].y};
                H1 = T2{h[1].x - k2 * h[4].x, h[1].y - k2 * h[4].y};
                H2 = T2{h[2].x - k2 * h[5].x, h[2].y - k2 * h[5].y};
                Hs = h[6];
            }
            const T2 kH = T2{kx * H0.x + ky * H1.x + kz * H2.x, kx * H0.y + ky * H1.y + kz * H2.y};
            const T2 pr = T2{kH.x * ik2, kH.y * ik2};
            // This FFT's forward transform carries exp(-i q.n), so Hhat(q) holds the moments'
            // structure factor at -k: the odd (i k) factors below are taken at -k.
            const T sq = -E * (T)0.25 * ik2;           // -i k/(4 k^2) E H_src
            const T2 iHs = T2{-Hs.y * sq, Hs.x * sq};
            o[0] = T2{Phi * (H0.x - kx * pr.x) + kx * iHs.x, Phi * (H0.y - kx * pr.y) + kx * iHs.y};
            o[1] = T2{Phi * (H1.x - ky * pr.x) + ky * iHs.x, Phi * (H1.y - ky * pr.y) + ky * iHs.y};
            o[2] = T2{Phi * (H2.x - kz * pr.x) + kz * iHs.x, Phi * (H2.y - kz * pr.y) + kz * iHs.y};
            const T cp = (T)-0.75 * E;                  // -(3/4) c E i k.H / k^2
            const T2 op = T2{-cp * pr.y, cp * pr.x};
            if constexpr (CO == 8) {
                o[3] = T2{-k2 * o[0].x, -k2 * o[0].y};
                o[4] = T2{-k2 * o[1].x, -k2 * o[1].y};
                o[5] = T2{-k2 * o[2].x, -k2 * o[2].y};
                o[6] = op;
            } else {
                o[3] = op;
            }
        }
        T2 *w = Y + z * NLO + q * CO;
#pragma unroll
        for (int c = 0; c < CO; ++c) w[c] = o[c];
    }
    __syncthreads();
    const T2 *Z = fft_run_dir<NLO, true>(Y, X, plan, tw);
    for (int e = threadIdx.x; e < NLO * M; e += blockDim.x) {
        const int l = e % NLO, z = e / NLO;
        if (l < nq * CO) speco[((size_t)z * zs + (size_t)y * Mh + q0) * CO + l] = Z[z * NLO + l];
    }
}

template <typename T, int CO, int LB, int CI = 4>
__global__ void __launch_bounds__(kFftThreads, 4) fft_z_scale(FftPlan plan, const typename C2<T>::t *twg,
                                                              const typename C2<T>::t *specf,
                                                              typename C2<T>::t *speco, T cnorm, T twopiL, T i4x2,
                                                              T ecoef, T gam)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    fft_z_scale_body<T, CO, LB, CI>(blockIdx.x, blockIdx.y, smraw, plan, twg, specf, speco, cnorm, twopiL, i4x2,
                                    ecoef, gam);
}

// z pass with a tabulated radial kernel in place of the Ewald one (the coarse spectral
// correction of SE_PRECOND_SPECTRAL): forward z transform of the force spectra, the
// transverse projection times h(|k|) for |k| <= kmax (zero beyond), the window
// compensation exp(2 pi^2 q^2/(alpha M^2)) (alpha/pi)^3 of the spread and gather
// Gaussians, inverse z transform.  The source and pressure outputs are zero.
template <typename T, int LB>
__global__ void __launch_bounds__(kFftThreads, 4) fft_z_table(FftPlan plan, const typename C2<T>::t *twg,
                                                              const typename C2<T>::t *specf,
                                                              typename C2<T>::t *speco, const T *tab, int ntab,
                                                              T kmax, T cnorm, T twopiL, T ecoef, T gam)
{
    using T2 = typename C2<T>::t;
    constexpr int NLI = 4 * LB, CO = 4, NLO = LB * CO, CPE = sizeof(T) == 4 ? 2 : 1;
    const int M = plan.M, Mh = M / 2 + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    T2 *tw, *A, *B;
    fft_smem(smraw, M, NLO, tw, A, B);
    for (int e = threadIdx.x; e < M; e += blockDim.x) tw[e] = twg[e];
    const int y = blockIdx.y;
    const int q0 = blockIdx.x * LB, nq = min(LB, Mh - q0);
    const size_t zs = (size_t)M * Mh;
    for (int e = threadIdx.x; e < (NLI / CPE) * M; e += blockDim.x) {
        const int k = e % (NLI / CPE), z = e / (NLI / CPE);
        T2 *d = A + z * NLI + k * CPE;
        if (k * CPE < nq * 4) cp_async16(d, specf + ((size_t)z * zs + (size_t)y * Mh + q0) * 4 + k * CPE);
        else
            for (int u = 0; u < CPE; ++u) d[u] = T2{0, 0};
    }
    cp_async_wait_all();
    __syncthreads();
    T2 *X = fft_run_dir<NLI, false>(A, B, plan, tw);
    T2 *Y = X == A ? B : A;
    const int ys = y <= M / 2 ? y : y - M;
    const T dk = kmax / (T)(ntab - 1);
    for (int e = threadIdx.x; e < LB * M; e += blockDim.x) {
        const int q = e % LB, z = e / LB;
        const int qx = q0 + q, zsn = z <= M / 2 ? z : z - M;
        T2 o[CO];
#pragma unroll
        for (int c = 0; c < CO; ++c) o[c] = T2{0, 0};
        // k = (2 pi / L)(q1, q2 - gamma q1, q3) (the sheared cell's reciprocal lattice)
        const T kx = twopiL * qx, ky = twopiL * ((T)ys - gam * (T)qx), kz = twopiL * zsn;
        const T k2 = kx * kx + ky * ky + kz * kz;
        const bool zero = q >= nq || (qx == 0 && ys == 0 && zsn == 0) || 2 * qx == M || 2 * ys == M ||
                          2 * zsn == M || k2 > kmax * kmax;
        if (!zero) {
            const T kk = sqrt(k2), u = kk / dk;
            const int i0 = min((int)u, ntab - 2);
            const T f = u - (T)i0;
            const T hk = tab[i0] + f * (tab[i0 + 1] - tab[i0]);
            const T q2 = (T)(qx * qx + ys * ys + zsn * zsn);
            T E;
            if constexpr (sizeof(T) == 4) E = expf(ecoef * q2) * cnorm * hk;
            else E = exp(ecoef * q2) * cnorm * hk;
            const T ik2 = 1 / k2;
            const T2 *hh = X + z * NLI + q * 4;
            const T2 H0 = hh[0], H1 = hh[1], H2 = hh[2];
            const T2 kH = T2{kx * H0.x + ky * H1.x + kz * H2.x, kx * H0.y + ky * H1.y + kz * H2.y};
            const T2 pr = T2{kH.x * ik2, kH.y * ik2};
            o[0] = T2{E * (H0.x - kx * pr.x), E * (H0.y - kx * pr.y)};
            o[1] = T2{E * (H1.x - ky * pr.x), E * (H1.y - ky * pr.y)};
            o[2] = T2{E * (H2.x - kz * pr.x), E * (H2.y - kz * pr.y)};
        }
        T2 *wv = Y + z * NLO + q * CO;
#pragma unroll
        for (int c = 0; c < CO; ++c) wv[c] = o[c];
    }
    __syncthreads();
    const T2 *Z = fft_run_dir<NLO, true>(Y, X, plan, tw);
    for (int e = threadIdx.x; e < NLO * M; e += blockDim.x) {
        const int l = e % NLO, z = e / NLO;
        if (l < nq * CO) speco[((size_t)z * zs + (size_t)y * Mh + q0) * CO + l] = Z[z * NLO + l];
    }
}

// x pass, inverse: pairs of half spectra are recombined into full complex lines
// Z = A + i B (A(M-q) = conj A(q) for real output), transformed, and written as the
// real grids A, B interleaved per point.
template <typename T, int CO>
__device__ __forceinline__ void fft_x_inv_body(int bx, unsigned char *sm, const FftPlan &plan,
                                               const typename C2<T>::t *twg, const typename C2<T>::t *speco, T *grid)
{
    using T2 = typename C2<T>::t;
    constexpr int NL = fft_nl<T>(), NP = CO / 2, NR = NL / NP, CPE = sizeof(T) == 4 ? 2 : 1;
    const int M = plan.M, Mh = M / 2 + 1;
    T2 *tw, *A, *B;
    fft_smem(sm, M, NL, tw, A, B);
    for (int e = threadIdx.x; e < M; e += blockDim.x) tw[e] = twg[e];
    const size_t row0 = (size_t)bx * NR;
    // the NR rows of half spectra are contiguous in HBM: stage them raw in B
    const int nraw = NR * Mh * CO;
    const T2 *src = speco + row0 * Mh * CO;
    for (int e = threadIdx.x; e < nraw / CPE; e += blockDim.x) cp_async16(B + e * CPE, src + e * CPE);
    cp_async_wait_all();
    __syncthreads();
    for (int e = threadIdx.x; e < NL * M; e += blockDim.x) {
        const int l = e % NL, x = e / NL, r = l / NP, pp = l - r * NP;
        const T2 *s = B + (size_t)r * Mh * CO + 2 * pp;
        T2 z;
        if (x <= M / 2) {
            const T2 a = s[x * CO], b = s[x * CO + 1];
            z = T2{a.x - b.y, a.y + b.x};
        } else {
            const T2 a = s[(M - x) * CO], b = s[(M - x) * CO + 1];
            z = T2{a.x + b.y, -a.y + b.x};
        }
        A[x * NL + l] = z;
    }
    __syncthreads();
    const T2 *Z = fft_run_dir<NL, true>(A, B, plan, tw);
    for (int e = threadIdx.x; e < NR * M; e += blockDim.x) {
        const int r = e % NR, x = e / NR;
        const T2 *s = Z + x * NL + r * NP;
        T *g = grid + ((row0 + r) * M + x) * CO;
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) {
            g[2 * pp] = s[pp].x;
            g[2 * pp + 1] = s[pp].y;
        }
    }
}

template <typename T, int CO>
__global__ void __launch_bounds__(kFftThreads, 4) fft_x_inv(FftPlan plan, const typename C2<T>::t *twg,
                                                            const typename C2<T>::t *speco, T *grid)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    fft_x_inv_body<T, CO>(blockIdx.x, smraw, plan, twg, speco, grid);
}

// ---------------------------------------------------------------- gather + combine

template <typename T>
__device__ __forceinline__ void kahan_add(T &sum, T &comp, T v)
{
    const T y = v - comp;
    const T t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// Wave sums acc[13] of particle i (internal order) -> outputs in the caller's order:
// Omega = alpha kappa sum g (s x v), E on the orthonormal basis from the symmetric sums,
// plus the real-space part and the self terms: isolated sphere (Eqs. faxen-f/t/s/p)
// minus the self term in the wave sum (Eq. uf-self and its torque/stresslet analogues).
template <typename T, typename TO, int CO>
__device__ __forceinline__ void combine_write(const SeParams &p, const T (&acc)[13], int i, const T *selfc,
                                              const int *perm, const T *xs, const T *yreal, TO *y,
                                              int ncomp_out, int with_self)
{
    const T alpha = (T)p.alpha, kap = (T)p.kappa;
    T out[kNC];
    out[0] = acc[0];
    out[1] = acc[1];
    out[2] = acc[2];
    const T ak = alpha * kap;
    out[3] = ak * acc[3];
    out[4] = ak * acc[4];
    out[5] = ak * acc[5];
    {
        // symmetric tensor A (xx yy zz xy xz yz) with off-diagonals stored as 2*A_xy
        const T f = CO == 8 ? 2 * alpha * kap : (T)1;
        const T Axx = f * acc[6], Ayy = f * acc[7], Azz = f * acc[8];
        const T Axy = f * acc[9] * (T)0.5, Axz = f * acc[10] * (T)0.5, Ayz = f * acc[11] * (T)0.5;
        const T r2 = (T)0.70710678118654752440, r6 = (T)0.40824829046386301637, s2 = (T)1.41421356237309504880;
        out[6] = r2 * (Axx - Ayy);
        out[7] = r6 * (2 * Azz - Axx - Ayy);
        out[8] = s2 * Axy;
        out[9] = s2 * Axz;
        out[10] = s2 * Ayz;
    }
    out[11] = acc[12];
    const T *xi_ = xs + (size_t)i * kNC;
    const T *yr = yreal + (size_t)i * kNC;
    T sc[4] = {0, 0, 0, 0};
    if (with_self) {
        sc[0] = selfc[4 * i];
        sc[1] = selfc[4 * i + 1];
        sc[2] = selfc[4 * i + 2];
        sc[3] = selfc[4 * i + 3];
    }
    TO *yo = y + (size_t)perm[i] * ncomp_out;
#pragma unroll
    for (int c = 0; c < kNC; ++c)
        if (c < ncomp_out) yo[c] = (TO)(out[c] + yr[c] + sc[c < 3 ? 0 : (c < 6 ? 1 : (c < 11 ? 2 : 3))] * xi_[c]);
}

// One warp per particle: trapezoid-rule convolution of the gathered grids with the
// particle's Gaussian (and its derivatives) over the P^3 support, then
// y = real + wave + self, written in the caller's order and dtype.
// The Gaussian is separable and every target weight is a polynomial of degree <= 3
// in s_z times g_z, so each lane (one (x, y) column of the support) sums the column
// against the per-warp table W_k = g_z (1, s_z, s_z^2, s_z^3) held in shared memory
// (13 FMAs per grid point) and converts the column moments into the 13 outputs
// U(3), s x v (3), sym(s (x) w) (6: xx yy zz, xy xz yz doubled), p (1) once per column.
// Column contributions are Kahan-compensated across the P^2 / 32 columns of a lane.
// The work of warp w_ (particle order[w_]); Wz and Zi: the warp's 32-entry tables.
template <typename T, typename TO, int CO, int NCOMP, int NCL = 1>
__device__ __forceinline__ void gather_body(int w_, int lane, typename V4<T>::t *Wz, int *Zi, const SeParams &p,
                                            int N, const int *order, const int *base, const T *s0g, const T *wg,
                                            const double *rad, const T *selfc, const int *perm, const T *grid,
                                            const T *xs, const T *yreal, TO *y, int ncomp_out, int with_wave,
                                            int with_self)
{
    constexpr int NA = 13;
    using T4 = typename V4<T>::t;
    if (w_ >= N) return;
    const int i = order ? order[w_] : w_;
    const int M = p.M, P = p.P;
    const double ad = rad[i];
    const T a = (T)ad;
    T acc[NA];
#pragma unroll
    for (int c = 0; c < NA; ++c) acc[c] = 0;
    const T alpha = (T)p.alpha, kap = (T)p.kappa;
    if (with_wave) {
        T cmp[NA];
#pragma unroll
        for (int c = 0; c < NA; ++c) cmp[c] = 0;
        const int bx = base[3 * i], by = base[3 * i + 1], bz = base[3 * i + 2];
        const T sx0 = s0g[3 * i], sy0 = s0g[3 * i + 1], sz0 = s0g[3 * i + 2];
        const T *wx = wg + (size_t)i * 3 * P, *wy = wx + P, *wz = wy + P;
        if (lane < P) {
            const T g = wz[lane], sz = sz0 + lane;
            Wz[lane] = T4{g, g * sz, g * sz * sz, g * sz * sz * sz};
            Zi[lane] = wrapi(bz + lane, M);
        }
        __syncwarp();
        const T a2k2 = a * a * kap * kap;
        // real-space approach weights (Faxen Laplacian on the Gaussian)
        const T A0 = 1 - a2k2 * alpha, A1 = (T)(2.0 / 3.0) * a2k2 * alpha * alpha;
        const T B0 = 2 * kap * alpha * (1 - a2k2 * alpha);
        const T B1 = (T)0.8 * kap * a2k2 * alpha * alpha * alpha;
        const T c6 = a * a / 6, c10 = a * a / 10;
        const size_t zs = (size_t)M * M * CO;
        // NCL = 2 (FP32, 4-component grids, P^2 close to a multiple of 64): each lane takes two
        // columns at a time, so that one read of a plane's W and offset (shared memory, the
        // same for every lane) serves two points.  A lane's columns are summed in the order
        // c = lane, lane + 32, ... either way.
        constexpr int kUnr = kGatherUnroll;
        for (int it = 0; it < P * P; it += 32 * NCL) {
            int cxa[NCL], cya[NCL];
            bool acta[NCL];
            const T *gpa[NCL];
            // column moments: Z0..Z3 of v (and of v'' in the hybrid mode), Zp of p
            T z0[NCL][3], z1[NCL][3], z2[NCL][3], z3[NCL][3], zp[NCL];
            bool any = false;
#pragma unroll
            for (int j = 0; j < NCL; ++j) {
                const int c = it + 32 * j + lane;
                acta[j] = c < P * P;
                any |= acta[j];
                cya[j] = acta[j] ? c / P : 0;
                cxa[j] = acta[j] ? c - cya[j] * P : 0;
                gpa[j] = grid + ((size_t)wrapi(by + cya[j], M) * M + wrapi(bx + cxa[j], M)) * CO;
#pragma unroll
                for (int q = 0; q < 3; ++q) z0[j][q] = z1[j][q] = z2[j][q] = z3[j][q] = 0;
                zp[j] = 0;
            }
            if (any) {
                auto plane = [&](int k, size_t off) {
                    const T4 w = Wz[k];
#pragma unroll
                    for (int j = 0; j < NCL; ++j) {
                        const T4 u0 = *reinterpret_cast<const T4 *>(gpa[j] + off);
                        if constexpr (CO == 8) {
                            const T4 u1 = *reinterpret_cast<const T4 *>(gpa[j] + off + 4);
                            // u0 = (v0 v1 v2 v''0), u1 = (v''1 v''2 p -): z0 = sum g v, z1 = sum g v'',
                            // z2 = sum g s_z v, z3 = sum g s_z v''
                            lazy_madd(z0[j][0], w.x, u0.x); lazy_madd(z0[j][1], w.x, u0.y); lazy_madd(z0[j][2], w.x, u0.z);
                            lazy_madd(z1[j][0], w.x, u0.w); lazy_madd(z1[j][1], w.x, u1.x); lazy_madd(z1[j][2], w.x, u1.y);
                            if constexpr (NCOMP >= 6) {
                                lazy_madd(z2[j][0], w.y, u0.x); lazy_madd(z2[j][1], w.y, u0.y); lazy_madd(z2[j][2], w.y, u0.z);
                                if constexpr (NCOMP >= 11) { lazy_madd(z3[j][0], w.y, u0.w); lazy_madd(z3[j][1], w.y, u1.x); lazy_madd(z3[j][2], w.y, u1.y); }
                            }
                            if constexpr (NCOMP >= 12) lazy_madd(zp[j], w.x, u1.z);
                        } else {
                            lazy_madd(z0[j][0], w.x, u0.x); lazy_madd(z0[j][1], w.x, u0.y); lazy_madd(z0[j][2], w.x, u0.z);
                            lazy_madd(z2[j][0], w.z, u0.x); lazy_madd(z2[j][1], w.z, u0.y); lazy_madd(z2[j][2], w.z, u0.z);
                            if constexpr (NCOMP >= 6) {
                                lazy_madd(z1[j][0], w.y, u0.x); lazy_madd(z1[j][1], w.y, u0.y); lazy_madd(z1[j][2], w.y, u0.z);
                                if constexpr (NCOMP >= 11) { lazy_madd(z3[j][0], w.w, u0.x); lazy_madd(z3[j][1], w.w, u0.y); lazy_madd(z3[j][2], w.w, u0.z); }
                            }
                            if constexpr (NCOMP >= 12) lazy_madd(zp[j], w.x, u0.w);
                        }
                    }
                };
                if (bz + P <= M) {
                    // the support does not wrap in z: the plane offsets follow from bz (no
                    // offset-table read per plane)
                    const size_t off0 = (size_t)bz * zs;
#pragma unroll kUnr
                    for (int k = 0; k < P; ++k) plane(k, off0 + (size_t)k * zs);
                } else {
#pragma unroll kUnr
                    for (int k = 0; k < P; ++k) plane(k, (size_t)Zi[k] * zs);
                }
                // double-floats: normalise the column sums once, after the z-loop
#pragma unroll
                for (int j = 0; j < NCL; ++j) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        lazy_finish(z0[j][q]);
                        lazy_finish(z1[j][q]);
                        lazy_finish(z2[j][q]);
                        lazy_finish(z3[j][q]);
                    }
                    lazy_finish(zp[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < NCL; ++j) {
                const int cx = cxa[j], cy = cya[j];
                const T gxy = acta[j] ? wx[cx] * wy[cy] : (T)0;
                // sheared cell: the physical direction of the window gradient (sx, sy - gamma sx, sz)
                const T sx = sx0 + cx, sy = sy0 + cy - (CO == 8 ? (T)p.gamma * (sx0 + cx) : (T)0);
                T col[NA];
                if constexpr (CO == 8) {
                    // U = sum g (v + a^2/6 v''); Omega ~ sum g s x v; E ~ sum g sym(s (x) (v + a^2/10 v''))
                    col[0] = gxy * (z0[j][0] + c6 * z1[j][0]);
                    col[1] = gxy * (z0[j][1] + c6 * z1[j][1]);
                    col[2] = gxy * (z0[j][2] + c6 * z1[j][2]);
                    col[3] = gxy * (sy * z0[j][2] - z2[j][1]);
                    col[4] = gxy * (z2[j][0] - sx * z0[j][2]);
                    col[5] = gxy * (sx * z0[j][1] - sy * z0[j][0]);
                    const T Q0 = z0[j][0] + c10 * z1[j][0], Q1 = z0[j][1] + c10 * z1[j][1], Q2 = z0[j][2] + c10 * z1[j][2];
                    const T R0 = z2[j][0] + c10 * z3[j][0], R1 = z2[j][1] + c10 * z3[j][1], R2 = z2[j][2] + c10 * z3[j][2];
                    col[6] = gxy * sx * Q0;
                    col[7] = gxy * sy * Q1;
                    col[8] = gxy * R2;
                    col[9] = gxy * (sx * Q1 + sy * Q0);
                    col[10] = gxy * (sx * Q2 + R0);
                    col[11] = gxy * (sy * Q2 + R1);
                } else {
                    // z0 = sum g v, z1 = sum g s_z v, z2 = sum g s_z^2 v, z3 = sum g s_z^3 v
                    const T sxy2 = sx * sx + sy * sy;
                    const T a0 = A0 + A1 * sxy2, b0 = B0 + B1 * sxy2;
                    col[0] = gxy * (a0 * z0[j][0] + A1 * z2[j][0]);
                    col[1] = gxy * (a0 * z0[j][1] + A1 * z2[j][1]);
                    col[2] = gxy * (a0 * z0[j][2] + A1 * z2[j][2]);
                    col[3] = gxy * (sy * z0[j][2] - z1[j][1]);
                    col[4] = gxy * (z1[j][0] - sx * z0[j][2]);
                    col[5] = gxy * (sx * z0[j][1] - sy * z0[j][0]);
                    const T Q0 = b0 * z0[j][0] + B1 * z2[j][0], Q1 = b0 * z0[j][1] + B1 * z2[j][1], Q2 = b0 * z0[j][2] + B1 * z2[j][2];
                    const T R0 = b0 * z1[j][0] + B1 * z3[j][0], R1 = b0 * z1[j][1] + B1 * z3[j][1], R2 = b0 * z1[j][2] + B1 * z3[j][2];
                    col[6] = gxy * sx * Q0;
                    col[7] = gxy * sy * Q1;
                    col[8] = gxy * R2;
                    col[9] = gxy * (sx * Q1 + sy * Q0);
                    col[10] = gxy * (sx * Q2 + R0);
                    col[11] = gxy * (sy * Q2 + R1);
                }
                col[12] = gxy * zp[j];
#pragma unroll
                for (int cc = 0; cc < NA; ++cc) kahan_add(acc[cc], cmp[cc], col[cc]);
            }
        }
#pragma unroll
        for (int cc = 0; cc < NA; ++cc) {
            T v = acc[cc] - cmp[cc];
            for (int off = 16; off > 0; off >>= 1) v += shfl_xor(0xffffffffu, v, off);
            acc[cc] = v;
        }
    }
    if (lane != 0) return;
    combine_write<T, TO, CO>(p, acc, i, selfc, perm, xs, yreal, y, ncomp_out, with_self);
}

#ifndef SE_GATHER_WPB
#define SE_GATHER_WPB 8
#endif
// warps per CTA of gather_kernel: 8 (two CTAs per SM) in FP32 and FP64; 16 (one CTA per SM,
// 16 particles in bin order sharing an L1) for double-floats, whose longer arithmetic per
// grid point leaves the L1 reuse to decide (measured: FP32 3.15 vs 3.22 ms, double-float
// 28.6 vs 27.4 ms at N = 2e5, P = 24)
template <typename T> constexpr int gather_wpb() { return std::is_same<T, ff>::value ? 16 : SE_GATHER_WPB; }
template <typename T, typename TO, int CO, int NCOMP, int NCL = 1, int WPB = gather_wpb<T>()>
__global__ void __launch_bounds__(32 * WPB, SE_GATHER_MINB * SE_GATHER_WPB / WPB) gather_kernel(SeParams p, int N, const int *order, const int *base,
                                                     const T *s0g, const T *wg, const double *rad, const T *selfc,
                                                     const int *perm, const T *grid, const T *xs, const T *yreal,
                                                     TO *y, int ncomp_out, int with_wave, int with_self)
{
    __shared__ typename V4<T>::t Wz[WPB][32];
    __shared__ int Zi[WPB][32];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    // particles in spreading-bin order (supports starting in the same 8^3 tile are
    // taken by neighbouring warps, so their grid reads share L1 lines)
    gather_body<T, TO, CO, NCOMP, NCL>(blockIdx.x * (blockDim.x >> 5) + wl, lane, Wz[wl], Zi[wl], p, N, order, base, s0g,
                                  wg, rad, selfc, perm, grid, xs, yreal, y, ncomp_out, with_wave, with_self);
}

// The FP32 gather (4 components, NCL columns per lane) with the real-space pair sum of its
// particle in front of it: the warp first sums its target's stored pairs
// (real_table_body_fused) into yreal, then gathers and combines.  In a launch of its own the
// pair-table stream runs at the HBM bound while the gather's short dependent z-loops wait on
// latency; in one kernel the table loads of some warps fill the memory pipe while others
// gather.  yreal is written and read back by the warp's lane 0, so no other thread's order
// matters.
template <typename TO, bool MONO, int NCL>
__global__ void __launch_bounds__(32 * SE_GATHER_WPB, SE_GATHER_MINB) gather_real_kernel(
    SeParams p, int N, const int *order, const int *base, const float *s0g, const float *wg, const double *rad,
    const float *selfc, const int *perm, const float *grid, const float *xs, float *yreal, TO *y, int ncomp_out,
    int with_wave, int with_self, const int *pair_off, size_t np, const int *pj, const float *px, const float *pc)
{
    __shared__ float4 Wz[SE_GATHER_WPB][32];
    __shared__ int Zi[SE_GATHER_WPB][32];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int w = blockIdx.x * SE_GATHER_WPB + wl;
    if (w < N) real_table_body_fused<MONO>(order[w], lane, N, pair_off, np, pj, px, pc, xs, yreal);
    gather_body<float, TO, 4, 12, NCL>(w, lane, Wz[wl], Zi[wl], p, N, order, base, s0g, wg, rad, selfc, perm, grid, xs,
                                     yreal, y, ncomp_out, with_wave, with_self);
}

// ---------------------------------------------------------------- staged gather
//
// The particles whose support starts in one kTile^3 tile (a spreading bin) share a
// window of U = kTile + P - 1 grid points per dimension.  A CTA takes one bin and
// stages the window in shared memory Z planes at a time (16-byte asynchronous copies,
// periodic wrap per point); every support row (y, z) of every particle of the bin is
// summed along x against the particle's table W_x = g_x (1, s_x, s_x^2, s_x^3): 13 FMAs
// per grid point, operands from shared memory.  The row moments become the 13 wave
// sums with the (y, z) polynomial weights (the transpose of the column form above).
// Rows of a slab are dealt to the warps in contiguous ranges of 32-row chunks; a warp
// reduces its row sums per particle into its own shared slot (Kahan-compensated) and
// the slots are added in warp order at the end, so the result does not depend on
// scheduling.
template <typename T>
struct StagedLayout {
    static constexpr int W = 8, NA = 13;
    int U, Z, G;
    __host__ __device__ size_t slab_bytes(int CO) const { return (size_t)Z * U * U * CO * sizeof(T); }
    __host__ __device__ size_t wx_off(int CO) const { return slab_bytes(CO); }
    __host__ __device__ size_t wyz_off(int CO, int P) const { return wx_off(CO) + (size_t)G * P * 4 * sizeof(T); }
    __host__ __device__ size_t slot_off(int CO, int P) const { return wyz_off(CO, P) + (size_t)G * 2 * P * sizeof(T); }
    __host__ __device__ size_t pf_off(int CO, int P) const { return slot_off(CO, P) + 2 * (size_t)W * G * NA * sizeof(T); }
    __host__ __device__ size_t pinf_off(int CO, int P) const { return pf_off(CO, P) + (size_t)G * 2 * sizeof(T); }
    __host__ __device__ size_t bytes(int CO, int P) const { return pinf_off(CO, P) + (size_t)(5 * G + 1) * sizeof(int); }
};

template <typename T, typename TO, int CO, int NCOMP>
__global__ void __launch_bounds__(256, 2) gather_staged_kernel(SeParams p, StagedLayout<T> lay, const int *tile_start,
                                                            const int *tile_perm, const int *base, const T *s0g,
                                                            const T *wg, const double *rad, const T *selfc,
                                                            const int *perm, const T *grid, const T *xs,
                                                            const T *yreal, TO *y, int ncomp_out, int with_self)
{
    constexpr int NA = 13, W = StagedLayout<T>::W, NV = CO / 4, CPP = CO * (int)sizeof(T) / 16;
    using T4 = typename V4<T>::t;
    const int P = p.P, M = p.M, nt = p.ntile, U = lay.U, Z = lay.Z, G = lay.G;
    const int bin = blockIdx.x;
    const int b0 = tile_start[bin], nb = tile_start[bin + 1] - b0;
    if (nb == 0) return;
    const int tx0 = (bin % nt) * kTile, ty0 = ((bin / nt) % nt) * kTile, tz0 = (bin / (nt * nt)) * kTile;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

    extern __shared__ __align__(32) unsigned char smstage[];
    T4 *slab = reinterpret_cast<T4 *>(smstage);                       // [Z][U][U][NV]
    T4 *Wx = reinterpret_cast<T4 *>(smstage + lay.wx_off(CO));        // [G][P]
    T *wyz = reinterpret_cast<T *>(smstage + lay.wyz_off(CO, P));     // [G][2][P]: g_y, g_z
    T *slot = reinterpret_cast<T *>(smstage + lay.slot_off(CO, P));   // [W][G][NA] sums, then compensations
    T *scomp = slot + (size_t)W * G * NA;
    T *pf = reinterpret_cast<T *>(smstage + lay.pf_off(CO, P));       // [G][2]: s_y0, s_z0
    int *pinf = reinterpret_cast<int *>(smstage + lay.pinf_off(CO, P));  // [G][4]: ox, oy, oz, i
    int *cpre = pinf + 4 * G;                                        // [G + 1] chunk prefix of a slab

    const T alpha = (T)p.alpha, kap = (T)p.kappa;

    for (int g0 = 0; g0 < nb; g0 += G) {
        const int ng = min(G, nb - g0);
        __syncthreads();
        for (int e = threadIdx.x; e < ng * P; e += blockDim.x) {
            const int q = e / P, t = e - q * P;
            const int i = tile_perm[b0 + g0 + q];
            const T *w = wg + (size_t)i * 3 * P;
            const T sx = s0g[3 * i] + (T)t, g = w[t];
            Wx[q * P + t] = T4{g, g * sx, g * sx * sx, g * sx * sx * sx};
            wyz[(2 * q) * P + t] = w[P + t];
            wyz[(2 * q + 1) * P + t] = w[2 * P + t];
        }
        for (int q = threadIdx.x; q < ng; q += blockDim.x) {
            const int i = tile_perm[b0 + g0 + q];
            pinf[4 * q] = base[3 * i] - tx0;
            pinf[4 * q + 1] = base[3 * i + 1] - ty0;
            pinf[4 * q + 2] = base[3 * i + 2] - tz0;
            pinf[4 * q + 3] = i;
            pf[2 * q] = s0g[3 * i + 1];
            pf[2 * q + 1] = s0g[3 * i + 2];
        }
        for (int e = threadIdx.x; e < 2 * W * G * NA; e += blockDim.x) slot[e] = 0;

        for (int zs = 0; zs < U; zs += Z) {
            const int nzs = min(Z, U - zs);
            __syncthreads();                       // tables staged, previous slab consumed
            // one warp per window row (uy, uz): lanes copy its points, wrapping in x
            for (int r = wid; r < nzs * U; r += W) {
                const int uy = r % U, uz = r / U;
                const T *rowp = grid + ((size_t)wrapi(tz0 + zs + uz, M) * M + wrapi(ty0 + uy, M)) * M * CO;
                for (int e = lane; e < U * CPP; e += 32) {
                    const int ux = e / CPP, h = e - ux * CPP;
                    cp_async16(smstage + ((size_t)r * U * CPP + e) * 16,
                               rowp + (size_t)wrapi(tx0 + ux, M) * CO + h * (16 / sizeof(T)));
                }
            }
            if (threadIdx.x == 0) {
                int acc = 0;
                for (int q = 0; q < ng; ++q) {
                    const int oz = pinf[4 * q + 2];
                    const int lo = max(oz, zs), hi = min(oz + P, zs + nzs);
                    cpre[q] = acc;
                    acc += hi > lo ? ((hi - lo) * P + 31) >> 5 : 0;
                }
                cpre[ng] = acc;
            }
            cp_async_wait_all();
            __syncthreads();
            const int nch = cpre[ng];
            const int c_lo = (int)((long long)nch * wid / W), c_hi = (int)((long long)nch * (wid + 1) / W);
            T o[NA];
#pragma unroll
            for (int c = 0; c < NA; ++c) o[c] = 0;
            int cur = -1, q = 0;
            auto flush = [&](int qq) {
#pragma unroll
                for (int c = 0; c < NA; ++c)
                    for (int off = 16; off > 0; off >>= 1) o[c] += __shfl_xor_sync(0xffffffffu, o[c], off);
                // lane c keeps component c: a Kahan step into this warp's slot
                T v = 0;
#pragma unroll
                for (int c = 0; c < NA; ++c)
                    if (lane == c) v = o[c];
                if (lane < NA) {
                    T *sm = slot + ((size_t)wid * G + qq) * NA + lane, *cm = scomp + ((size_t)wid * G + qq) * NA + lane;
                    T s = *sm, cc = *cm;
                    kahan_add(s, cc, v);
                    *sm = s;
                    *cm = cc;
                }
#pragma unroll
                for (int c = 0; c < NA; ++c) o[c] = 0;
            };
            for (int ci = c_lo; ci < c_hi; ++ci) {
                while (cpre[q + 1] <= ci) ++q;
                if (q != cur) {
                    if (cur >= 0) flush(cur);
                    cur = q;
                }
                const int ox = pinf[4 * q], oy = pinf[4 * q + 1], oz = pinf[4 * q + 2];
                const int lo = max(oz, zs), hi = min(oz + P, zs + nzs);
                const int j = (ci - cpre[q]) * 32 + lane;
                if (j >= (hi - lo) * P) continue;
                const int yr = j % P, zr = lo - oz + j / P;
                const T4 *g = slab + ((size_t)((oz + zr - zs) * U + oy + yr) * U + ox) * NV;
                const T4 *wx = Wx + q * P;
                T x0[3] = {0, 0, 0}, x1[3] = {0, 0, 0}, x2[3] = {0, 0, 0}, x3[3] = {0, 0, 0}, xp = 0;
#pragma unroll 4
                for (int t = 0; t < P; ++t) {
                    const T4 wv = wx[t];
                    const T4 u0 = g[t * NV];
                    if constexpr (CO == 8) {
                        const T4 u1 = g[t * NV + 1];
                        // x0 = sum g v, x1 = sum g v'', x2 = sum g s_x v, x3 = sum g s_x v''
                        x0[0] += wv.x * u0.x; x0[1] += wv.x * u0.y; x0[2] += wv.x * u0.z;
                        x1[0] += wv.x * u0.w; x1[1] += wv.x * u1.x; x1[2] += wv.x * u1.y;
                        if constexpr (NCOMP >= 6) {
                            x2[0] += wv.y * u0.x; x2[1] += wv.y * u0.y; x2[2] += wv.y * u0.z;
                            if constexpr (NCOMP >= 11) { x3[0] += wv.y * u0.w; x3[1] += wv.y * u1.x; x3[2] += wv.y * u1.y; }
                        }
                        if constexpr (NCOMP >= 12) xp += wv.x * u1.z;
                    } else {
                        // x0..x3 = sum g s_x^k v, k = 0..3
                        x0[0] += wv.x * u0.x; x0[1] += wv.x * u0.y; x0[2] += wv.x * u0.z;
                        x2[0] += wv.z * u0.x; x2[1] += wv.z * u0.y; x2[2] += wv.z * u0.z;
                        if constexpr (NCOMP >= 6) {
                            x1[0] += wv.y * u0.x; x1[1] += wv.y * u0.y; x1[2] += wv.y * u0.z;
                            if constexpr (NCOMP >= 11) { x3[0] += wv.w * u0.x; x3[1] += wv.w * u0.y; x3[2] += wv.w * u0.z; }
                        }
                        if constexpr (NCOMP >= 12) xp += wv.x * u0.w;
                    }
                }
                const T gyz = wyz[(2 * q) * P + yr] * wyz[(2 * q + 1) * P + zr];
                const T sy = pf[2 * q] + (T)yr, sz = pf[2 * q + 1] + (T)zr;
                T r[NA];
                if constexpr (CO == 8) {
                    const T ad = (T)rad[pinf[4 * q + 3]];
                    const T c6 = ad * ad / 6, c10 = ad * ad / 10;
                    r[0] = x0[0] + c6 * x1[0];
                    r[1] = x0[1] + c6 * x1[1];
                    r[2] = x0[2] + c6 * x1[2];
                    r[3] = sy * x0[2] - sz * x0[1];
                    r[4] = sz * x0[0] - x2[2];
                    r[5] = x2[1] - sy * x0[0];
                    const T Q0 = x0[0] + c10 * x1[0], Q1 = x0[1] + c10 * x1[1], Q2 = x0[2] + c10 * x1[2];
                    const T R0 = x2[0] + c10 * x3[0], R1 = x2[1] + c10 * x3[1], R2 = x2[2] + c10 * x3[2];
                    r[6] = R0;
                    r[7] = sy * Q1;
                    r[8] = sz * Q2;
                    r[9] = R1 + sy * Q0;
                    r[10] = R2 + sz * Q0;
                    r[11] = sy * Q2 + sz * Q1;
                } else {
                    const T ad = (T)rad[pinf[4 * q + 3]];
                    const T a2k2 = ad * ad * kap * kap;
                    const T A0 = 1 - a2k2 * alpha, A1 = (T)(2.0 / 3.0) * a2k2 * alpha * alpha;
                    const T B0 = 2 * kap * alpha * (1 - a2k2 * alpha);
                    const T B1 = (T)0.8 * kap * a2k2 * alpha * alpha * alpha;
                    const T syz2 = sy * sy + sz * sz, a0 = A0 + A1 * syz2, b0 = B0 + B1 * syz2;
                    r[0] = a0 * x0[0] + A1 * x2[0];
                    r[1] = a0 * x0[1] + A1 * x2[1];
                    r[2] = a0 * x0[2] + A1 * x2[2];
                    r[3] = sy * x0[2] - sz * x0[1];
                    r[4] = sz * x0[0] - x1[2];
                    r[5] = x1[1] - sy * x0[0];
                    const T Q0 = b0 * x0[0] + B1 * x2[0], Q1 = b0 * x0[1] + B1 * x2[1], Q2 = b0 * x0[2] + B1 * x2[2];
                    const T R0 = b0 * x1[0] + B1 * x3[0], R1 = b0 * x1[1] + B1 * x3[1], R2 = b0 * x1[2] + B1 * x3[2];
                    r[6] = R0;
                    r[7] = sy * Q1;
                    r[8] = sz * Q2;
                    r[9] = R1 + sy * Q0;
                    r[10] = R2 + sz * Q0;
                    r[11] = sy * Q2 + sz * Q1;
                }
                r[12] = xp;
#pragma unroll
                for (int c = 0; c < NA; ++c) o[c] += gyz * r[c];
            }
            if (cur >= 0) flush(cur);
        }
        __syncthreads();
        // the W slots of a particle, added in warp order, then combined and written
        for (int qq = wid; qq < ng; qq += W) {
            T v = 0;
            if (lane < NA)
                for (int ww = 0; ww < W; ++ww) {
                    const size_t k = ((size_t)ww * G + qq) * NA + lane;
                    v += slot[k] - scomp[k];
                }
            T acc[NA];
#pragma unroll
            for (int c = 0; c < NA; ++c) acc[c] = __shfl_sync(0xffffffffu, v, c);
            if (lane == 0) {
                const int i = pinf[4 * qq + 3];
                combine_write<T, TO, CO>(p, acc, i, selfc, perm, xs, yreal, y, ncomp_out, with_self);
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- host launchers

template <typename T2>
static size_t fft_smem_bytes(int M, int nlb)
{
    return ((size_t)((M + 1) & ~1) + 2 * (size_t)nlb * (M + 2)) * sizeof(T2);
}
constexpr size_t kSmemMax = 227 * 1024;
constexpr size_t kStagedBudget = 110 * 1024;   // staged gather: two CTAs per SM
constexpr int kStagedMaxP = 0;                 // default: staged gather up to this support (measured slower at P = 14 and 24)

void make_twiddles(se_ctx *c, int prec)
{
    const int M = c->M;
    if (prec == 1) {
        std::vector<double2> h(M);
        for (int k = 0; k < M; ++k) h[k] = double2{cos(2 * kPi * k / M), -sin(2 * kPi * k / M)};
        cudaMemcpyAsync(c->b.tw[1], h.data(), M * sizeof(double2), cudaMemcpyHostToDevice, c->stream);
    } else {
        std::vector<float2> h(M);
        for (int k = 0; k < M; ++k) h[k] = float2{(float)cos(2 * kPi * k / M), (float)-sin(2 * kPi * k / M)};
        cudaMemcpyAsync(c->b.tw[0], h.data(), M * sizeof(float2), cudaMemcpyHostToDevice, c->stream);
    }
    cudaStreamSynchronize(c->stream);
}

template <typename T>
void setup_support(se_ctx *c, cudaStream_t s)
{
    SeParams p = make_params(c);
    std::vector<double> e3(2 * c->P + 1);
    for (int j = -c->P; j <= c->P; ++j) e3[j + c->P] = exp(-p.alpha * j * j);
    double *de3 = nullptr;
    cudaMalloc(&de3, e3.size() * sizeof(double));
    cudaMemcpyAsync(de3, e3.data(), e3.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    const int N = (int)c->N;
    support_kernel<T><<<(N + 127) / 128, 128, 0, s>>>(N, p, c->b.pos, de3, c->b.sup_base, (T *)c->b.sup_s0[pix<T>()],
                                                       (T *)c->b.sup_w[pix<T>()]);
    self_coef_kernel<T><<<(N + 127) / 128, 128, 0, s>>>(N, c->xi, c->eta, c->b.rad, (T *)c->b.self_c[pix<T>()]);
    c->launches += 2;
    cudaStreamSynchronize(s);
    cudaFree(de3);
}

// CTAs sharing a 16-plane tile (each sums every ns-th chunk of its particles into its own
// partial grid): at least two waves of CTAs on the SMs, and, where the tiles fill the last
// wave poorly (M = 144: 2916 tiles on 1184 CTA slots, 2.46 waves), as many parts as bring
// the wave efficiency to the best of 1..maxparts (+2% per extra part)
int spread16_split(int sms, int ntiles, int maxparts)
{
    const int slots = sms * SE_SPREAD16_MINB;
    int ns = std::min(maxparts, std::max(1, (2 * sms * 8 + ntiles - 1) / ntiles));
    double best = 0;
    for (int q = ns; q <= maxparts; ++q) {
        const double w = (double)ntiles * q / slots, eff = w / std::ceil(w);
        if (eff > best + 0.02) {
            best = eff;
            ns = q;
        }
    }
    return std::max(1, ns);
}

// whether spread16_kernel applies: FP32, and the nbin + 1 z-bins of a 16-plane tile
// are distinct bins of the grid
static bool use_spread16(const se_ctx *c, const SeParams &p, bool fp32)
{
    const int nbin = (p.P - 1 + kTile - 1) / kTile + 1;
    return fp32 && (c->spread == 0 || c->spread == 2) && nbin + 1 <= p.ntile;
}

static void launch_spread16(se_ctx *c, const SeParams &p, const float *xs, cudaStream_t s, int ncomp)
{
    const int nt = p.ntile, ntiles = nt * nt * ((nt + 1) / 2);
    // the one-warp 8 x 4 x 16 blocks (default) are twice as many as the two-warp tiles at twice
    // the CTAs per SM, so the wave arithmetic of the split is the same
    const int ns = spread16_split(c->sms, ntiles, std::min(c->nsplit[0], c->split_cap));
    float *out = ns > 1 ? (float *)c->b.grid_part[0] : (float *)c->b.grid_f[0];
    if (c->spread == 0) {
        auto argw = [&](auto kern) {
            kern<<<dim3(2 * ntiles, ns), 32, 0, s>>>(p, c->b.tile_start, c->b.tile_perm, c->b.sup_base,
                                                      (const float *)c->b.sup_s0[0], (const float *)c->b.sup_w[0],
                                                      c->b.rad, xs, out, ns);
        };
        if (ns > 1) {
            if (ncomp <= 3) argw(spread16w_kernel<3, true>);
            else if (ncomp <= 6) argw(spread16w_kernel<6, true>);
            else if (ncomp <= 11) argw(spread16w_kernel<11, true>);
            else argw(spread16w_kernel<12, true>);
        } else {
            if (ncomp <= 3) argw(spread16w_kernel<3, false>);
            else if (ncomp <= 6) argw(spread16w_kernel<6, false>);
            else if (ncomp <= 11) argw(spread16w_kernel<11, false>);
            else argw(spread16w_kernel<12, false>);
        }
        c->launches++;
        if (ns > 1) {
            const size_t n4 = (size_t)p.M * p.M * p.M;
            sum_parts_kernel<float><<<(unsigned)((n4 + 255) / 256), 256, 0, s>>>(n4, ns, out, (float *)c->b.grid_f[0]);
            c->launches++;
        }
        return;
    }
    auto args = [&](auto kern) {
        kern<<<dim3(ntiles, ns), 64, 0, s>>>(p, c->b.tile_start, c->b.tile_perm, c->b.sup_base,
                                              (const float *)c->b.sup_s0[0], (const float *)c->b.sup_w[0], c->b.rad,
                                              xs, out, ns);
    };
    if (ns > 1) {
        if (ncomp <= 3) args(spread16_kernel<3, true>);
        else if (ncomp <= 6) args(spread16_kernel<6, true>);
        else if (ncomp <= 11) args(spread16_kernel<11, true>);
        else args(spread16_kernel<12, true>);
    } else {
        if (ncomp <= 3) args(spread16_kernel<3, false>);
        else if (ncomp <= 6) args(spread16_kernel<6, false>);
        else if (ncomp <= 11) args(spread16_kernel<11, false>);
        else args(spread16_kernel<12, false>);
    }
    c->launches++;
    if (ns > 1) {
        const size_t n4 = (size_t)p.M * p.M * p.M;
        sum_parts_kernel<float><<<(unsigned)((n4 + 255) / 256), 256, 0, s>>>(n4, ns, out, (float *)c->b.grid_f[0]);
        c->launches++;
    }
}

template <typename T>
static void launch_spread(se_ctx *c, const SeParams &p, const T *xs, cudaStream_t s, int ncomp)
{
    if constexpr (std::is_same<T, float>::value) {
        if (!p.wsrc && use_spread16(c, p, true)) {
            launch_spread16(c, p, xs, s, ncomp);
            return;
        }
    }
    // 8^3 tiles: partial grids only where the tiles alone leave SMs idle (about two waves)
    const int nt = p.ntile, ntiles = nt * nt * nt;
    const int ns = std::min(std::min(c->nsplit[pix<T>()], c->split_cap), std::max(1, (2 * c->sms * 11 + ntiles - 1) / ntiles));
    T *out = ns > 1 ? (T *)c->b.grid_part[pix<T>()] : (T *)c->b.grid_f[pix<T>()];
    auto args = [&](auto kern) {
        kern<<<dim3(ntiles, ns), 64, 0, s>>>(p, c->b.tile_start, c->b.tile_perm, c->b.sup_base,
                                              (const T *)c->b.sup_s0[pix<T>()], (const T *)c->b.sup_w[pix<T>()],
                                              c->b.rad, xs, out, ns);
    };
    auto pick = [&](auto split, auto ws) {
        constexpr bool SP = decltype(split)::value, WS = decltype(ws)::value;
        if (ncomp <= 3) args(spread_kernel<T, 3, SP, WS>);
        else if (ncomp <= 6) args(spread_kernel<T, 6, SP, WS>);
        else if (ncomp <= 11) args(spread_kernel<T, 11, SP, WS>);
        else args(spread_kernel<T, 12, SP, WS>);
    };
    using yes = std::true_type;
    using no = std::false_type;
    if (ns > 1) {
        if (p.wsrc) pick(yes{}, yes{});
        else pick(yes{}, no{});
    } else {
        if (p.wsrc) pick(no{}, yes{});
        else pick(no{}, no{});
    }
    c->launches++;
    if (ns > 1) {
        // sum over the parts in units of 4 components
        const size_t n4 = (size_t)p.M * p.M * p.M * (p.wsrc ? 2 : 1);
        sum_parts_kernel<T><<<(unsigned)((n4 + 255) / 256), 256, 0, s>>>(n4, ns, out, (T *)c->b.grid_f[pix<T>()]);
        c->launches++;
    }
}

template <typename T, int CO, int LB, int CI = 4>
static void launch_z(se_ctx *c, const SeParams &p, const typename C2<T>::t *tw, const typename C2<T>::t *sf,
                     typename C2<T>::t *so, T cnorm, cudaStream_t s)
{
    using T2 = typename C2<T>::t;
    const int M = c->M, Mh = M / 2 + 1;
    const size_t smem = fft_smem_bytes<T2>(M, CO * LB);
    // k = 2 pi q / L; net exponent -k^2/(4 xi^2) + 2 pi^2 q^2/(alpha M^2) (see the file header)
    const T twopiL = (T)(2.0 * kPi / p.L), i4x2 = (T)(0.25 / (p.xi * p.xi));
    const T ecoef = (T)(2.0 * kPi * kPi / (p.alpha * (double)M * M));
    cudaFuncSetAttribute(fft_z_scale<T, CO, LB, CI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    fft_z_scale<T, CO, LB, CI><<<dim3((Mh + LB - 1) / LB, M), kFftThreads, smem, s>>>(c->plan, tw, sf, so, cnorm,
                                                                                     twopiL, i4x2, ecoef,
                                                                                     (T)p.gamma);
}

template <typename T, int CO, int CI = 4>
static void launch_z_fit(se_ctx *c, const SeParams &p, const typename C2<T>::t *tw, const typename C2<T>::t *sf,
                         typename C2<T>::t *so, T cnorm, cudaStream_t s)
{
    using T2 = typename C2<T>::t;
    constexpr int LB0 = fft_nl<T>() / 4;
    if (fft_smem_bytes<T2>(c->M, CO * LB0) <= kSmemMax) launch_z<T, CO, LB0, CI>(c, p, tw, sf, so, cnorm, s);
    else if (fft_smem_bytes<T2>(c->M, CO * 2) <= kSmemMax) launch_z<T, CO, 2, CI>(c, p, tw, sf, so, cnorm, s);
    else launch_z<T, CO, 1, CI>(c, p, tw, sf, so, cnorm, s);
}

template <typename T, int C, bool INV>
static void launch_y(se_ctx *c, const typename C2<T>::t *tw, typename C2<T>::t *data, cudaStream_t s)
{
    using T2 = typename C2<T>::t;
    constexpr int NL = fft_nl<T>(), LB = NL / C;
    const int M = c->M, Mh = M / 2 + 1;
    const size_t smem = fft_smem_bytes<T2>(M, NL);
    cudaFuncSetAttribute(fft_y<T, C, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    fft_y<T, C, INV><<<dim3((Mh + LB - 1) / LB, M), kFftThreads, smem, s>>>(c->plan, tw, data);
}

template <typename T>
void launch_wave_spread(se_ctx *c, const T *xs, cudaStream_t s, int ncomp)
{
    const SeParams p = make_params(c);
    stage_mark(c, SE_STAGE_SPREAD, s, false);
    launch_spread<T>(c, p, xs, s, ncomp);
    stage_mark(c, SE_STAGE_SPREAD, s, true);
}

template <typename T>
void launch_wave_fft(se_ctx *c, cudaStream_t s)
{
    using T2 = typename C2<T>::t;
    constexpr int NL = fft_nl<T>();
    const SeParams p = make_params(c);
    const int M = c->M;
    const T2 *tw = (const T2 *)c->b.tw[pix<T>()];
    T2 *sf = (T2 *)c->b.spec_f[pix<T>()], *so = (T2 *)c->b.spec_o[pix<T>()];
    const int CO = p.hybrid ? 8 : 4;
    const size_t smem = fft_smem_bytes<T2>(M, NL);

    stage_mark(c, SE_STAGE_FFT_XF, s, false);
    if (p.wsrc) {
        cudaFuncSetAttribute(fft_x_fwd<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fft_x_fwd<T, 8><<<M * M / (NL / 4), kFftThreads, smem, s>>>(c->plan, tw, (const T *)c->b.grid_f[pix<T>()],
                                                                     sf);
    } else {
        cudaFuncSetAttribute(fft_x_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fft_x_fwd<T><<<M * M / (NL / 2), kFftThreads, smem, s>>>(c->plan, tw, (const T *)c->b.grid_f[pix<T>()], sf);
    }
    c->launches++;
    stage_mark(c, SE_STAGE_FFT_XF, s, true);

    stage_mark(c, SE_STAGE_FFT_YF, s, false);
    if (p.wsrc) launch_y<T, 8, false>(c, tw, sf, s);
    else launch_y<T, 4, false>(c, tw, sf, s);
    c->launches++;
    stage_mark(c, SE_STAGE_FFT_YF, s, true);

    const T cnorm = (T)(pow(p.alpha / kPi, 3.0) / (p.eta * p.L * p.L * p.L));
    stage_mark(c, SE_STAGE_FFT_Z, s, false);
    if (c->ktab_on && CO == 4) {
        constexpr int LB = fft_nl<T>() / 4;
        const int Mh = M / 2 + 1;
        const size_t zsm = fft_smem_bytes<T2>(M, 4 * LB);
        const T twopiL = (T)(2.0 * kPi / p.L), ecoef = (T)(2.0 * kPi * kPi / (p.alpha * (double)M * M));
        const T cn = (T)pow(p.alpha / kPi, 3.0);
        cudaFuncSetAttribute(fft_z_table<T, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsm);
        fft_z_table<T, LB><<<dim3((Mh + LB - 1) / LB, M), kFftThreads, zsm, s>>>(
            c->plan, tw, sf, so, (const T *)c->ktab[pix<T>()], c->ktab_n, (T)c->ktab_kmax, cn, twopiL, ecoef,
            (T)p.gamma);
    } else if (p.wsrc) launch_z_fit<T, 8, 8>(c, p, tw, sf, so, cnorm, s);
    else if (CO == 8) launch_z_fit<T, 8>(c, p, tw, sf, so, cnorm, s);
    else launch_z_fit<T, 4>(c, p, tw, sf, so, cnorm, s);
    c->launches++;
    stage_mark(c, SE_STAGE_FFT_Z, s, true);

    stage_mark(c, SE_STAGE_FFT_YI, s, false);
    if (CO == 8) launch_y<T, 8, true>(c, tw, so, s);
    else launch_y<T, 4, true>(c, tw, so, s);
    c->launches++;
    stage_mark(c, SE_STAGE_FFT_YI, s, true);

    stage_mark(c, SE_STAGE_FFT_XI, s, false);
    if (CO == 8) {
        cudaFuncSetAttribute(fft_x_inv<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fft_x_inv<T, 8><<<M * M / (NL / 4), kFftThreads, smem, s>>>(c->plan, tw, so, (T *)c->b.grid_o[pix<T>()]);
    } else {
        cudaFuncSetAttribute(fft_x_inv<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fft_x_inv<T, 4><<<M * M / (NL / 2), kFftThreads, smem, s>>>(c->plan, tw, so, (T *)c->b.grid_o[pix<T>()]);
    }
    c->launches++;
    stage_mark(c, SE_STAGE_FFT_XI, s, true);
}

// Whether the FP32 product runs the real-space sum inside the gather (gather_real_kernel):
// SE_OPT_OVERLAP 3, both parts on, the stored FP32 pair table, F T S (S_tr) moments (for F or
// F T the in-line sum reads fewer coefficient rows than the 12-component one), the
// real-space size approach (4-component gather) and no staged gather.
bool fused_real_gather(const se_ctx *c, int ncomp, int with_wave)
{
    const bool staged = c->shear == 0 && (c->gather == 2 || (c->gather == 0 && c->P <= kStagedMaxP));
    return c->overlap == 3 && (c->parts & 1) && with_wave && ncomp > 6 && c->pairs_ok[0] && c->size_mode == 1 &&
           !staged;
}

template <typename T, typename TO>
void launch_gather_combine(se_ctx *c, const T *xs, const T *yreal, TO *y, int ncomp, int with_wave,
                           cudaStream_t s)
{
    const SeParams p = make_params(c);
    const int N = (int)c->N;
    const int wpb = gather_wpb<T>();
    dim3 grid((N + wpb - 1) / wpb);
    const int with_self = (c->parts & 4) ? 1 : 0;
    auto go = [&](auto kern) {
        kern<<<grid, wpb * 32, 0, s>>>(p, N, with_wave ? c->b.tile_perm : nullptr, c->b.sup_base,
                                       (const T *)c->b.sup_s0[pix<T>()], (const T *)c->b.sup_w[pix<T>()],
                                       c->b.rad, (const T *)c->b.self_c[pix<T>()], c->b.perm,
                                       (const T *)c->b.grid_o[pix<T>()], xs, yreal, y, ncomp, with_wave, with_self);
    };
    const bool staged = !std::is_same<T, ff>::value && c->shear == 0 &&
                        (c->gather == 2 || (c->gather == 0 && c->P <= kStagedMaxP));
    if constexpr (!std::is_same<T, ff>::value) if (with_wave && staged) {
        // staged gather: one CTA per spreading bin (see gather_staged_kernel)
        const int CO = p.hybrid ? 8 : 4;
        StagedLayout<T> lay;
        lay.U = kTile + c->P - 1;
        lay.G = sizeof(T) == 4 ? 32 : 16;
        lay.Z = 1;
        lay.Z = (int)std::max<size_t>(1, std::min<size_t>(8, (kStagedBudget - (lay.bytes(CO, c->P) - lay.slab_bytes(CO))) /
                                                            ((size_t)lay.U * lay.U * CO * sizeof(T))));
        const size_t smem = lay.bytes(CO, c->P);
        const int ntiles = p.ntile * p.ntile * p.ntile;
        auto st = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kern<<<ntiles, 256, smem, s>>>(p, lay, c->b.tile_start, c->b.tile_perm, c->b.sup_base,
                                           (const T *)c->b.sup_s0[pix<T>()], (const T *)c->b.sup_w[pix<T>()], c->b.rad,
                                           (const T *)c->b.self_c[pix<T>()], c->b.perm,
                                           (const T *)c->b.grid_o[pix<T>()], xs, yreal, y, ncomp, with_self);
        };
        if (p.hybrid) {
            if (ncomp <= 3) st(gather_staged_kernel<T, TO, 8, 3>);
            else if (ncomp <= 6) st(gather_staged_kernel<T, TO, 8, 6>);
            else if (ncomp <= 11) st(gather_staged_kernel<T, TO, 8, 11>);
            else st(gather_staged_kernel<T, TO, 8, 12>);
        } else {
            if (ncomp <= 3) st(gather_staged_kernel<T, TO, 4, 3>);
            else if (ncomp <= 6) st(gather_staged_kernel<T, TO, 4, 6>);
            else if (ncomp <= 11) st(gather_staged_kernel<T, TO, 4, 11>);
            else st(gather_staged_kernel<T, TO, 4, 12>);
        }
        c->launches++;
        return;
    }
    if (p.hybrid) {
        if (ncomp <= 3) go(gather_kernel<T, TO, 8, 3>);
        else if (ncomp <= 6) go(gather_kernel<T, TO, 8, 6>);
        else if (ncomp <= 11) go(gather_kernel<T, TO, 8, 11>);
        else go(gather_kernel<T, TO, 8, 12>);
    } else {
        // FP32: two support columns per lane where few column slots of the last 64-column
        // chunk stay idle
        // (ncomp 6 and 11 take the 12-component kernel, which writes only the caller's
        // components: measured at N = 2e5, P = 24 it runs 3.04 ms against 3.24 and 3.84 ms
        // for the 6- and 11-component instantiations, whose compiled z-loops schedule worse)
        if constexpr (std::is_same<T, float>::value) {
            if (fused_real_gather(c, ncomp, with_wave)) {
                // the gather's columns per lane as for the unfused kernel below
                const bool ncl2 = SE_GATHER_NCL == 2 && ((c->P * c->P) % 64 == 0 || (c->P * c->P) % 64 > 32);
                auto fr = [&](auto kern) {
                    kern<<<grid, wpb * 32, 0, s>>>(p, N, c->b.tile_perm, c->b.sup_base, (const T *)c->b.sup_s0[0],
                                                   (const T *)c->b.sup_w[0], c->b.rad, (const T *)c->b.self_c[0],
                                                   c->b.perm, (const T *)c->b.grid_o[0], xs, const_cast<T *>(yreal),
                                                   y, ncomp, with_wave, with_self, c->b.pair_off, c->npairs,
                                                   c->b.pair_j,
                                                   (const T *)c->b.pair_x[0], (const T *)c->b.pair_c[0]);
                };
                if (ncl2) {
                    if (c->pair_mono[0]) fr(gather_real_kernel<TO, true, 2>);
                    else fr(gather_real_kernel<TO, false, 2>);
                } else {
                    if (c->pair_mono[0]) fr(gather_real_kernel<TO, true, 1>);
                    else fr(gather_real_kernel<TO, false, 1>);
                }
                c->launches++;
                return;
            }
        }
        if constexpr (std::is_same<T, float>::value && SE_GATHER_NCL == 2) {
            if ((c->P * c->P) % 64 == 0 || (c->P * c->P) % 64 > 32) {
                if (ncomp <= 3) go(gather_kernel<T, TO, 4, 3, 2>);
                else go(gather_kernel<T, TO, 4, 12, 2>);
                c->launches++;
                return;
            }
        }
        if (ncomp <= 3) go(gather_kernel<T, TO, 4, 3>);
        else if (ncomp <= 6) go(gather_kernel<T, TO, 4, 6>);
        else if (ncomp <= 11) go(gather_kernel<T, TO, 4, 11>);
        else go(gather_kernel<T, TO, 4, 12>);
    }
    c->launches++;
}

template void setup_support<float>(se_ctx *, cudaStream_t);
template void setup_support<double>(se_ctx *, cudaStream_t);
template void launch_wave_spread<float>(se_ctx *, const float *, cudaStream_t, int);
template void launch_wave_spread<double>(se_ctx *, const double *, cudaStream_t, int);
template void launch_wave_fft<float>(se_ctx *, cudaStream_t);
template void launch_wave_fft<double>(se_ctx *, cudaStream_t);
template void launch_gather_combine<float, float>(se_ctx *, const float *, const float *, float *, int, int, cudaStream_t);
template void launch_gather_combine<float, double>(se_ctx *, const float *, const float *, double *, int, int, cudaStream_t);
template void launch_gather_combine<double, float>(se_ctx *, const double *, const double *, float *, int, int, cudaStream_t);
template void launch_gather_combine<double, double>(se_ctx *, const double *, const double *, double *, int, int, cudaStream_t);
template void launch_wave_spread<ff>(se_ctx *, const ff *, cudaStream_t, int);
template void launch_gather_combine<ff, float>(se_ctx *, const ff *, const ff *, float *, int, int, cudaStream_t);
template void launch_gather_combine<ff, double>(se_ctx *, const ff *, const ff *, double *, int, int, cudaStream_t);

}  // namespace se

#include "se_wave_ws.cuh"

// ---------------------------------------------------------------- persistent batched product
//
// The products of a batch of independent boxes (own N, M, P, xi, rc each) in ONE
// cooperative launch of 2 CTAs per SM.  Each box runs eight phases in order:
//   0 inputs into cell order   1 real-space pair sum and spreading (4 tiles per CTA,
//   64 threads each)   2 x pass   3 y pass   4 z pass with the k-space scaling
//   5 inverse y pass   6 inverse x pass   7 gather + combine,
// each a list of work items.  There is no grid-wide barrier: every box keeps, per
// phase, a counter of claimed and a counter of finished items, and a CTA takes an
// item of any box whose earlier phases have finished (a warp scans the boxes, the
// latest phase first, then the box with the most work), so one box's latency-bound FFT
// passes run beside other boxes' spreading and gather.  A CTA never holds an item while
// it waits, so the launch cannot deadlock.  The stage code is that of the per-box
// kernels (the *_body functions).  Every wait is bounded in time (globaltimer): past the
// limit the CTA raises the launch's abort flag and the sticky failure flag that the
// host reads (se_batch_status), and every CTA returns.
#include "se_real_table.cuh"

namespace se {

namespace {

constexpr int kPersistPhases = 8;
constexpr int kPersistThreads = 256;
// The real-space, FFT and gather items each take kSubItems of the per-box kernels' CTA
// tasks in turn, so a claim (an atomic round trip) and a completion count are paid once
// per few tasks: small boxes have many short tasks.
constexpr int kSubItems = 16;
// Shared memory of one 64-thread group spreading 8^3 tiles (the 16-plane tiles are spread by
// the CTA's eight warps, each with a Spread16wSmem).
constexpr size_t kGroupSmem = sizeof(Spread8Smem<float>);

struct BoxDesc {
    SeParams p;
    FftPlan plan;
    int N, co, s16, with_wave, with_real, with_self;
    int nreal_items;                  // real-space sub-items (8 targets each), also the gather's
    int nreal_groups;                 // phase-1 items of the real-space sum (kSubItems sub-items each)
    int nsub[kPersistPhases];         // sub-items of the FFT phases 2..6
    int prio;                         // 0..1023, larger for boxes with more work
    float cnorm, twopiL, i4x2, ecoef;
    const void *x;
    void *y;
    float *xs, *yreal;
    const int *perm, *tile_start, *tile_perm, *sup_base;
    const float *sup_s0, *sup_w, *selfc;
    const double *rad;
    float *grid_f, *grid_o;
    float2 *spec_f, *spec_o;
    const float2 *tw;
    const int *pair_off, *pair_j;
    const float *pair_x, *pair_c;
    size_t npairs;
    int pair_mono;                    // the FP32 table stores the 13 monodisperse coefficients
};

// ctl: [0] abort flag, then per box kBoxWords words (claimed items of each phase,
// finished items of each phase), then the sticky failure flag (not reset per launch)
constexpr int kCtlAbort = 0, kCtlHdr = 4, kBoxWords = 2 * kPersistPhases;
inline int ctl_words(int nbox) { return kCtlHdr + nbox * kBoxWords + 1; }

__device__ __forceinline__ unsigned ld_acquire(const unsigned *a)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void bar_named(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Warp 0 of a CTA claims the next item: returns the box (>= 0) with *ph and *it set,
// -1 when every item of every box has been claimed, -2 when the launch is aborted.
// A CTA keeps taking items of the (box, phase) it took last while that phase has
// unclaimed items (one atomic per item); only then does the warp scan the boxes.  A
// phase may start once the latest earlier phase with items has finished (that phase's
// items all started after the phases before it had finished).  stall_box >= 0 is a
// test hook: that box's phase 1 never counts as finished, so waits for it run out.
__device__ int claim_item(const BoxDesc *__restrict__ bd, int nbox, const int *__restrict__ cnt, unsigned *ctl,
                          long long wait_ns, int stall_box, int last_box, int last_ph, int *ph_out, int *it_out)
{
    const int lane = threadIdx.x & 31;
    if (last_box >= 0) {
        int got = -1;
        if (lane == 0) {
            const unsigned old = atomicAdd(ctl + kCtlHdr + last_box * kBoxWords + last_ph, 1u);
            got = (int)old < cnt[last_box * kPersistPhases + last_ph] ? (int)old : -1;
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got >= 0) {
            *ph_out = last_ph;
            *it_out = got;
            return last_box;
        }
    }
    long long t_wait = -1;
    for (;;) {
        if (ld_acquire(ctl + kCtlAbort)) return -2;
        unsigned best = 0;          // (phase + 1) << 26 | prio << 16 | box
        bool left = false;
        for (int b = lane; b < nbox; b += 32) {
            const unsigned *bw = ctl + kCtlHdr + b * kBoxWords;
            const int *cb = cnt + b * kPersistPhases;
            // the box's claimed and finished counters in four 16-byte loads
            unsigned w[kBoxWords];
#pragma unroll
            for (int v = 0; v < kBoxWords / 4; ++v)
                asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(w[4 * v]), "=r"(w[4 * v + 1]), "=r"(w[4 * v + 2]), "=r"(w[4 * v + 3])
                             : "l"(bw + 4 * v)
                             : "memory");
            int cur = 0;
            while (cur < kPersistPhases && (int)w[cur] >= cb[cur]) ++cur;
            if (cur >= kPersistPhases) continue;
            left = true;
            int q = cur - 1;
            while (q >= 0 && cb[q] == 0) --q;
            const bool ready = q < 0 || (int)w[kPersistPhases + q] >= cb[q] + (b == stall_box && q == 1 ? 1 : 0);
            if (ready) {
                const unsigned key = ((unsigned)(cur + 1) << 26) | ((unsigned)bd[b].prio << 16) | (unsigned)b;
                best = key > best ? key : best;
            }
        }
        // the finished counts were read relaxed: a lane that saw a finished phase fences
        // (acquire side of the producers' fence + atomic), and the CTA barrier after the
        // claim orders that before every thread's reads of the item's inputs
        if (best != 0) __threadfence();
        const unsigned top = __reduce_max_sync(0xffffffffu, best);
        const bool any_left = __any_sync(0xffffffffu, left);
        if (!any_left) return -1;
        if (top != 0) {
            const int b = (int)(top & 0xffffu), ph = (int)(top >> 26) - 1;
            int got = -1;
            if (lane == 0) {
                const unsigned old = atomicAdd(ctl + kCtlHdr + b * kBoxWords + ph, 1u);
                got = (int)old < cnt[b * kPersistPhases + ph] ? (int)old : -1;
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            if (got >= 0) {
                *ph_out = ph;
                *it_out = got;
                return b;
            }
            continue;               // another CTA took the last item of that phase
        }
        // nothing ready yet: every remaining item waits for items in flight elsewhere
        const long long now = global_ns();
        if (t_wait < 0) t_wait = now;
        if (now - t_wait > wait_ns) {
            if (lane == 0) {
                atomicExch(ctl + kCtlAbort, 1u);
                atomicExch(ctl + kCtlHdr + nbox * kBoxWords, 1u);
            }
            __syncwarp();
            return -2;
        }
        __nanosleep(256);
    }
}

template <int NCOMP, typename TO>
__global__ void __launch_bounds__(kPersistThreads, 2) batch_persistent_kernel(const BoxDesc *__restrict__ bd, int nbox,
                                                                              const int *__restrict__ cnt,
                                                                              unsigned *ctl, long long wait_ns,
                                                                              int stall_box)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_box, s_ph, s_it;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int last_box = -1, last_ph = 0;
    for (;;) {
        __syncthreads();                          // the previous item's shared buffers are free
        if (warp == 0) {
            int ph = 0, it = 0;
            const int b = claim_item(bd, nbox, cnt, ctl, wait_ns, stall_box, last_box, last_ph, &ph, &it);
            if (lane == 0) {
                s_box = b;
                s_ph = ph;
                s_it = it;
            }
        }
        __syncthreads();
        const int box = s_box, ph = s_ph, it = s_it;
        if (box < 0) return;
        last_box = box;
        last_ph = ph;
        {
            const BoxDesc &d = bd[box];
            const int Mh = d.p.M / 2 + 1;
            switch (ph) {
            case 0: {
                const int k = it * kPersistThreads + threadIdx.x;
                if (k < d.N) {
                    const TO *src = (const TO *)d.x + (size_t)d.perm[k] * NCOMP;
                    float *dst = d.xs + (size_t)k * kNC;
#pragma unroll
                    for (int c = 0; c < kNC; ++c) dst[c] = c < NCOMP ? (float)src[c] : 0.f;
                }
                break;
            }
            case 1:
                if (it < d.nreal_groups) {
                    for (int u = 0; u < kSubItems; ++u) {
                        const int sub = it * kSubItems + u;
                        if (sub >= d.nreal_items) break;
                        const int i = sub * (kPersistThreads / 32) + warp;
                        if (d.with_real) {
                            if (d.pair_mono)
                                real_table_body<float, NCOMP, float, true>(i, lane, d.N, d.pair_off, d.npairs,
                                                                           d.pair_j, d.pair_x, d.pair_c, d.xs, d.yreal);
                            else
                                real_table_body<float, NCOMP>(i, lane, d.N, d.pair_off, d.npairs, d.pair_j, d.pair_x,
                                                              d.pair_c, d.xs, d.yreal);
                        } else if (i < d.N && lane < kNC) {
                            d.yreal[(size_t)i * kNC + lane] = 0.f;
                        }
                    }
                } else {
                    const int grp = threadIdx.x >> 6, tid = threadIdx.x & 63;
                    const int nt = d.p.ntile;
                    const int ntiles = d.s16 ? nt * nt * ((nt + 1) / 2) : nt * nt * nt;
                    if (d.s16) {
                        // 16-plane tiles: eight one-warp 8 x 4 x 16 blocks per item (spread16w_body)
                        const int blk = (it - d.nreal_groups) * 8 + warp;
                        if (blk < 2 * ntiles) {
                            auto &smw = *reinterpret_cast<Spread16wSmem *>(smraw + (size_t)warp * sizeof(Spread16wSmem));
                            spread16w_body<NCOMP, false>(blk, 0, lane, smw, d.p, d.tile_start, d.tile_perm, d.sup_base,
                                                         d.sup_s0, d.sup_w, d.rad, d.xs, d.grid_f, 1);
                        }
                        break;
                    }
                    const int tile = (it - d.nreal_groups) * 4 + grp;
                    if (tile < ntiles) {
                        auto sync = [grp] { bar_named(1 + grp, 64); };
                        {
                            Spread8Smem<float> &sm = *reinterpret_cast<Spread8Smem<float> *>(
                                smraw + (size_t)grp * kGroupSmem);
                            spread_body<float, NCOMP, false>(tile, 0, tid, sync, sm, d.p, d.tile_start, d.tile_perm,
                                                             d.sup_base, d.sup_s0, d.sup_w, d.rad, d.xs, d.grid_f,
                                                             1);
                        }
                    }
                }
                break;
            case 7: {
                float4 *Wz = reinterpret_cast<float4 *>(smraw) + warp * 32;
                int *Zi = reinterpret_cast<int *>(smraw + (kPersistThreads / 32) * 32 * sizeof(float4)) + warp * 32;
                const int *order = d.with_wave ? d.tile_perm : nullptr;
                for (int u = 0; u < kSubItems; ++u) {
                    const int sub = it * kSubItems + u;
                    if (sub >= d.nreal_items) break;
                    __syncwarp();                 // the warp's tables are free again
                    const int w_ = sub * (kPersistThreads / 32) + warp;
                    if (d.co == 8)
                        gather_body<float, TO, 8, NCOMP>(w_, lane, Wz, Zi, d.p, d.N, order, d.sup_base, d.sup_s0,
                                                         d.sup_w, d.rad, d.selfc, d.perm, d.grid_o, d.xs, d.yreal,
                                                         (TO *)d.y, NCOMP, d.with_wave, d.with_self);
                    else
                        gather_body<float, TO, 4, NCOMP>(w_, lane, Wz, Zi, d.p, d.N, order, d.sup_base, d.sup_s0,
                                                         d.sup_w, d.rad, d.selfc, d.perm, d.grid_o, d.xs, d.yreal,
                                                         (TO *)d.y, NCOMP, d.with_wave, d.with_self);
                }
                break;
            }
            default:
                // FFT phases: kSubItems CTA tasks of the per-box pass in turn
                for (int u = 0; u < kSubItems; ++u) {
                    const int sub = it * kSubItems + u;
                    if (sub >= d.nsub[ph]) break;
                    if (u > 0) __syncthreads();   // the previous task's shared buffers are free
                    switch (ph) {
                    case 2:
                        fft_x_fwd_body<float>(sub, smraw, d.plan, d.tw, d.grid_f, d.spec_f);
                        break;
                    case 3: {
                        const int nbx = (Mh + 3) / 4;
                        fft_y_body<float, 4, false>(sub % nbx, sub / nbx, smraw, d.plan, d.tw, d.spec_f);
                        break;
                    }
                    case 4: {
                        const int nbx = (Mh + 3) / 4;
                        if (d.co == 8)
                            fft_z_scale_body<float, 8, 4>(sub % nbx, sub / nbx, smraw, d.plan, d.tw, d.spec_f,
                                                          d.spec_o, d.cnorm, d.twopiL, d.i4x2, d.ecoef);
                        else
                            fft_z_scale_body<float, 4, 4>(sub % nbx, sub / nbx, smraw, d.plan, d.tw, d.spec_f,
                                                          d.spec_o, d.cnorm, d.twopiL, d.i4x2, d.ecoef);
                        break;
                    }
                    case 5: {
                        if (d.co == 8) {
                            const int nbx = (Mh + 1) / 2;
                            fft_y_body<float, 8, true>(sub % nbx, sub / nbx, smraw, d.plan, d.tw, d.spec_o);
                        } else {
                            const int nbx = (Mh + 3) / 4;
                            fft_y_body<float, 4, true>(sub % nbx, sub / nbx, smraw, d.plan, d.tw, d.spec_o);
                        }
                        break;
                    }
                    default:
                        if (d.co == 8) fft_x_inv_body<float, 8>(sub, smraw, d.plan, d.tw, d.spec_o, d.grid_o);
                        else fft_x_inv_body<float, 4>(sub, smraw, d.plan, d.tw, d.spec_o, d.grid_o);
                        break;
                    }
                }
                break;
            }
        }
        // the item's writes are visible device-wide before it counts as finished
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(ctl + kCtlHdr + box * kBoxWords + kPersistPhases + ph, 1u);
        }
    }
}

template <int NCOMP, typename TO>
const void *persist_kernel_for() { return (const void *)batch_persistent_kernel<NCOMP, TO>; }

const void *persist_kernel(int ncomp, int dtype)
{
    if (dtype == SE_F64) {
        if (ncomp <= 3) return persist_kernel_for<3, double>();
        if (ncomp <= 6) return persist_kernel_for<6, double>();
        if (ncomp <= 11) return persist_kernel_for<11, double>();
        return persist_kernel_for<12, double>();
    }
    if (ncomp <= 3) return persist_kernel_for<3, float>();
    if (ncomp <= 6) return persist_kernel_for<6, float>();
    if (ncomp <= 11) return persist_kernel_for<11, float>();
    return persist_kernel_for<12, float>();
}

}  // namespace

void persist_free(PersistPlan &pl)
{
    if (pl.desc) cudaFree(pl.desc);
    if (pl.pref) cudaFree(pl.pref);
    if (pl.ctl) cudaFree(pl.ctl);
    pl = PersistPlan();
}

int persist_prepare(se_ctx *const *box, int nbox, int ncomp, const void *const *x, void *const *y, int dtype,
                    PersistPlan &pl, std::string &err)
{
    persist_free(pl);
    std::vector<BoxDesc> h(nbox);
    std::vector<int> cnt((size_t)kPersistPhases * nbox, 0);
    std::vector<double> work(nbox, 0.0);
    size_t smem = std::max((size_t)4 * kGroupSmem, (size_t)(kPersistThreads / 32) * sizeof(Spread16wSmem));
    for (int b = 0; b < nbox; ++b) {
        se_ctx *c = box[b];
        const int with_real = (c->parts & 1) ? 1 : 0, with_wave = (c->parts & 2) ? 1 : 0;
        if (c->precision != 0 || !c->support_ok[0] || !c->b.grid_f[0] || (with_real && !c->pairs_ok[0]) ||
            c->ktab_on || c->size_mode >= 2) {
            err = "box " + std::to_string(b) + ": the persistent batch needs FP32 products, the stored pair "
                  "table (run the batch once without it first) and the real-space or hybrid size approach";
            return SE_ERR_STATE;
        }
        const SeParams p = make_params(c);
        BoxDesc &d = h[b];
        d.p = p;
        d.plan = c->plan;
        d.N = (int)c->N;
        d.co = p.hybrid ? 8 : 4;
        d.s16 = use_spread16(c, p, true) ? 1 : 0;
        d.with_wave = with_wave;
        d.with_real = with_real;
        d.with_self = (c->parts & 4) ? 1 : 0;
        d.nreal_items = (d.N + kPersistThreads / 32 - 1) / (kPersistThreads / 32);
        d.cnorm = (float)(pow(p.alpha / kPi, 3.0) / (p.eta * p.L * p.L * p.L));
        d.twopiL = (float)(2.0 * kPi / p.L);
        d.i4x2 = (float)(0.25 / (p.xi * p.xi));
        d.ecoef = (float)(2.0 * kPi * kPi / (p.alpha * (double)p.M * p.M));
        d.x = x[b];
        d.y = y[b];
        d.xs = (float *)c->b.xs[0];
        d.yreal = (float *)c->b.yreal[0];
        d.perm = c->b.perm;
        d.tile_start = c->b.tile_start;
        d.tile_perm = c->b.tile_perm;
        d.sup_base = c->b.sup_base;
        d.sup_s0 = (const float *)c->b.sup_s0[0];
        d.sup_w = (const float *)c->b.sup_w[0];
        d.selfc = (const float *)c->b.self_c[0];
        d.rad = c->b.rad;
        d.grid_f = (float *)c->b.grid_f[0];
        d.grid_o = (float *)c->b.grid_o[0];
        d.spec_f = (float2 *)c->b.spec_f[0];
        d.spec_o = (float2 *)c->b.spec_o[0];
        d.tw = (const float2 *)c->b.tw[0];
        d.pair_off = c->b.pair_off;
        d.pair_j = c->b.pair_j;
        d.pair_x = (const float *)c->b.pair_x[0];
        d.pair_c = (const float *)c->b.pair_c[0];
        d.pair_mono = c->pair_mono[0] ? 1 : 0;
        d.npairs = c->npairs;
        const int M = p.M, Mh = M / 2 + 1, nt = p.ntile;
        const int ntiles = d.s16 ? nt * nt * ((nt + 1) / 2) : nt * nt * nt;
        const int nw = with_wave;
        // CTA tasks of the per-box kernels; FFT and real-space/gather items take kSubItems each
        const int sub[kPersistPhases] = {0, 0, nw * M * M / 8, nw * ((Mh + 3) / 4) * M, nw * ((Mh + 3) / 4) * M,
                                         nw * (d.co == 8 ? (Mh + 1) / 2 : (Mh + 3) / 4) * M,
                                         nw * M * M / (d.co == 8 ? 4 : 8), 0};
        for (int ph = 0; ph < kPersistPhases; ++ph) d.nsub[ph] = sub[ph];
        d.nreal_groups = (d.nreal_items + kSubItems - 1) / kSubItems;
        auto groups = [](int n) { return (n + kSubItems - 1) / kSubItems; };
        const int items[kPersistPhases] = {
            (d.N + kPersistThreads - 1) / kPersistThreads,
            d.nreal_groups + nw * (ntiles + 3) / 4,
            groups(sub[2]), groups(sub[3]), groups(sub[4]), groups(sub[5]), groups(sub[6]),
            d.nreal_groups};
        for (int ph = 0; ph < kPersistPhases; ++ph) cnt[(size_t)b * kPersistPhases + ph] = items[ph];
        work[b] = (double)d.N * p.P * p.P * p.P + (double)M * M * M;
        smem = std::max(smem, fft_smem_bytes<float2>(M, fft_nl<float>()));
        smem = std::max(smem, fft_smem_bytes<float2>(M, 4 * d.co));
    }
    if (smem > kSmemMax) {
        err = "a box's grid is too large for the persistent batch";
        return SE_ERR_GRID;
    }
    if (nbox > 65535) {
        err = "the persistent batch takes at most 65535 boxes";
        return SE_ERR_ARG;
    }
    // priority: rank by work, so the largest boxes start first
    {
        std::vector<int> order(nbox);
        for (int b = 0; b < nbox; ++b) order[b] = b;
        std::sort(order.begin(), order.end(), [&](int u, int v) { return work[u] > work[v]; });
        for (int r = 0; r < nbox; ++r) h[order[r]].prio = 1023 - std::min(r, 1023);
    }
    const void *kern = persist_kernel(ncomp, dtype);
    int dev = 0, nsm = 0, occ = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kPersistThreads, smem) != cudaSuccess ||
        occ < 1 || !coop) {
        cudaGetLastError();
        err = "the persistent batch kernel cannot be launched cooperatively on this device";
        return SE_ERR_CUDA;
    }
    const int nw = ctl_words(nbox);
    if (cudaMalloc(&pl.desc, nbox * sizeof(BoxDesc)) != cudaSuccess ||
        cudaMalloc(&pl.pref, cnt.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&pl.ctl, nw * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        persist_free(pl);
        err = "persistent batch allocation failed";
        return SE_ERR_NOMEM;
    }
    if (cudaMemcpy(pl.desc, h.data(), nbox * sizeof(BoxDesc), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(pl.pref, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(pl.ctl, 0, nw * sizeof(unsigned)) != cudaSuccess) {
        persist_free(pl);
        err = "persistent batch upload failed";
        return SE_ERR_CUDA;
    }
    pl.nbox = nbox;
    pl.ctl_words = nw;
    pl.ncomp = ncomp;
    pl.dtype = dtype;
    pl.grid = occ * nsm;
    pl.smem = smem;
    pl.kernel = kern;
    return SE_OK;
}

int persist_launch(const PersistPlan &pl, cudaStream_t s, std::string &err)
{
    // fresh abort flag and item counters; the sticky failure flag (the last word) stays
    cudaError_t e = cudaMemsetAsync(pl.ctl, 0, (pl.ctl_words - 1) * sizeof(unsigned), s);
    if (e == cudaSuccess) {
        const BoxDesc *bd = (const BoxDesc *)pl.desc;
        int nbox = pl.nbox;
        const int *cnt = pl.pref;
        unsigned *ctl = pl.ctl;
        long long wait_ns = pl.wait_ns;
        int stall_box = pl.stall_box;
        void *args[] = {(void *)&bd, (void *)&nbox, (void *)&cnt, (void *)&ctl, (void *)&wait_ns, (void *)&stall_box};
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.gridDim = dim3(pl.grid);
        cfg.blockDim = dim3(kPersistThreads);
        cfg.dynamicSmemBytes = pl.smem;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelExC(&cfg, pl.kernel, args);
    }
    if (e != cudaSuccess) {
        err = std::string("persistent batch launch: ") + cudaGetErrorString(e);
        return SE_ERR_CUDA;
    }
    return SE_OK;
}

int persist_failed(const PersistPlan &pl, cudaStream_t s)
{
    unsigned f = 0;
    unsigned *failed = pl.ctl + pl.ctl_words - 1;
    cudaMemcpyAsync(&f, failed, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    cudaMemsetAsync(failed, 0, sizeof(unsigned), s);
    return f ? 1 : 0;
}

}  // namespace se
