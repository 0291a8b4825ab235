// Real-space pair sum from the stored pair table (see se_real.cu for the table and the
// coefficients): one warp per target, the lanes stream the target's stored pairs
// (coalesced SoA loads), contract them with the neighbours' moments and reduce over
// the warp.  Shared by the product's real-space kernel and the persistent batched
// kernel.
#pragma once

#include "se_internal.cuh"

namespace se {

// Monodisperse tables (every radius equal) store 13 of the 19 coefficients: with a_i = a_j
// the Faxen factors of source and target coincide, so c3 = c2, c9 = -c6, c10 = -c7,
// c11 = -c8, c17 = 3 c15 and c18 = -3 c16.  mono_slot(q): the stored slot of c_q, -1 for the
// derived ones.
__host__ __device__ constexpr int mono_slot(int q)
{
    return q <= 2 ? q : q == 3 ? -1 : q <= 8 ? q - 1 : q <= 11 ? -1 : q <= 16 ? q - 4 : -1;
}

// target i, lane 0..31 of its warp; the table is stored at precision TL and read into T
// (the FP64-equivalent product contracts the FP64 table in double-float arithmetic);
// MONO: the table holds the 13 stored slots of a monodisperse configuration.
template <typename T, int NCOMP, typename TL = T, bool MONO = false>
__device__ __forceinline__ void real_table_body(int i, int lane, int N, const int *off, size_t np, const int *pj,
                                                const TL *px, const TL *pc, const T *xs, T *yreal)
{
    if (i >= N) return;
    T a[13];
#pragma unroll
    for (int c = 0; c < 13; ++c) a[c] = 0;
    const int k1 = off[i + 1];
    // coefficient q of pair k (slot q, or its monodisperse slot)
    auto C = [&](int q, int k) -> T { return T(pc[(size_t)(MONO ? mono_slot(q) : q) * np + k]); };
    for (int k = off[i] + lane; k < k1; k += 32) {
        const int j = pj[k];
        const T x0 = T(px[k]), x1 = T(px[np + k]), x2 = T(px[2 * np + k]);
        const T *xj = xs + (size_t)j * kNC;
        const T F0 = xj[0], F1 = xj[1], F2 = xj[2];
        const T xF = x0 * F0 + x1 * F1 + x2 * F2;
        {
            const T aF = C(0, k), bF = C(1, k) * xF;
            a[0] += aF * F0 - bF * x0;
            a[1] += aF * F1 - bF * x1;
            a[2] += aF * F2 - bF * x2;
        }
        if constexpr (NCOMP >= 6) {
            const T T0 = xj[3], T1 = xj[4], T2 = xj[5];
            const T xT0 = x1 * T2 - x2 * T1, xT1 = x2 * T0 - x0 * T2, xT2 = x0 * T1 - x1 * T0;
            const T uT = C(2, k);
            T oF;
            if constexpr (MONO) oF = uT; else oF = C(3, k);
            a[0] += uT * xT0;
            a[1] += uT * xT1;
            a[2] += uT * xT2;
            a[3] += oF * (x1 * F2 - x2 * F1);
            a[4] += oF * (x2 * F0 - x0 * F2);
            a[5] += oF * (x0 * F1 - x1 * F0);
            const T oTa = C(4, k) * (x0 * T0 + x1 * T1 + x2 * T2), oTb = C(5, k);
            a[3] += oTa * x0 - oTb * T0;
            a[4] += oTa * x1 - oTb * T1;
            a[5] += oTa * x2 - oTb * T2;
            if constexpr (NCOMP >= 11) {
                const T r2h = (T)0.70710678118654752440, r6 = (T)0.40824829046386301637;
                const T Sxx = r2h * xj[6] - r6 * xj[7], Syy = -r2h * xj[6] - r6 * xj[7], Szz = 2 * r6 * xj[7],
                        Sxy = r2h * xj[8], Sxz = r2h * xj[9], Syz = r2h * xj[10];
                const T Sx0 = Sxx * x0 + Sxy * x1 + Sxz * x2, Sx1 = Sxy * x0 + Syy * x1 + Syz * x2,
                        Sx2 = Sxz * x0 + Syz * x1 + Szz * x2;
                const T xSx = x0 * Sx0 + x1 * Sx1 + x2 * Sx2;
                {   // U <- S
                    const T c6 = C(6, k), c7 = C(7, k);
                    const T ua = c6, ub = c7 * xSx;
                    a[0] += ua * Sx0 + ub * x0;
                    a[1] += ua * Sx1 + ub * x1;
                    a[2] += ua * Sx2 + ub * x2;
                }
                {   // Om <- S
                    const T o = C(8, k);
                    a[3] += o * (x1 * Sx2 - x2 * Sx1);
                    a[4] += o * (x2 * Sx0 - x0 * Sx2);
                    a[5] += o * (x0 * Sx1 - x1 * Sx0);
                }
                // E (symmetric tensor xx yy zz xy xz yz) <- F, T, S
                T ea, eb, et;
                if constexpr (MONO) {
                    ea = -C(6, k);
                    eb = -C(7, k) * xF;
                    et = -C(8, k);
                } else {
                    ea = C(9, k);
                    eb = C(10, k) * xF;
                    et = C(11, k);
                }
                const T sa = C(12, k), sb = C(13, k), sc = C(14, k) * xSx;
                a[6] += ea * x0 * F0 + eb * x0 * x0 + et * x0 * xT0 + sa * Sxx + sb * x0 * Sx0 + sc * x0 * x0;
                a[7] += ea * x1 * F1 + eb * x1 * x1 + et * x1 * xT1 + sa * Syy + sb * x1 * Sx1 + sc * x1 * x1;
                a[8] += ea * x2 * F2 + eb * x2 * x2 + et * x2 * xT2 + sa * Szz + sb * x2 * Sx2 + sc * x2 * x2;
                a[9] += (T)0.5 * (ea * (x0 * F1 + x1 * F0) + et * (x0 * xT1 + x1 * xT0) + sb * (x0 * Sx1 + x1 * Sx0)) +
                        eb * x0 * x1 + sa * Sxy + sc * x0 * x1;
                a[10] += (T)0.5 * (ea * (x0 * F2 + x2 * F0) + et * (x0 * xT2 + x2 * xT0) + sb * (x0 * Sx2 + x2 * Sx0)) +
                         eb * x0 * x2 + sa * Sxz + sc * x0 * x2;
                a[11] += (T)0.5 * (ea * (x1 * F2 + x2 * F1) + et * (x1 * xT2 + x2 * xT1) + sb * (x1 * Sx2 + x2 * Sx1)) +
                         eb * x1 * x2 + sa * Syz + sc * x1 * x2;
                if constexpr (NCOMP >= 12) {
                    const T Str = xj[11];
                    const T c15 = C(15, k), c16 = C(16, k);
                    const T uq = c15 * Str, eq = c16 * Str;
                    a[0] += uq * x0;
                    a[1] += uq * x1;
                    a[2] += uq * x2;
                    a[6] += eq * x0 * x0;
                    a[7] += eq * x1 * x1;
                    a[8] += eq * x2 * x2;
                    a[9] += eq * x0 * x1;
                    a[10] += eq * x0 * x2;
                    a[11] += eq * x1 * x2;
                    if constexpr (MONO) a[12] += 3 * c15 * xF - 3 * c16 * xSx;
                    else a[12] += C(17, k) * xF + C(18, k) * xSx;
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 13; ++c)
        for (int o = 16; o > 0; o >>= 1) a[c] += shfl_xor(0xffffffffu, a[c], o);
    if (lane == 0) {
        T *yo = yreal + (size_t)i * kNC;
        yo[0] = a[0];
        yo[1] = a[1];
        yo[2] = a[2];
        yo[3] = a[3];
        yo[4] = a[4];
        yo[5] = a[5];
        const T r2h = (T)0.70710678118654752440, r6 = (T)0.40824829046386301637, sq2 = (T)1.41421356237309504880;
        yo[6] = r2h * (a[6] - a[7]);
        yo[7] = r6 * (2 * a[8] - a[6] - a[7]);
        yo[8] = sq2 * a[9];
        yo[9] = sq2 * a[10];
        yo[10] = sq2 * a[11];
        yo[11] = a[12];
    }
}


// The same sum for one target inside the gather kernel (FP32, F T S S_tr): there only a few of
// the SM's warps stream the table at a time, so each lane keeps fused_pairs() pairs in flight
// (all their values loaded before any is contracted), and the table is read with streaming
// loads (evict-first) so that it does not push the gather's grid points out of L1.  Measured
// per product at N = 2e5, P = 24 (8.33 ms with the sum in a kernel of its own): plain loads, 1
// pair 8.98 ms, 2 pairs 8.69 ms; evict-first loads, 2 pairs 8.01 ms, 3 pairs 7.94 ms, 4 pairs
// 8.13 ms (the registers of four pairs spill).  A pair of the 19-coefficient table holds six
// registers more: on a bidisperse box (N = 1e5, P = 24) 3 pairs took 3.83 ms against 3.76 ms for
// 2, so that table keeps 2.  The arithmetic is that of real_table_body<float, 12, float, MONO>,
// pair by pair in the same order (a masked pair adds exact zeros), so the result is the same.
template <bool MONO> constexpr int fused_pairs() { return MONO ? 3 : 2; }
template <bool MONO>
__device__ __forceinline__ void real_table_body_fused(int i, int lane, int N, const int *off, size_t np,
                                                      const int *pj, const float *px, const float *pc,
                                                      const float *xs, float *yreal)
{
    using T = float;
    if (i >= N) return;
    constexpr int NQ = MONO ? 13 : 19;              // stored coefficient slots
    T a[13];
#pragma unroll
    for (int c = 0; c < 13; ++c) a[c] = 0;
    const int k1 = off[i + 1], k0 = off[i] + lane;
    struct PD {
        T x0, x1, x2, c[NQ], m[kNC];
    };
    // pair k's separation, stored coefficients and source moments (zero moments for ok = false,
    // which then adds nothing: every coupling is linear in the source's moments)
    auto load = [&](int k, bool ok, PD &d) {
        const int kk = ok ? k : k0;
        const int j = __ldcs(pj + kk);
        d.x0 = __ldcs(px + kk);
        d.x1 = __ldcs(px + np + kk);
        d.x2 = __ldcs(px + 2 * np + kk);
#pragma unroll
        for (int q = 0; q < NQ; ++q) d.c[q] = __ldcs(pc + (size_t)q * np + kk);
        const float4 *xj = reinterpret_cast<const float4 *>(xs + (size_t)j * kNC);
        const float4 m0 = xj[0], m1 = xj[1], m2 = xj[2];
        const T z = ok ? 1.f : 0.f;
        d.m[0] = z * m0.x; d.m[1] = z * m0.y; d.m[2] = z * m0.z; d.m[3] = z * m0.w;
        d.m[4] = z * m1.x; d.m[5] = z * m1.y; d.m[6] = z * m1.z; d.m[7] = z * m1.w;
        d.m[8] = z * m2.x; d.m[9] = z * m2.y; d.m[10] = z * m2.z; d.m[11] = z * m2.w;
    };
    // coefficient q of a loaded pair (its slot, or derived from a stored one for MONO)
    auto C = [](const PD &d, int q) -> T { return d.c[MONO ? mono_slot(q) : q]; };
    auto acc = [&](const PD &d) {
        const T x0 = d.x0, x1 = d.x1, x2 = d.x2;
        const T F0 = d.m[0], F1 = d.m[1], F2 = d.m[2];
        const T xF = x0 * F0 + x1 * F1 + x2 * F2;
        {
            const T aF = C(d, 0), bF = C(d, 1) * xF;
            a[0] += aF * F0 - bF * x0;
            a[1] += aF * F1 - bF * x1;
            a[2] += aF * F2 - bF * x2;
        }
        const T T0 = d.m[3], T1 = d.m[4], T2 = d.m[5];
        const T xT0 = x1 * T2 - x2 * T1, xT1 = x2 * T0 - x0 * T2, xT2 = x0 * T1 - x1 * T0;
        const T uT = C(d, 2);
        T oF;
        if constexpr (MONO) oF = uT; else oF = C(d, 3);
        a[0] += uT * xT0;
        a[1] += uT * xT1;
        a[2] += uT * xT2;
        a[3] += oF * (x1 * F2 - x2 * F1);
        a[4] += oF * (x2 * F0 - x0 * F2);
        a[5] += oF * (x0 * F1 - x1 * F0);
        const T oTa = C(d, 4) * (x0 * T0 + x1 * T1 + x2 * T2), oTb = C(d, 5);
        a[3] += oTa * x0 - oTb * T0;
        a[4] += oTa * x1 - oTb * T1;
        a[5] += oTa * x2 - oTb * T2;
        const T r2h = (T)0.70710678118654752440, r6 = (T)0.40824829046386301637;
        const T Sxx = r2h * d.m[6] - r6 * d.m[7], Syy = -r2h * d.m[6] - r6 * d.m[7], Szz = 2 * r6 * d.m[7],
                Sxy = r2h * d.m[8], Sxz = r2h * d.m[9], Syz = r2h * d.m[10];
        const T Sx0 = Sxx * x0 + Sxy * x1 + Sxz * x2, Sx1 = Sxy * x0 + Syy * x1 + Syz * x2,
                Sx2 = Sxz * x0 + Syz * x1 + Szz * x2;
        const T xSx = x0 * Sx0 + x1 * Sx1 + x2 * Sx2;
        {   // U <- S
            const T c6 = C(d, 6), c7 = C(d, 7);
            const T ua = c6, ub = c7 * xSx;
            a[0] += ua * Sx0 + ub * x0;
            a[1] += ua * Sx1 + ub * x1;
            a[2] += ua * Sx2 + ub * x2;
        }
        {   // Om <- S
            const T o = C(d, 8);
            a[3] += o * (x1 * Sx2 - x2 * Sx1);
            a[4] += o * (x2 * Sx0 - x0 * Sx2);
            a[5] += o * (x0 * Sx1 - x1 * Sx0);
        }
        T ea, eb, et;
        if constexpr (MONO) {
            ea = -C(d, 6);
            eb = -C(d, 7) * xF;
            et = -C(d, 8);
        } else {
            ea = C(d, 9);
            eb = C(d, 10) * xF;
            et = C(d, 11);
        }
        const T sa = C(d, 12), sb = C(d, 13), sc = C(d, 14) * xSx;
        a[6] += ea * x0 * F0 + eb * x0 * x0 + et * x0 * xT0 + sa * Sxx + sb * x0 * Sx0 + sc * x0 * x0;
        a[7] += ea * x1 * F1 + eb * x1 * x1 + et * x1 * xT1 + sa * Syy + sb * x1 * Sx1 + sc * x1 * x1;
        a[8] += ea * x2 * F2 + eb * x2 * x2 + et * x2 * xT2 + sa * Szz + sb * x2 * Sx2 + sc * x2 * x2;
        a[9] += (T)0.5 * (ea * (x0 * F1 + x1 * F0) + et * (x0 * xT1 + x1 * xT0) + sb * (x0 * Sx1 + x1 * Sx0)) +
                eb * x0 * x1 + sa * Sxy + sc * x0 * x1;
        a[10] += (T)0.5 * (ea * (x0 * F2 + x2 * F0) + et * (x0 * xT2 + x2 * xT0) + sb * (x0 * Sx2 + x2 * Sx0)) +
                 eb * x0 * x2 + sa * Sxz + sc * x0 * x2;
        a[11] += (T)0.5 * (ea * (x1 * F2 + x2 * F1) + et * (x1 * xT2 + x2 * xT1) + sb * (x1 * Sx2 + x2 * Sx1)) +
                 eb * x1 * x2 + sa * Syz + sc * x1 * x2;
        const T Str = d.m[11];
        const T c15 = C(d, 15), c16 = C(d, 16);
        const T uq = c15 * Str, eq = c16 * Str;
        a[0] += uq * x0;
        a[1] += uq * x1;
        a[2] += uq * x2;
        a[6] += eq * x0 * x0;
        a[7] += eq * x1 * x1;
        a[8] += eq * x2 * x2;
        a[9] += eq * x0 * x1;
        a[10] += eq * x0 * x2;
        a[11] += eq * x1 * x2;
        if constexpr (MONO) a[12] += 3 * c15 * xF - 3 * c16 * xSx;
        else a[12] += C(d, 17) * xF + C(d, 18) * xSx;
    };
    constexpr int U = fused_pairs<MONO>();
    for (int k = k0; k < k1; k += 32 * U) {
        PD d[U];
#pragma unroll
        for (int u = 0; u < U; ++u) load(k + 32 * u, k + 32 * u < k1, d[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) acc(d[u]);
    }
#pragma unroll
    for (int c = 0; c < 13; ++c)
        for (int o = 16; o > 0; o >>= 1) a[c] += shfl_xor(0xffffffffu, a[c], o);
    if (lane == 0) {
        T *yo = yreal + (size_t)i * kNC;
        yo[0] = a[0];
        yo[1] = a[1];
        yo[2] = a[2];
        yo[3] = a[3];
        yo[4] = a[4];
        yo[5] = a[5];
        const T r2h = (T)0.70710678118654752440, r6 = (T)0.40824829046386301637, sq2 = (T)1.41421356237309504880;
        yo[6] = r2h * (a[6] - a[7]);
        yo[7] = r6 * (2 * a[8] - a[6] - a[7]);
        yo[8] = sq2 * a[9];
        yo[9] = sq2 * a[10];
        yo[10] = sq2 * a[11];
        yo[11] = a[12];
    }
}

}  // namespace se
