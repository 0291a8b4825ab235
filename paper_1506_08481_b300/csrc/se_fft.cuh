// Mixed-radix (2, 3, 4, 8) Stockham FFT of many lines held in shared memory.
//
// Each stage of radix R over a line of length M performs M/R butterflies
//   v_r = x[j + r M/R] * W_{Ns R}^{r (j mod Ns)},  X = DFT_R(v),
//   y[(j div Ns) Ns R + (j mod Ns) + r Ns] = X_r,
// with Ns the product of the radices already applied (the self-sorting Stockham
// ordering, so no bit reversal pass is needed).  A CTA transforms `nlines` lines
// of `lstride`-strided storage in place: every thread first loads the inputs of
// its butterflies into registers, the block synchronises, then the outputs are
// written back.  Twiddles come from a table tw[t] = exp(-2 pi i t / M).
#pragma once

#include "se_internal.cuh"

namespace se {

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b)
{
    return T2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T2>
__device__ __forceinline__ T2 cadd(T2 a, T2 b) { return T2{a.x + b.x, a.y + b.y}; }
template <typename T2>
__device__ __forceinline__ T2 csub(T2 a, T2 b) { return T2{a.x - b.x, a.y - b.y}; }
// multiply by -i (forward transform) or +i (inverse transform)
template <typename T2>
__device__ __forceinline__ T2 mul_mi(T2 a, bool inv) { return inv ? T2{-a.y, a.x} : T2{a.y, -a.x}; }

template <int R, typename T2>
__device__ __forceinline__ void dft_generic(T2 (&v)[R], bool inv)
{
    using T = decltype(v[0].x);
    if constexpr (R == 2) {
        T2 a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    } else if constexpr (R == 3) {
        const T s3 = (T)0.86602540378443864676;
        T2 t1 = cadd(v[1], v[2]);
        T2 t2 = T2{v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y};
        T2 d = csub(v[1], v[2]);
        T2 t3 = mul_mi(T2{s3 * d.x, s3 * d.y}, inv);
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    } else if constexpr (R == 4) {
        T2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        T2 t2 = cadd(v[1], v[3]), t3 = mul_mi(csub(v[1], v[3]), inv);
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    } else if constexpr (R == 8) {
        const T h = (T)0.70710678118654752440;
        T2 e[4] = {v[0], v[2], v[4], v[6]};
        T2 o[4] = {v[1], v[3], v[5], v[7]};
        dft_generic<4>(e, inv);
        dft_generic<4>(o, inv);
        // W8^k o_k, W8 = exp(-+ i pi/4)
        T2 w1 = inv ? T2{h * (o[1].x - o[1].y), h * (o[1].x + o[1].y)}
                    : T2{h * (o[1].x + o[1].y), h * (o[1].y - o[1].x)};
        T2 w2 = mul_mi(o[2], inv);
        T2 w3 = inv ? T2{-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y)}
                    : T2{h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y)};
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], w1);
        v[5] = csub(e[1], w1);
        v[2] = cadd(e[2], w2);
        v[6] = csub(e[2], w2);
        v[3] = cadd(e[3], w3);
        v[7] = csub(e[3], w3);
    }
}

// One radix-R stage over `nlines` lines (elements per thread bounded by EPT).
template <int R, int EPT, typename T2>
__device__ __forceinline__ void fft_stage(T2 *buf, int M, int nlines, int lstride, int Ns,
                                          const T2 *tw, bool inv)
{
    constexpr int K = (EPT + R - 1) / R;
    const int nbl = M / R;
    const int nb = nbl * nlines;
    const int tstep = M / (Ns * R);
    T2 v[K][R];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        int b = threadIdx.x + k * blockDim.x;
        if (b < nb) {
            int line = b / nbl, j = b - line * nbl;
            const T2 *src = buf + line * lstride + j;
#pragma unroll
            for (int r = 0; r < R; ++r) v[k][r] = src[r * nbl];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        int b = threadIdx.x + k * blockDim.x;
        if (b < nb) {
            int line = b / nbl, j = b - line * nbl;
            int kk = j % Ns;
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    T2 w = tw[r * kk * tstep];
                    if (inv) w.y = -w.y;
                    v[k][r] = cmul(v[k][r], w);
                }
            }
            dft_generic<R>(v[k], inv);
            T2 *dst = buf + line * lstride + (j - kk) * R + kk;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[r * Ns] = v[k][r];
        }
    }
    __syncthreads();
}

// Full transform of nlines lines (unnormalised; inv selects exp(+2 pi i ...)).
template <int EPT, typename T2>
__device__ void fft_lines(T2 *buf, int nlines, int lstride, const FftPlan &plan, const T2 *tw, bool inv)
{
    int Ns = 1;
    for (int s = 0; s < plan.nst; ++s) {
        const int R = plan.rad[s];
        if (R == 8) fft_stage<8, EPT>(buf, plan.M, nlines, lstride, Ns, tw, inv);
        else if (R == 4) fft_stage<4, EPT>(buf, plan.M, nlines, lstride, Ns, tw, inv);
        else if (R == 3) fft_stage<3, EPT>(buf, plan.M, nlines, lstride, Ns, tw, inv);
        else fft_stage<2, EPT>(buf, plan.M, nlines, lstride, Ns, tw, inv);
        Ns *= R;
    }
}

}  // namespace se
