// Mixed-radix (2, 3, 4, 6, 8, 9) Stockham FFT of a batch of NL lines held in shared
// memory in element-major order (element e of line l at index e * NL + l), computed
// out of place between two buffers so that a thread takes its butterflies one at a
// time (few registers, several CTAs per SM to overlap the global traffic of one CTA
// with the arithmetic of the others).
//
// A stage of radix R over lines of length M performs M/R butterflies per line:
//   v_r = x[j + r M/R] W_{Ns R}^{r (j mod Ns)},  X = DFT_R(v),
//   y[(j div Ns) Ns R + (j mod Ns) + r Ns] = X_r,
// with Ns the product of the radices already applied (the self-sorting Stockham
// ordering: no digit-reversal pass).  Twiddles come from tw[t] = exp(-2 pi i t / M);
// the inverse transform conjugates them and is unnormalised.  Consecutive threads
// take consecutive lines at one butterfly position, so with NL >= 16 (8-byte complex)
// or NL >= 8 (16-byte complex) every warp access is a contiguous run of words.
// Radices 6 and 9 are two-level Cooley-Tukey butterflies (inner radix 3).
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
// multiply by exp(-+ i theta) given c = cos(theta), s = sin(theta)
template <typename T2, typename T>
__device__ __forceinline__ T2 rot(T2 a, T c, T s, bool inv)
{
    return inv ? T2{a.x * c - a.y * s, a.y * c + a.x * s} : T2{a.x * c + a.y * s, a.y * c - a.x * s};
}

template <typename T2>
__device__ __forceinline__ void dft3(T2 &v0, T2 &v1, T2 &v2, bool inv)
{
    using T = decltype(v0.x);
    const T s3 = (T)0.86602540378443864676;
    const T2 t1 = cadd(v1, v2);
    const T2 t2 = T2{v0.x - (T)0.5 * t1.x, v0.y - (T)0.5 * t1.y};
    const T2 d = csub(v1, v2);
    const T2 t3 = mul_mi(T2{s3 * d.x, s3 * d.y}, inv);
    v0 = cadd(v0, t1);
    v1 = cadd(t2, t3);
    v2 = csub(t2, t3);
}

template <int R, typename T2>
__device__ __forceinline__ void dft_generic(T2 (&v)[R], bool inv)
{
    using T = decltype(v[0].x);
    if constexpr (R == 2) {
        const T2 a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    } else if constexpr (R == 3) {
        dft3(v[0], v[1], v[2], inv);
    } else if constexpr (R == 4) {
        const T2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        const T2 t2 = cadd(v[1], v[3]), t3 = mul_mi(csub(v[1], v[3]), inv);
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    } else if constexpr (R == 6) {
        // n = n1 + 2 n2, k = k1 + 3 k2: radix-3 over n2, twiddle W6^(n1 k1), radix-2 over n1
        dft3(v[0], v[2], v[4], inv);
        dft3(v[1], v[3], v[5], inv);
        const T h = (T)0.5, s3 = (T)0.86602540378443864676;
        const T2 b1 = rot(v[3], h, s3, inv);       // W6^1
        const T2 b2 = rot(v[5], -h, s3, inv);      // W6^2
        const T2 a0 = v[0], a1 = v[2], a2 = v[4];
        v[0] = cadd(a0, v[1]);
        v[3] = csub(a0, v[1]);
        v[1] = cadd(a1, b1);
        v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2);
        v[5] = csub(a2, b2);
    } else if constexpr (R == 8) {
        const T h = (T)0.70710678118654752440;
        T2 e[4] = {v[0], v[2], v[4], v[6]};
        T2 o[4] = {v[1], v[3], v[5], v[7]};
        dft_generic<4>(e, inv);
        dft_generic<4>(o, inv);
        const T2 w1 = rot(o[1], h, h, inv);
        const T2 w2 = mul_mi(o[2], inv);
        const T2 w3 = rot(o[3], -h, h, inv);
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], w1);
        v[5] = csub(e[1], w1);
        v[2] = cadd(e[2], w2);
        v[6] = csub(e[2], w2);
        v[3] = cadd(e[3], w3);
        v[7] = csub(e[3], w3);
    } else if constexpr (R == 9) {
        // n = n1 + 3 n2, k = k1 + 3 k2: radix-3 over n2, twiddle W9^(n1 k1), radix-3 over n1
        dft3(v[0], v[3], v[6], inv);
        dft3(v[1], v[4], v[7], inv);
        dft3(v[2], v[5], v[8], inv);
        const T c1 = (T)0.76604444311897803520, s1 = (T)0.64278760968653932632;    // 2 pi / 9
        const T c2 = (T)0.17364817766693034885, s2 = (T)0.98480775301220805936;    // 4 pi / 9
        const T c4 = (T)-0.93969262078590838405, s4 = (T)0.34202014332566873304;   // 8 pi / 9
        // inner results a[n1][k1] sit at v[n1 + 3 k1]
        v[4] = rot(v[4], c1, s1, inv);
        v[7] = rot(v[7], c2, s2, inv);
        v[5] = rot(v[5], c2, s2, inv);
        v[8] = rot(v[8], c4, s4, inv);
        T2 x0 = v[0], x1 = v[1], x2 = v[2];
        dft3(x0, x1, x2, inv);
        T2 y0 = v[3], y1 = v[4], y2 = v[5];
        dft3(y0, y1, y2, inv);
        T2 z0 = v[6], z1 = v[7], z2 = v[8];
        dft3(z0, z1, z2, inv);
        // X[k1 + 3 k2] = (k1-th group)[k2]
        v[0] = x0; v[3] = x1; v[6] = x2;
        v[1] = y0; v[4] = y1; v[7] = y2;
        v[2] = z0; v[5] = z1; v[8] = z2;
    }
}

// One out-of-place radix-R stage over NL element-major lines of length M (INV selects
// the inverse transform at compile time).  inv_ns = 1/Ns: j mod Ns is formed as
// j - Ns floor((j + 1/2)/Ns), exact for the j < 512, Ns <= 256 that occur (the fraction
// stays >= 1/(2 Ns) away from an integer).
template <int R, int NL, bool INV, typename T2>
__device__ __forceinline__ void fft_stage(const T2 *__restrict__ src, T2 *__restrict__ dst, int M, int Ns,
                                          float inv_ns, const T2 *__restrict__ tw)
{
    const int nbl = M / R;
    const int tstep = M / (Ns * R);
    const int nb = nbl * NL;
    const int sstride = nbl * NL, dstride = Ns * NL;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int l = b % NL, j = b / NL;
        T2 v[R];
        const T2 *s = src + b;                 // = src + j NL + l
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[r * sstride];
        int kk = 0;
        if (Ns > 1) {
            const int q = __float2int_rz(((float)j + 0.5f) * inv_ns);
            kk = j - q * Ns;
            const int step = kk * tstep;
            int t = step;
#pragma unroll
            for (int r = 1; r < R; ++r, t += step) {
                T2 w = tw[t];
                if constexpr (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft_generic<R>(v, INV);
        T2 *d = dst + ((j - kk) * R + kk) * NL + l;
#pragma unroll
        for (int r = 0; r < R; ++r) d[r * dstride] = v[r];
    }
    __syncthreads();
}

// Full transform of NL lines starting in buffer a (b is scratch of the same size);
// returns the buffer that holds the result.
template <int NL, bool INV, typename T2>
__device__ T2 *fft_run_dir(T2 *a, T2 *b, const FftPlan &plan, const T2 *tw)
{
    int Ns = 1;
    // at most four radix passes for every admissible M (the plan puts 8 and 9 first);
    // the radices are read with constant indices so the plan stays in registers
    const int rads[4] = {plan.rad[0], plan.nst > 1 ? plan.rad[1] : 1, plan.nst > 2 ? plan.rad[2] : 1,
                         plan.nst > 3 ? plan.rad[3] : 1};
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (s >= plan.nst) break;
        const int R = rads[s];
        const float inv_ns = 1.0f / (float)Ns;
        switch (R) {
        case 8: fft_stage<8, NL, INV>(a, b, plan.M, Ns, inv_ns, tw); break;
        case 9: fft_stage<9, NL, INV>(a, b, plan.M, Ns, inv_ns, tw); break;
        case 6: fft_stage<6, NL, INV>(a, b, plan.M, Ns, inv_ns, tw); break;
        case 4: fft_stage<4, NL, INV>(a, b, plan.M, Ns, inv_ns, tw); break;
        case 3: fft_stage<3, NL, INV>(a, b, plan.M, Ns, inv_ns, tw); break;
        default: fft_stage<2, NL, INV>(a, b, plan.M, Ns, inv_ns, tw); break;
        }
        Ns *= R;
        T2 *t = a;
        a = b;
        b = t;
    }
    return a;
}

template <int NL, typename T2>
__device__ T2 *fft_run(T2 *a, T2 *b, const FftPlan &plan, const T2 *tw, bool inv)
{
    return inv ? fft_run_dir<NL, true>(a, b, plan, tw) : fft_run_dir<NL, false>(a, b, plan, tw);
}

// 16-byte asynchronous global -> shared copies (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;\n" ::: "memory");
}

}  // namespace se
