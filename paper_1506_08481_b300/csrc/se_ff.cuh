// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// (|lo| <= ulp(hi) / 2 after normalisation), carrying about 44 significant bits.  The
// products of the FP64-equivalent mode (SE_OPT_PRECISION 2) run their spread and gather
// in it: B300's FP32 pipe issues many times the FMAs of its FP64 pipe, and a double-float
// multiply-add costs about a dozen FP32 instructions.  The type `ff` carries the
// arithmetic operators the templated spread, gather and combine code uses, so those
// kernels are instantiated on it unchanged.
//
// Building blocks (exact transformations of FP32 arithmetic; Dekker 1971, Knuth's
// TwoSum): fl(a b) + fma(a, b, -fl(a b)) = a b, and two_sum(a, b) = a + b exactly as s + e.
// Products keep the cross terms a.hi b.lo + a.lo b.hi; sums add the low parts after
// the exact sum of the high parts (the "sloppy" double-float sum: relative error
// ~2^-44 of the larger operand).
#pragma once

#include <cuda_runtime.h>

namespace se {

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)   // |a| >= |b|
{
    s = a + b;
    e = b - (s - a);
}

struct ff {
    float hi, lo;
    ff() = default;
    __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    __device__ ff(int v) : hi((float)v), lo((float)(v - (int)(float)v)) {}
    __device__ ff(float v) : hi(v), lo(0.f) {}
    __device__ ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __device__ explicit operator float() const { return hi + lo; }
    __device__ explicit operator int() const { return (int)((double)hi + (double)lo); }
};

__device__ __forceinline__ ff ff_norm(float hi, float lo)
{
    ff r;
    fast_two_sum(hi, lo, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ ff operator+(ff a, ff b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return ff_norm(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return ff_norm(p, e);
}
__device__ __forceinline__ ff operator/(ff a, ff b)
{
    // q1 = a/b to FP32, one correction step on the double-float remainder
    const float q1 = a.hi / b.hi;
    const ff r = a - b * ff(q1);
    const float q2 = r.hi / b.hi;
    return ff_norm(q1, q2);
}
__device__ __forceinline__ ff &operator+=(ff &a, ff b) { return a = a + b; }
__device__ __forceinline__ ff &operator-=(ff &a, ff b) { return a = a - b; }
__device__ __forceinline__ ff &operator*=(ff &a, ff b) { return a = a * b; }
__device__ __forceinline__ bool operator==(ff a, ff b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(ff a, ff b) { return !(a == b); }

// Multiply-add loops.  lazy_madd(acc, a, b) is acc += a b; on double-floats the product's
// high part joins the accumulator's high part by an exact TwoSum and every error term (the
// TwoSum's, the product's rounding and its cross terms) collects in the low part, which is
// left unnormalised until lazy_finish(acc): about a dozen FP32 instructions per term
// instead of the two normalisations of a separate multiply and add.  A loop of n terms
// leaves |lo| up to about n ulp(hi), so it is finished after tens of terms, not thousands.
template <typename T>
__device__ __forceinline__ void lazy_madd(T &acc, T a, T b) { acc += a * b; }
__device__ __forceinline__ void lazy_madd(ff &acc, ff a, ff b)
{
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    float s, err;
    two_sum(acc.hi, p, s, err);
    acc.hi = s;
    acc.lo += err + e;
}
template <typename T>
__device__ __forceinline__ void lazy_finish(T &) {}
__device__ __forceinline__ void lazy_finish(ff &acc) { acc = ff_norm(acc.hi, acc.lo); }

// warp exchange of any arithmetic type or of a double-float
template <typename T>
__device__ __forceinline__ T shfl_xor(unsigned mask, T v, int off) { return __shfl_xor_sync(mask, v, off); }
__device__ __forceinline__ ff shfl_xor(unsigned mask, ff v, int off)
{
    return ff(__shfl_xor_sync(mask, v.hi, off), __shfl_xor_sync(mask, v.lo, off));
}

// Square root of a double-float: one Newton step from the FP32 root, r = s + (a - s^2) / (2 s),
// with s^2 formed exactly (two-product); relative error about 2^-44.
__device__ __forceinline__ ff ff_sqrt(ff a)
{
    const float s = sqrtf(a.hi);
    const float p = s * s, e = fmaf(s, s, -p);
    const ff d = a - ff(p, e);
    return ff_norm(s, d.hi / (2.0f * s));
}

// exp(t) of a double-float argument, -87 < t <= 0 (results stay normal FP32 numbers): the
// textbook argument reduction t = k ln 2 + u, |u| <= ln2 / 2, with ln 2 = L1 + L2 split so that
// k L1 is exact (L1 = 2839 / 4096 has 12 significant bits, |k| < 2^7), exp(u) by its Taylor
// series to degree 11 in double-float Horner form (truncation 6e-15 relative at |u| = ln2 / 2),
// then the exact scaling by 2^k.
__device__ __forceinline__ ff ff_exp(ff t)
{
    // 1/n! as double-floats, n = 0..11
    constexpr float c[12][2] = {{1.0f, 0.0f},
                                {1.0f, 0.0f},
                                {0.5f, 0.0f},
                                {0.1666666716337204f, -4.967053879312289e-09f},
                                {0.0416666679084301f, -1.2417634698280722e-09f},
                                {0.008333333767950535f, -4.34617203337595e-10f},
                                {0.0013888889225199819f, -3.3631094437103215e-11f},
                                {0.00019841270113829523f, -2.725596874933456e-12f},
                                {2.4801587642286904e-05f, -3.40699609366682e-13f},
                                {2.7557318844628753e-06f, 3.793571224297229e-14f},
                                {2.755731998149713e-07f, -7.575112209051195e-15f},
                                {2.5052107943679403e-08f, 4.4176230446483665e-16f}};
    constexpr float L1 = 0.693115234375f, L2h = 3.194618329871446e-05f, L2l = 1.6465949697480609e-12f;
    const float k = rintf(t.hi * 1.44269504088896341f);
    const ff u = (t - ff(k * L1, 0.f)) - ff(k) * ff(L2h, L2l);
    ff q(c[11][0], c[11][1]);
#pragma unroll
    for (int n = 10; n >= 0; --n) q = q * u + ff(c[n][0], c[n][1]);
    const int ki = (int)k;
    return ff(ldexpf(q.hi, ki), ldexpf(q.lo, ki));
}

struct __align__(32) ff4 {
    ff x, y, z, w;
};

}  // namespace se
