// Two-float ("double-float") arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi)/2, giving about 48 significant bits on the FP32 pipes.  On
// B300 the FP64 pipe delivers 1/64 of the FP32 rate, so these operations (7-20 FP32
// instructions each) run several times faster than native FP64 while keeping the element
// kernels within the FP64 parity tolerance.
//
// Building blocks (error-free transformations):
//   TwoSum (Knuth):       s = a + b exactly as s + e, any |a|, |b|
//   FastTwoSum (Dekker):  same when |a| >= |b|
//   TwoProduct (FMA):     p = a * b exactly as p + e with e = fma(a, b, -p)
// Every FP32 operation below uses an explicit round-to-nearest intrinsic so the compiler
// cannot contract or reorder it.  Additions are the "sloppy" variant (error bounded by
// 2^-47 (|a| + |b|)), sufficient for the normwise error metric used by this library.
#pragma once

#include <cuda_runtime.h>

namespace jetsci {

// 8-byte aligned, so that a value moves through shared memory in one 64-bit access.
struct __align__(8) df64 {
    float h, l;
    df64() = default;
    __host__ __device__ constexpr df64(float hi, float lo) : h(hi), l(lo) {}
    __host__ __device__ constexpr df64(int i) : h((float)i), l(0.0f) {}
    __host__ __device__ constexpr df64(float f) : h(f), l(0.0f) {}
    __host__ __device__ constexpr df64(double d) : h((float)d), l((float)(d - (double)(float)d)) {}
    __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
};

__device__ __forceinline__ df64 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return df64(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
    df64 s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.h, -a.l); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return fast_two_sum(p, e);
}

// a * b + c with one renormalisation.
__device__ __forceinline__ df64 df_fma(df64 a, df64 b, df64 c) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    df64 s = two_sum(p, c.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(e, c.l)));
}

// Accumulation step c + a * b for running sums: as df_fma without the final renormalisation
// (12 instead of 15 FP32 instructions).  The low part of the result is not reduced below
// ulp(hi)/2, so it may only feed further df_fma_acc steps and then df_acc_norm.  Over a few
// dozen terms the low part stays a few ulps of the high part, and the error stays ~2^-47 of the
// terms' magnitudes.
__device__ __forceinline__ df64 df_fma_acc(df64 a, df64 b, df64 c) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const df64 s = two_sum(c.h, p);
    return df64(s.h, __fadd_rn(c.l, __fadd_rn(s.l, e)));
}
__device__ __forceinline__ df64 df_acc_norm(df64 a) { return fast_two_sum(a.h, a.l); }

__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }

__device__ __forceinline__ bool operator>(df64 a, df64 b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }
__device__ __forceinline__ bool operator<(df64 a, df64 b) { return b > a; }

__device__ __forceinline__ bool isfinite(df64 a) { return ::isfinite(a.h) && ::isfinite(a.l); }

// 1/a: FP32 reciprocal refined by one Newton step x1 = x0 + x0 (1 - a x0) in two-float
// arithmetic (quadratic convergence: 2^-24 -> about 2^-48).
__device__ __forceinline__ df64 df_rcp(df64 a) {
    const df64 x0(__frcp_rn(a.h), 0.0f);
    const df64 r = df_fma(-a, x0, df64(1.0f));
    return df_fma(x0, r, x0);
}

__device__ __forceinline__ df64 operator/(df64 a, df64 b) { return a * df_rcp(b); }

// ln x for x > 0: x = 2^k m with m in [sqrt(1/2), sqrt(2)), exact scaling of both parts;
// ln m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), s = (m - 1)/(m + 1), |s| <= 0.1716, so
// s^2 <= 0.0295 and eleven terms of the series leave a truncation error below 2^-50.
__device__ __forceinline__ df64 df_log(df64 x) {
    int k;
    float f = frexpf(x.h, &k);  // x.h = f 2^k, f in [0.5, 1)
    if (f < 0.70710678f) k -= 1;
    const df64 m(ldexpf(x.h, -k), ldexpf(x.l, -k));
    const df64 s = (m - df64(1.0f)) * df_rcp(m + df64(1.0f));
    const df64 z = s * s;
    // Horner in z for sum_{j=0}^{10} z^j / (2j + 1)
    df64 p(1.0 / 21.0);
    p = df_fma(p, z, df64(1.0 / 19.0));
    p = df_fma(p, z, df64(1.0 / 17.0));
    p = df_fma(p, z, df64(1.0 / 15.0));
    p = df_fma(p, z, df64(1.0 / 13.0));
    p = df_fma(p, z, df64(1.0 / 11.0));
    p = df_fma(p, z, df64(1.0 / 9.0));
    p = df_fma(p, z, df64(1.0 / 7.0));
    p = df_fma(p, z, df64(1.0 / 5.0));
    p = df_fma(p, z, df64(1.0 / 3.0));
    p = df_fma(p, z, df64(1.0f));
    const df64 lnm = (s + s) * p;
    const df64 ln2(0.69314718055994530942);
    return df_fma(ln2, df64((float)k), lnm);
}

// ---------------------------------------------------------------------------------------
// Conversions by bit manipulation.  On B300 every FP64 instruction, conversions included,
// issues on the narrow FP64 pipe; these use integer and FP32 instructions only.

// float -> double, exact for normal floats and zero (subnormal floats flush to zero).
__device__ __forceinline__ double f2d_bits(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xFFu;
    if (e == 0) return 0.0;
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    const unsigned long long ex = (e == 0xFFu) ? 0x7FFull : (unsigned long long)(e - 127u + 1023u);
    const unsigned long long man = (unsigned long long)(b & 0x7FFFFFu) << 29;
    return __longlong_as_double((long long)(sign | (ex << 52) | man));
}

// double -> two-float: hi = the leading 24 significant bits (truncated), lo = the remaining
// 29 bits rounded to float, so hi + lo carries about 48 bits.  Magnitudes below 2^-100 flush
// to zero; magnitudes beyond the float range become infinities.
__device__ __forceinline__ df64 split_double(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int ue = (int)((b >> 52) & 0x7FFull) - 1023;
    const uint32_t s = (uint32_t)(b >> 63);
    if (ue < -100) return df64(0.0f, 0.0f);
    if (ue > 127) return df64(__uint_as_float((s << 31) | 0x7F800000u), 0.0f);
    const unsigned long long man = b & 0xFFFFFFFFFFFFFull;
    const float hi = __uint_as_float((s << 31) | ((uint32_t)(ue + 127) << 23) | (uint32_t)(man >> 29));
    float lo = ldexpf(__uint2float_rn((uint32_t)(man & 0x1FFFFFFFull)), ue - 52);
    return df64(hi, s ? -lo : lo);
}

__device__ __forceinline__ double df_to_double(df64 x) { return f2d_bits(x.h) + f2d_bits(x.l); }

__device__ __forceinline__ df64 shfl_df(df64 v, int src, int width) {
    return df64(__shfl_sync(0xffffffffu, v.h, src, width), __shfl_sync(0xffffffffu, v.l, src, width));
}

__device__ __forceinline__ df64 shfl_xor_df(df64 v, int mask, int width) {
    return df64(__shfl_xor_sync(0xffffffffu, v.h, mask, width), __shfl_xor_sync(0xffffffffu, v.l, mask, width));
}

}  // namespace jetsci
