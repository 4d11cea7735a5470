// dfloat.cuh -- double-float arithmetic for the residual transforms of the
// refined precision form.
//
// A df32 carries a real number as the unevaluated sum hi + lo of two FP32
// values with |lo| <= ulp(hi) / 2: a 48-bit significand (unit roundoff
// ~2^-48 = 3.6e-15) in the exponent range of FP32, which covers the stresses
// and spectra of this solver by many orders of magnitude.  The operations are
// the classical error-free transformations: Knuth's two-sum for the sum of the
// leading parts, the exact FMA residual a*b - fl(a*b) for products, and a
// fast two-sum renormalisation (Dekker 1971; the "sloppy" double-double sum,
// whose error is bounded relative to |a| + |b|, which is the bound a
// norm-wise FFT error analysis uses).  Every step goes through the _rn
// intrinsics so the compiler cannot contract or reorder it.
//
// FP32 runs ~63x faster than FP64 on this GPU (combo_arith_rates); a df32 add or multiply costs
// 7-11 FP32 instructions, so transforms in df32 run several times faster than
// in FP64 while their rounding error stays far below the 1e-8 equilibrium
// tolerance the residual is compared against.
#pragma once
#include <cuda_runtime.h>

namespace combo {

struct __align__(8) df32 {
    float hi, lo;
    df32() = default;
    __host__ __device__ constexpr df32(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr explicit df32(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ constexpr explicit operator float() const { return hi + lo; }
};

struct __align__(16) df2 {
    df32 x, y;
};

// s + e with |e| small against s -> normalised pair
__device__ __forceinline__ df32 df_fast_two_sum(float s, float e)
{
    const float h = __fadd_rn(s, e);
    return df32(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ df32 operator+(df32 a, df32 b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(s, e);
}

__device__ __forceinline__ df32 operator-(df32 a) { return df32(-a.hi, -a.lo); }
__device__ __forceinline__ df32 operator-(df32 a, df32 b) { return a + (-b); }

__device__ __forceinline__ df32 operator*(df32 a, df32 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

__device__ __forceinline__ df32 operator/(df32 a, df32 b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const df32 r = a - b * df32(q1, 0.f);
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return df_fast_two_sum(q1, q2);
}

__device__ __forceinline__ df32& operator+=(df32& a, df32 b) { return a = a + b; }
__device__ __forceinline__ df32& operator-=(df32& a, df32 b) { return a = a - b; }
__device__ __forceinline__ df32& operator*=(df32& a, df32 b) { return a = a * b; }

__device__ __forceinline__ bool operator>(df32 a, df32 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(df32 a, df32 b) { return b > a; }

// Natural logarithm of x > 0 (x.hi a normal FP32 number) in double-float
// arithmetic, from the series ln m = 2 atanh((m - 1)/(m + 1)) =
// 2 sum_j u^(2j+1) / (2j+1) (Abramowitz & Stegun 4.1.27) after the range
// reduction x = 2^k m, m in [1/sqrt(2), sqrt(2)) (scaling by a power of two is
// exact), so |u| <= 0.1716 and u^2 <= 0.0295: the terms up to j = 10 leave a
// truncation below 0.0295^11 / 23 < 2^-60 relative.  Horner in w = u^2, all in
// double-float; ln 2 enters as the double-float split of its FP64 value.
// Keeps the logarithm of the double-float Neo-Hookean stress off the FP64 pipe.
__device__ __forceinline__ df32 df_log(df32 x)
{
    int k;
    float mh = frexpf(x.hi, &k);  // x.hi = mh 2^k, mh in [0.5, 1)
    if (mh < 0.70710678f) k -= 1;
    const float sc = ldexpf(1.f, -k);
    const df32 m(x.hi * sc, x.lo * sc);
    const df32 one(1.f, 0.f);
    const df32 u = (m - one) / (m + one);
    const df32 w = u * u;
    constexpr df32 c[12] = {df32(1.0),        df32(1.0 / 3.0),  df32(1.0 / 5.0),  df32(1.0 / 7.0),
                            df32(1.0 / 9.0),  df32(1.0 / 11.0), df32(1.0 / 13.0), df32(1.0 / 15.0),
                            df32(1.0 / 17.0), df32(1.0 / 19.0), df32(1.0 / 21.0), df32(1.0 / 23.0)};
    df32 s = c[11];
#pragma unroll
    for (int j = 10; j >= 1; j--) s = c[j] + w * s;
    const df32 at = u + u * (w * s);
    constexpr df32 ln2(0.6931471805599453);
    return ln2 * df32((float)k, 0.f) + (at + at);
}

}  // namespace combo
