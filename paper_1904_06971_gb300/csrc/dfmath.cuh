// Double-float ("df64") arithmetic on the FP32 pipe: a value is the
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2 (about 48
// significand bits).  Built on two error-free transformations: Knuth's
// two-sum (a + b = s + e exactly) and the FMA two-product (a * b = p + e
// exactly).  Every step uses the _rn intrinsics so the compiler can neither
// contract nor reorder it.
//
// The elementary functions are evaluated from their Taylor series (Horner
// form) on the bounded arguments the coefficient kernel needs:
//   sin(pi y), cos(pi y) for |pi y| <= 0.5   (terms up to y^17)
//   exp(x)               for |x| <= 1      (exp(x) = (exp(x/4))^4, terms up to (x/4)^14)
// so the truncation error stays below 2^-50 relative.
#pragma once

#include <cuda_runtime.h>

namespace iga {

struct df2 {
    float h, l;
};

__device__ __forceinline__ df2 df_make(float h, float l) { return df2{h, l}; }

__device__ __forceinline__ df2 df_from_double(double v)
{
    const float h = __double2float_rn(v);
    return df2{h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double df_to_double(df2 a) { return (double)a.h + (double)a.l; }

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// s + e = a + b exactly, assuming |a| >= |b| (or a = 0)
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df2 df_add(df2 a, df2 b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    float h, l;
    quick_two_sum(s, e, h, l);
    return df2{h, l};
}

__device__ __forceinline__ df2 df_neg(df2 a) { return df2{-a.h, -a.l}; }
__device__ __forceinline__ df2 df_sub(df2 a, df2 b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df2 df_mul(df2 a, df2 b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    float h, l;
    quick_two_sum(p, e, h, l);
    return df2{h, l};
}

// a * b + c
__device__ __forceinline__ df2 df_fma(df2 a, df2 b, df2 c) { return df_add(df_mul(a, b), c); }

// a / b: first quotient, one correction from the df remainder
__device__ __forceinline__ df2 df_div(df2 a, df2 b)
{
    const float q1 = __fdiv_rn(a.h, b.h);
    const df2 r = df_sub(a, df_mul(b, df2{q1, 0.f}));
    const float q2 = __fdiv_rn(r.h, b.h);
    float h, l;
    quick_two_sum(q1, q2, h, l);
    return df2{h, l};
}

__device__ __forceinline__ df2 df_abs(df2 a) { return a.h < 0.f ? df_neg(a) : a; }

// Taylor coefficients 1/k!, k = 0..17, and pi as exact float pairs (hi, lo):
// hi = 1/k! rounded to float, lo = the rest rounded to float (computed offline
// in 200-bit arithmetic).  Indexed with constants, so they fold to immediates.
__device__ __forceinline__ df2 df_inv_fact(int k)
{
    constexpr float H[18] = {
        0x1.000000p+0f, 0x1.000000p+0f, 0x1.000000p-1f, 0x1.555556p-3f, 0x1.555556p-5f, 0x1.111112p-7f,
        0x1.6c16c2p-10f, 0x1.a01a02p-13f, 0x1.a01a02p-16f, 0x1.71de3ap-19f, 0x1.27e4fcp-22f, 0x1.ae6456p-26f,
        0x1.1eed8ep-29f, 0x1.612462p-33f, 0x1.93974ap-37f, 0x1.ae7f3ep-41f, 0x1.ae7f3ep-45f, 0x1.952c78p-49f};
    constexpr float L[18] = {
        0.0f, 0.0f, 0.0f, -0x1.555556p-28f, -0x1.555556p-30f, -0x1.ddddde0p-32f,
        -0x1.27d27ep-35f, -0x1.7f97fap-39f, -0x1.7f97fap-42f, 0x1.55b1ccp-45f, -0x1.10ec14p-47f, 0x1.fd5138p-52f,
        0x1.ff1b12p-54f, -0x1.8af25ep-58f, 0x1.180f94p-62f, 0x1.ccee08p-67f, 0x1.ccee08p-71f, -0x1.f9ea56p-74f};
    return df2{H[k], L[k]};
}

__device__ __forceinline__ df2 df_pi() { return df2{0x1.921fb6p+1f, -0x1.777a5cp-24f}; }

// sin(pi y) and cos(pi y) for |pi y| <= 0.5: with t = pi y,
//   sin t = t (1 - t^2/3! + t^4/5! - ...),  cos t = 1 - t^2/2! + t^4/4! - ...
__device__ __forceinline__ void df_sincospi_small(df2 y, df2& s, df2& c)
{
    const df2 t = df_mul(df_pi(), y);
    const df2 t2 = df_mul(t, t);
    // sin: sum_{k=0..8} (-1)^k t^{2k} / (2k+1)!
    df2 ps = df_inv_fact(17);
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        ps = df_neg(df_mul(ps, t2));
        ps = df_add(ps, df_inv_fact(2 * k + 1));
    }
    s = df_mul(t, ps);
    // cos: sum_{k=0..8} (-1)^k t^{2k} / (2k)!
    df2 pc = df_inv_fact(16);
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        pc = df_neg(df_mul(pc, t2));
        pc = df_add(pc, df_inv_fact(2 * k));
    }
    c = pc;
}

// exp(x) for |x| <= 1: exp(x) = e(x/4)^4 with e(u) = sum_{k=0..14} u^k / k!
__device__ __forceinline__ df2 df_exp_small(df2 x)
{
    const df2 u = df2{__fmul_rn(x.h, 0.25f), __fmul_rn(x.l, 0.25f)};   // exact scaling by a power of 2
    df2 e = df_inv_fact(14);
#pragma unroll
    for (int k = 13; k >= 0; --k) e = df_add(df_mul(e, u), df_inv_fact(k));
    e = df_mul(e, e);
    return df_mul(e, e);
}

}  // namespace iga
