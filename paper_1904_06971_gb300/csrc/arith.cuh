// Arithmetic policies of the quadrature contractions.
//
// GB300 executes FP32 FMAs about 64x faster than FP64 FMAs, so FP64-accurate
// contractions are also offered in double-float ("df64") arithmetic: a value
// is an unevaluated sum hi + lo of two floats (about 48 significand bits), a
// product is formed exactly with an FMA (Dekker/Ogita-Rump-Oishi error-free
// product) and sums use Knuth's error-free two-sum, with the low parts
// accumulated separately and renormalised when a sum is stored.  All the
// error-free steps use the _rn intrinsics so the compiler cannot contract or
// reorder them.
//
//   PolF64  : store double, accumulate double (FP64 pipe)
//   PolDF   : store float2 (hi, lo), accumulate double-float (FP32 pipe)
//   PolF32  : store float, accumulate float (FP32 pipe)
#pragma once

#include <cuda_runtime.h>

#include <cstring>

namespace iga {

enum Arith { kArithF64 = 0, kArithDF = 1, kArithF32 = 2 };

struct PolF64 {
    using store = double;
    using acc = double;
    static constexpr int kind = kArithF64;
    __device__ __forceinline__ static acc zero() { return 0.0; }
    __device__ __forceinline__ static void mac(acc& a, store x, store v) { a = fma(x, v, a); }
    __device__ __forceinline__ static double to_double(const acc& a) { return a; }
    __device__ __forceinline__ static float to_float(const acc& a) { return __double2float_rn(a); }
    __device__ __forceinline__ static store to_store(const acc& a) { return a; }
    __device__ __forceinline__ static store from_double(double v) { return v; }
};

struct DFAcc {
    float h, l;
};

// Exact float -> double conversion by integer operations only (sign, rebiased
// exponent, widened significand; subnormals normalised with a leading-zero
// count; infinities and NaNs keep their payload), so it stays off GB300's
// slow FP64 pipe where the hardware conversion instruction runs.  Every case
// is integer arithmetic and selects: no branch that could fall back on the
// hardware conversion.  Host-callable for testing.
__host__ __device__ __forceinline__ unsigned int f2d_bits_of(float f)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    unsigned int u;
    memcpy(&u, &f, sizeof(u));
    return u;
#endif
}
__host__ __device__ __forceinline__ int f2d_clz(unsigned int x)
{
#ifdef __CUDA_ARCH__
    return __clz(x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}
__host__ __device__ __forceinline__ double f2d_exact(float f)
{
    const unsigned int u = f2d_bits_of(f);
    const unsigned int e = (u >> 23) & 0xffu;
    const unsigned int m = u & 0x7fffffu;
    // normal: exponent e - 127 + 1023; infinity / NaN: 0x7ff
    unsigned long long ed = (e == 0xffu) ? 0x7ffull : (unsigned long long)(e + 896u);
    unsigned long long md = (unsigned long long)m << 29;
    if (e == 0u) {
        // m 2^-149 with the leading one of m at bit 31 - lz: exponent 905 - lz,
        // the bits below it left-aligned in the 52-bit field (zero: m = 0)
        const int lz = f2d_clz(m);
        ed = m ? (unsigned long long)(905 - lz) : 0ull;
        md = m ? (((unsigned long long)m << (21 + lz)) & 0xfffffffffffffull) : 0ull;
    }
    const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) | (ed << 52) | md;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)d);
#else
    double r;
    memcpy(&r, &d, sizeof(r));
    return r;
#endif
}

__host__ __device__ __forceinline__ unsigned long long df_bits64(double d)
{
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(d);
#else
    unsigned long long u;
    memcpy(&u, &d, sizeof(u));
    return u;
#endif
}
__host__ __device__ __forceinline__ double df_from_bits64(unsigned long long u)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double d;
    memcpy(&d, &u, sizeof(d));
    return d;
#endif
}
__host__ __device__ __forceinline__ float df_add_rn(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}

// The double nearest to the exact sum h + l of two floats, computed with FP32
// adds and integer operations only (no FP64 instruction on the common path):
// a two-sum makes the pair non-overlapping (|l| <= ulp(h)/2); the double of h
// is built from its bits, and l is added as a whole number k of double ulps of
// h, rounded to nearest-even (k < 2^30, so it only changes the low bits of the
// significand; when h is a power of two and l has the other sign the result
// lies in the binade below, whose ulp is half as large).  Equal, bit for bit,
// to (double)h + (double)l.  Zeros, subnormals, infinities and NaNs take the
// plain FP64 add.  Host-callable for testing.
__host__ __device__ __forceinline__ double df2d_exact(float h0, float l0)
{
    const float h = df_add_rn(h0, l0);
    const float z = df_add_rn(h, -h0);
    const float l = df_add_rn(df_add_rn(h0, -df_add_rn(h, -z)), df_add_rn(l0, -z));
    const unsigned int hb = f2d_bits_of(h), lb = f2d_bits_of(l);
    const unsigned int eh = (hb >> 23) & 0xffu, el = (lb >> 23) & 0xffu;
    if (eh == 0u || eh == 0xffu || (el == 0u && (lb & 0x7fffffffu)) || el == 0xffu)
        return f2d_exact(h0) + f2d_exact(l0);
    const unsigned long long H = ((unsigned long long)(hb & 0x80000000u) << 32) |
                                 ((unsigned long long)(eh + 896u) << 52) |
                                 ((unsigned long long)(hb & 0x7fffffu) << 29);
    if (el == 0u) return df_from_bits64(H);            // l == 0
    const bool opposite = ((hb ^ lb) >> 31) != 0u;
    const bool down = opposite && (hb & 0x7fffffu) == 0u;
    const unsigned long long ml = (unsigned long long)((lb & 0x7fffffu) | 0x800000u);
    // l = ml 2^(el-150); one double ulp of h is 2^(eh-179) (2^(eh-180) in the binade below)
    const int sh = (int)el - (int)eh + 29 + (down ? 1 : 0);
    unsigned long long k;
    if (sh >= 0) {
        k = ml << sh;
    } else if (sh > -26) {
        const int r = -sh;
        k = (ml + ((1ull << (r - 1)) - 1ull) + ((ml >> r) & 1ull)) >> r;     // round half to even
    } else {
        k = 0ull;
    }
    return df_from_bits64(opposite ? H - k : H + k);
}

__host__ __device__ __forceinline__ float f_from_bits(unsigned int u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, sizeof(f));
    return f;
#endif
}

// (hi, lo) floats with hi + lo = v to about 48 bits, by integer operations:
// hi keeps the top 24 significand bits of v (truncated), lo the next 24 of the
// remaining 29 (truncated), so |v - hi - lo| < 2^-47 |v|.  Values below 2^-74
// in magnitude (lo would be subnormal), infinities and NaNs take the FP64
// conversion.  Host-callable for testing.
__host__ __device__ __forceinline__ float2 d2df_split(double v)
{
    const unsigned long long u = df_bits64(v);
    const int e = (int)((u >> 52) & 0x7ffu);
    const int ef = e - 896;                             // float exponent field of hi
    if (ef < 53 || ef > 254) {
        const float h = (float)v;
        return make_float2(h, (float)(v - (double)h));
    }
    const unsigned int sign = (unsigned int)(u >> 32) & 0x80000000u;
    const float h = f_from_bits(sign | ((unsigned int)ef << 23) | ((unsigned int)(u >> 29) & 0x7fffffu));
    const unsigned int r = (unsigned int)u & 0x1fffffffu;   // v - h = r 2^(e - 1075)
    if (r == 0u) return make_float2(h, 0.f);
    const int b = 31 - f2d_clz(r);                       // leading one of r (0..28)
    const unsigned int m = (b >= 23) ? (r >> (b - 23)) : (r << (23 - b));
    const float l = f_from_bits(sign | ((unsigned int)(b + e - 948) << 23) | (m & 0x7fffffu));
    return make_float2(h, l);
}

struct PolDF {
    using store = float2;
    using acc = DFAcc;
    static constexpr int kind = kArithDF;
    __device__ __forceinline__ static acc zero() { return DFAcc{0.f, 0.f}; }
    __device__ __forceinline__ static void mac(acc& a, store x, store v)
    {
        // x*v = ph + pe exactly for the high parts; the cross terms join pe
        const float ph = __fmul_rn(x.x, v.x);
        float pe = __fmaf_rn(x.x, v.x, -ph);
        pe = __fmaf_rn(x.x, v.y, pe);
        pe = __fmaf_rn(x.y, v.x, pe);
        // two-sum of the running high part and ph
        const float s = __fadd_rn(a.h, ph);
        const float z = __fsub_rn(s, a.h);
        const float t = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, z)), __fsub_rn(ph, z));
        a.h = s;
        a.l = __fadd_rn(a.l, __fadd_rn(t, pe));
    }
    // the double nearest to hi + lo (bit for bit df2d_exact): two exact conversions and one FP64 add;
    // the quadrature stages convert one value per ~10^2 multiply-adds, where the add is free and the
    // integer-only df2d_exact costs more issue slots (kernels bound by the FP64 pipe call df2d_exact)
    __device__ __forceinline__ static double to_double(const acc& a) { return f2d_exact(a.h) + f2d_exact(a.l); }
    // the float nearest to hi + lo: one rounding of the exact sum
    __device__ __forceinline__ static float to_float(const acc& a) { return __fadd_rn(a.h, a.l); }
    __device__ __forceinline__ static store to_store(const acc& a)
    {
        const float s = __fadd_rn(a.h, a.l);
        return make_float2(s, __fsub_rn(a.l, __fsub_rn(s, a.h)));
    }
    __device__ __forceinline__ static store from_double(double v)
    {
        const float h = __double2float_rn(v);
        return make_float2(h, __double2float_rn(v - (double)h));
    }
};

struct PolF32 {
    using store = float;
    using acc = float;
    static constexpr int kind = kArithF32;
    __device__ __forceinline__ static acc zero() { return 0.f; }
    __device__ __forceinline__ static void mac(acc& a, store x, store v) { a = __fmaf_rn(x, v, a); }
    __device__ __forceinline__ static double to_double(const acc& a) { return (double)a; }
    __device__ __forceinline__ static float to_float(const acc& a) { return a; }
    __device__ __forceinline__ static store to_store(const acc& a) { return a; }
    __device__ __forceinline__ static store from_double(double v) { return __double2float_rn(v); }
};

}  // namespace iga
