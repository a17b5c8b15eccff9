// Host check of the integer double-float -> double conversion (arith.cuh
// df2d_exact): for pairs (h, l) of floats it must equal the IEEE double sum
// (double)h + (double)l bit for bit.  Cases: seeded random pairs over every
// exponent gap from overlapping to negligible, both signs, powers of two with
// a low part of the other sign (the result falls into the binade below),
// exact half-ulp ties (round half to even), zeros, subnormals, infinities and
// NaNs.  Also d2df_split, the integer split of a double into (hi, lo) floats:
// hi must be v truncated to 24 significand bits and |v - hi - lo| < 2^-47 |v|.
// Prints the mismatch count; exit status 0 iff none.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "arith.cuh"

static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint64_t next()
{
    state ^= state << 13;
    state ^= state >> 7;
    state ^= state << 17;
    return state;
}
static float f_of(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint64_t bits(double d) { uint64_t u; memcpy(&u, &d, 8); return u; }

static unsigned long long bad = 0, total = 0;
static void check(float h, float l)
{
    const double a = iga::df2d_exact(h, l), b = (double)h + (double)l;
    ++total;
    bool ok = bits(a) == bits(b) || (std::isnan(a) && std::isnan(b));
    if (!ok && bad++ < 8)
        printf("mismatch h=%a l=%a: %a vs %a\n", (double)h, (double)l, a, b);
}

int main()
{
    // random pairs: h with a random exponent in [-60, 60], l = h 2^-gap times a random significand
    for (int n = 0; n < 20000000; ++n) {
        const uint64_t r = next();
        const int eh = (int)(r % 121) - 60;
        const uint32_t mh = (uint32_t)(r >> 8) & 0x7fffffu;
        const uint32_t sh = (uint32_t)(r >> 40) & 1u, sl = (uint32_t)(r >> 41) & 1u;
        const int gap = (int)((r >> 42) % 64);          // 0: overlapping parts
        const uint32_t ml = (uint32_t)(next()) & 0x7fffffu;
        const float h = f_of((sh << 31) | ((uint32_t)(eh + 127) << 23) | ((n % 7 == 0) ? 0u : mh));
        const int el = eh - gap;
        const float l = (el > -126) ? f_of((sl << 31) | ((uint32_t)(el + 127) << 23) | ml) : 0.0f;
        check(h, l);
    }
    // exact ties: l = half a double ulp of h (and 3/2, 5/2 ...), both signs, odd and even h significands
    for (int eh = -20; eh <= 20; ++eh)
        for (uint32_t mh = 0; mh < 64; ++mh)
            for (int k = 1; k < 16; k += 2)
                for (int s = 0; s < 4; ++s) {
                    const float h = f_of(((uint32_t)(s & 1) << 31) | ((uint32_t)(eh + 127) << 23) | (mh * 131071u & 0x7fffffu));
                    const float l = (float)std::ldexp((s & 2) ? -(double)k : (double)k, eh - 53);
                    check(h, l);
                    check(h, std::nextafter(l, 0.0f));
                    check(h, std::nextafter(l, 1e30f));
                }
    // specials
    const float sp[] = {0.0f, -0.0f, 1.0f, -1.0f, 1e-45f, -1e-45f, 1e-40f, 1.17549435e-38f, 3.4e38f, -3.4e38f,
                        INFINITY, -INFINITY, NAN, 0.5f, 2.0f, 1.0000001f, 0.99999994f, 1e-30f, 1e30f};
    for (float a : sp)
        for (float b : sp) check(a, b);
    // d2df_split over random doubles of magnitude 2^-70 .. 2^120 and both signs
    for (int n = 0; n < 5000000; ++n) {
        const uint64_t r = next();
        const uint64_t e = 1023 - 70 + (r % 190);
        const uint64_t bitsv = ((r >> 63) << 63) | (e << 52) | (next() & 0xfffffffffffffull);
        double v;
        memcpy(&v, &bitsv, 8);
        const float2 p = iga::d2df_split(v);
        const uint64_t tbits = bitsv & ~((1ull << 29) - 1);      // v truncated to 24 significand bits
        double hi_trunc;
        memcpy(&hi_trunc, &tbits, 8);
        const double err = std::fabs(v - (double)p.x - (double)p.y);
        ++total;
        if (((double)p.x != hi_trunc || !(err <= std::ldexp(std::fabs(v), -47))) && bad++ < 8)
            printf("split mismatch v=%a: hi=%a lo=%a\n", v, (double)p.x, (double)p.y);
    }
    printf("cases: %llu mismatches: %llu\n", total, bad);
    return bad != 0;
}
