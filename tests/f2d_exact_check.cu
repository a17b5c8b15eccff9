// Host check of the integer float -> double conversion used by the double-float
// kernels (arith.cuh f2d_exact): every one of the 2^32 float bit patterns against
// the host compiler's conversion, bit for bit (NaNs up to the quiet bit, which a
// host conversion may set).  Prints the mismatch count; exit status 0 iff none.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "arith.cuh"

int main()
{
    unsigned long long bad = 0;
    for (uint64_t k = 0; k <= 0xffffffffull; ++k) {
        const uint32_t u = (uint32_t)k;
        float f;
        memcpy(&f, &u, sizeof(f));
        const double a = iga::f2d_exact(f), b = (double)f;
        uint64_t ba, bb;
        memcpy(&ba, &a, sizeof(ba));
        memcpy(&bb, &b, sizeof(bb));
        bool ok = ba == bb;
        if (!ok && std::isnan(a) && std::isnan(b)) ok = (ba | (1ull << 51)) == (bb | (1ull << 51));
        if (!ok && bad++ < 8)
            printf("mismatch %08x: %016llx vs %016llx\n", u, (unsigned long long)ba, (unsigned long long)bb);
    }
    printf("mismatches: %llu\n", bad);
    return bad != 0;
}
