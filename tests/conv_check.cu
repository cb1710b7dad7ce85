// Host check of the integer-pipe float <-> double conversions used by the
// FP32 path against the compiler's own IEEE conversions: exact widening and
// round-to-nearest-even narrowing, with the stated flush of values below the
// smallest normal float to signed zero; a NaN stays a NaN of the same sign.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "stage.cuh"

static uint64_t dbits(double d) { uint64_t u; memcpy(&u, &d, 8); return u; }
static uint32_t fb(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

int main() {
    long bad = 0, n = 0;
    for (uint64_t u = 0; u <= 0xffffffffull; u += 1) {
        const uint32_t v = (uint32_t)u;
        float f;
        memcpy(&f, &v, 4);
        const double got = osb::f2d_bits(f);
        double want = (double)f;
        if ((v & 0x7f800000u) == 0) want = std::copysign(0.0, (double)f);  // flush
        ++n;
        if (std::isnan(want) ? !std::isnan(got) || (dbits(got) >> 63) != (dbits(want) >> 63)
                             : dbits(got) != dbits(want)) {
            if (bad++ < 5) printf("widen %08x\n", v);
        }
    }
    std::mt19937_64 rng(2024);
    for (int e = 0; e < 2048; ++e)
        for (int s = 0; s < 2; ++s)
            for (int k = 0; k < 4000; ++k) {
                uint64_t m = rng() & 0xfffffffffffffull;
                if (k % 4 == 1) m = (m & ~0x1fffffffull) | 0x10000000ull;  // exact ties
                if (k % 4 == 2) m |= 0x1fffffffull;                         // just below a carry
                const uint64_t x = ((uint64_t)s << 63) | ((uint64_t)e << 52) | m;
                double d;
                memcpy(&d, &x, 8);
                const float got = osb::d2f_bits(d);
                float want = (float)d;
                if (std::fabs(want) < 1.17549435e-38f) want = std::copysign(0.0f, want);  // flush
                ++n;
                const bool ok = std::isnan(want) ? (std::isnan(got) && (fb(got) & 0x400000u) &&
                                                    (fb(got) >> 31) == (fb(want) >> 31))
                                                 : fb(got) == fb(want);
                if (!ok && bad++ < 10) printf("narrow %016llx\n", (unsigned long long)x);
            }
    printf("checked %ld values, %ld mismatches\n", n, bad);
    return bad ? 1 : 0;
}
