// dd.cuh -- double-float ("double-word") arithmetic: a value is the unevaluated
// sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant
// bits.  On GB300 the FP64 pipe issues at 1/64 of the FP32 rate, so a handful
// of FP32 operations per FP64-class operation is the faster way to carry
// FP64-level accuracy through the stencil arithmetic.
//
// Building blocks (error-free transformations, exact in IEEE FP32 with FMA):
//   TwoSum      -- Knuth, TAOCP vol. 2, Section 4.2.2 (6 operations)
//   FastTwoSum  -- Dekker, Numer. Math. 18 (1971), requires |a| >= |b| (3 ops)
//   TwoProd     -- product and its exact error with one FMA (2 ops)
// Double-word operations follow Joldes, Muller and Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic", ACM TOMS
// 44 (2017): AccurateDWPlusDW (their Algorithm 6, relative error below
// 3u^2/(1 - 4u), u = 2^-24) and DWTimesDW with FMA (their Algorithm 12).
// Division: the FP32 quotient of the heads refined by two corrections with
// the double-word remainder.
//
// Conversions from and to FP64 run on the integer pipes (no FP64 instruction):
// the double is split into its correctly rounded FP32 head and the exactly
// computed remainder, rounded to FP32.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

namespace osb {

// Rounded FP32 operations that the compiler may not fuse into FMAs: the
// error-free transformations below rely on every sum and product being
// rounded on its own.
__host__ __device__ __forceinline__ float fadd_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
__host__ __device__ __forceinline__ float fsub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
__host__ __device__ __forceinline__ float fmul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}

__host__ __device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = fadd_rn(a, b);
    const float ap = fsub_rn(s, b);
    const float bp = fsub_rn(s, ap);
    e = fadd_rn(fsub_rn(a, ap), fsub_rn(b, bp));
}
__host__ __device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = fadd_rn(a, b);
    e = fsub_rn(b, fsub_rn(s, a));
}
__host__ __device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

__host__ __device__ __forceinline__ uint64_t dbl_bits(double d) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t u;
    memcpy(&u, &d, 8);
    return u;
#endif
}
__host__ __device__ __forceinline__ double bits_dbl(uint64_t u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double d;
    memcpy(&d, &u, 8);
    return d;
#endif
}
__host__ __device__ __forceinline__ float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}

// Exact float -> double on the integer pipes (normal floats and zero; values
// below the smallest normal float become signed zero; infinities and NaNs
// stay infinite / NaN).
__host__ __device__ __forceinline__ double dd_f2d(float f) {
#ifdef __CUDA_ARCH__
    const uint32_t b = __float_as_uint(f);
#else
    uint32_t b;
    memcpy(&b, &f, 4);
#endif
    const uint32_t sign = b & 0x80000000u, a = b & 0x7fffffffu;
    uint32_t hi = (a >> 3) + (a >= 0x7f800000u ? 0x70000000u : 0x38000000u);
    uint32_t lo = b << 29;
    const bool tiny = a < 0x00800000u;
    hi = tiny ? 0u : hi;
    lo = tiny ? 0u : lo;
    return bits_dbl(((uint64_t)(sign | hi) << 32) | lo);
}

struct __align__(8) dd {
    float hi, lo;

    __host__ __device__ constexpr dd() : hi(0.f), lo(0.f) {}
    __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
    // from double: head = x rounded to FP32 (nearest even), tail = the exact
    // remainder x - head rounded to FP32.  Integer operations only.
    __host__ __device__ explicit dd(double x) {
        const uint64_t b = dbl_bits(x);
        const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
        const int e = (int)((b >> 52) & 0x7ff);
        const uint64_t m = (b & 0xfffffffffffffull) | (1ull << 52);  // 53-bit significand
        if (e == 0x7ff) {  // infinity or NaN
            hi = u2f(sign | 0x7f800000u | ((b & 0xfffffffffffffull) ? 0x400000u : 0u));
            lo = 0.f;
            return;
        }
        const int fe = e - 1023 + 127;  // FP32 exponent field of the head
        if (e == 0 || fe <= 0) {        // zero, or below the smallest normal float
            hi = u2f(sign);
            lo = 0.f;
            return;
        }
        if (fe >= 0xff) {  // overflows FP32
            hi = u2f(sign | 0x7f800000u);
            lo = 0.f;
            return;
        }
        // head: top 24 bits of the significand, rounded to nearest even
        const uint64_t top = m >> 29, rest = m & 0x1fffffffull;
        const uint64_t inc = (rest > 0x10000000ull || (rest == 0x10000000ull && (top & 1))) ? 1 : 0;
        const uint64_t mh = top + inc;  // 24 or 25 bits
        const uint32_t hbits = ((uint32_t)fe << 23) + (uint32_t)(mh - (1ull << 23));  // carry into exponent is fine
        hi = u2f(sign | hbits);
        if (hbits >= 0x7f800000u) {  // rounded up to infinity
            lo = 0.f;
            return;
        }
        // tail: x - head = (rest - inc * 2^29) * 2^(e - 1075), |.| <= 2^28 units
        const int32_t r = (int32_t)rest - (int32_t)(inc << 29);
        // r * 2^(e-1075) as a float: convert r exactly-ish (|r| < 2^29: rounded to
        // 24 bits by the conversion) and scale by a power of two built from bits
        const float rf = (float)r;
        const int pe = e - 1075 + 127;  // exponent field of 2^(e-1075)
        float scale;
        if (pe >= 1) {
            scale = u2f((uint32_t)pe << 23);
        } else {
            // 2^(e-1075) is below the normal FP32 range: fold part of it into r
            scale = u2f((uint32_t)(pe + 60) << 23) * u2f((uint32_t)(127 - 60) << 23);
        }
        const float t = rf * scale;
        lo = sign ? -t : t;
    }
    // to double: head and tail widened exactly, one FP64 addition
    __host__ __device__ explicit operator double() const { return dd_f2d(hi) + dd_f2d(lo); }
};

__host__ __device__ __forceinline__ dd dd_norm(float s, float e) {
    dd r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

// AccurateDWPlusDW (Joldes-Muller-Popescu Algorithm 6)
__host__ __device__ __forceinline__ dd operator+(const dd &x, const dd &y) {
    float sh, sl, th, tl, vh, vl;
    two_sum(x.hi, y.hi, sh, sl);
    two_sum(x.lo, y.lo, th, tl);
    const float c = fadd_rn(sl, th);
    fast_two_sum(sh, c, vh, vl);
    const float w = fadd_rn(tl, vl);
    return dd_norm(vh, w);
}
__host__ __device__ __forceinline__ dd operator-(const dd &x) { return dd(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ dd operator-(const dd &x, const dd &y) { return x + (-y); }

// DWTimesDW with FMA (Joldes-Muller-Popescu Algorithm 12)
__host__ __device__ __forceinline__ dd operator*(const dd &x, const dd &y) {
    float ch, cl1;
    two_prod(x.hi, y.hi, ch, cl1);
    const float tl0 = fmul_rn(x.lo, y.lo);
    const float tl1 = fmaf(x.hi, y.lo, tl0);
    const float cl2 = fmaf(x.lo, y.hi, tl1);
    return dd_norm(ch, fadd_rn(cl1, cl2));
}

__host__ __device__ __forceinline__ dd fma(const dd &a, const dd &b, const dd &c) { return a * b + c; }
// the scalar fused multiply-adds, visible beside the double-float one inside
// namespace osb
__host__ __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__host__ __device__ __forceinline__ float fma(float a, float b, float c) { return ::fmaf(a, b, c); }

// x / y: q0 = x.hi / y.hi, then two corrections with the double-word
// remainder r = x - y q:  q <- q + r.hi / y.hi.
__host__ __device__ __forceinline__ dd operator/(const dd &x, const dd &y) {
    const float q0 = x.hi / y.hi;
    const dd r = x - y * dd(q0, 0.f);
    const float q1 = r.hi / y.hi;
    const dd q = dd(q0, 0.f) + dd(q1, 0.f);
    const dd r2 = x - y * q;
    return q + dd(r2.hi / y.hi, 0.f);
}

// exact scaling by a power of two s
__host__ __device__ __forceinline__ dd dd_scale(const dd &x, float s) { return dd(fmul_rn(x.hi, s), fmul_rn(x.lo, s)); }

__host__ __device__ __forceinline__ dd &operator+=(dd &a, const dd &b) { return a = a + b; }
__host__ __device__ __forceinline__ dd &operator-=(dd &a, const dd &b) { return a = a - b; }

// sum_k w_k (f_{+k} - f_{-k}) style accumulations used by the stencils:
// terms are formed unnormalised and summed with TwoSum on the heads and plain
// sums of the tails; one normalisation at the end.
struct dd_acc {
    float s = 0.f, e = 0.f;
    // add w * (a - b)
    __host__ __device__ __forceinline__ void add_wdiff(const dd &w, const dd &a, const dd &b) {
        float dh, d1;
        two_sum(a.hi, -b.hi, dh, d1);
        const float dl = fadd_rn(d1, fsub_rn(a.lo, b.lo));
        add_prod(w, dh, dl);
    }
    // add w * (a + b)
    __host__ __device__ __forceinline__ void add_wsum(const dd &w, const dd &a, const dd &b) {
        float dh, d1;
        two_sum(a.hi, b.hi, dh, d1);
        const float dl = fadd_rn(d1, fadd_rn(a.lo, b.lo));
        add_prod(w, dh, dl);
    }
    // add w * (dh + dl)
    __host__ __device__ __forceinline__ void add_prod(const dd &w, float dh, float dl) {
        float p, pe;
        two_prod(w.hi, dh, p, pe);
        pe = fmaf(w.hi, dl, pe);
        pe = fmaf(w.lo, dh, pe);
        const float s0 = s;
        float t;
        two_sum(s0, p, s, t);
        e = fadd_rn(e, fadd_rn(t, pe));
    }
    __host__ __device__ __forceinline__ dd get() const { return dd_norm(s, e); }
};

}  // namespace osb
