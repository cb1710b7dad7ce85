// Host check of the double-float arithmetic (dd.cuh) against long double:
// conversions from double, the accurate sum, the product, the quotient and
// the stencil accumulator, on random operands over wide exponent ranges and
// near-cancelling pairs.  Prints the worst relative error of each in units of
// u^2 = 2^-48 and fails when a bound is exceeded.  The stencil accumulator
// forms differences of heads exactly and of tails in FP32, so its error is
// bounded relative to the sum of the operand magnitudes (the size of the
// rounding already present in double-float operands), not to the result.
#include <cmath>
#include <cstdio>
#include <random>

#include "dd.cuh"

using osb::dd;
typedef long double ld;

static ld val(const dd &a) { return (ld)a.hi + (ld)a.lo; }
static const ld U2 = std::ldexp((ld)1, -48);

int main() {
    std::mt19937_64 rng(7);
    std::uniform_real_distribution<double> uni(-1.0, 1.0);
    std::uniform_int_distribution<int> ex(-30, 30);
    auto rnd_double = [&]() { return std::ldexp(uni(rng), ex(rng)); };
    auto rnd_dd = [&]() { return dd(rnd_double()); };
    int bad = 0;
    ld worst_conv = 0, worst_add = 0, worst_mul = 0, worst_div = 0, worst_acc = 0;
    for (int it = 0; it < 2000000; ++it) {
        const double x = rnd_double();
        const dd a(x);
        if (a.hi != (float)x) ++bad;  // head is x rounded to nearest float
        const ld ec = std::fabs(val(a) - (ld)x) / std::fabs((ld)x);
        worst_conv = std::max(worst_conv, ec / U2);
        if (std::fabs((ld)(double)a - val(a)) > std::fabs(val(a)) * std::ldexp((ld)1, -53)) ++bad;

        dd b = rnd_dd(), c = rnd_dd();
        if (it % 3 == 0) b = dd(-(double)c * (1.0 + std::ldexp(uni(rng), -20)));  // near cancellation
        const ld s = val(b) + val(c);
        if (s != 0) worst_add = std::max(worst_add, std::fabs(val(b + c) - s) / std::fabs(s) / U2);
        const ld p = val(b) * val(c);
        if (p != 0) worst_mul = std::max(worst_mul, std::fabs(val(b * c) - p) / std::fabs(p) / U2);
        if (val(c) != 0) {
            const ld q = val(b) / val(c);
            worst_div = std::max(worst_div, std::fabs(val(b / c) - q) / std::fabs(q) / U2);
        }
        // stencil accumulator: sum_k w_k (f+k - f-k) + sum_k w'_k (g+k + g-k)
        osb::dd_acc acc;
        ld ex_sum = 0, mag = 0;
        for (int k = 0; k < 4; ++k) {
            const dd w = rnd_dd(), f1 = rnd_dd();
            const dd f2 = (k % 2) ? dd((double)val(f1) * (1.0 + std::ldexp(uni(rng), -12))) : rnd_dd();
            acc.add_wdiff(w, f1, f2);
            ex_sum += val(w) * (val(f1) - val(f2));
            mag += std::fabs(val(w)) * (std::fabs(val(f1)) + std::fabs(val(f2)));
            const dd g1 = rnd_dd(), g2 = rnd_dd();
            acc.add_wsum(w, g1, g2);
            ex_sum += val(w) * (val(g1) + val(g2));
            mag += std::fabs(val(w)) * (std::fabs(val(g1)) + std::fabs(val(g2)));
        }
        worst_acc = std::max(worst_acc, std::fabs(val(acc.get()) - ex_sum) / mag / U2);
    }
    printf("worst relative error / 2^-48: conversion %.3Lf add %.3Lf mul %.3Lf div %.3Lf stencil-acc %.3Lf; bad %d\n",
           worst_conv, worst_add, worst_mul, worst_div, worst_acc, bad);
    const bool ok = bad == 0 && worst_conv <= 1.0 && worst_add <= 3.0 && worst_mul <= 5.0 && worst_div <= 16.0 &&
                    worst_acc <= 16.0;
    return ok ? 0 : 1;
}
