// Host check of the phase-estimation sweep's complex64 phase evaluation
// (qft_phase64.cuh), run on the CPU from the kernel's own __host__ __device__
// functions against long double sin/cos:
//   * sincospi_quarter on a dense grid of [-1/4, 1/4] (and its endpoints):
//     within 1.5 units of 2^-24 of sin(pi x), cos(pi x);
//   * phase64_f32 on random and edge-case 64-bit phases: within 2 units of
//     2^-24 of cos, sin(2 pi phase / 2^64), the quarter-turn reduction exact
//     (sin^2 + cos^2 = 1 to FP32 rounding, and the signs of each quadrant).
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>

#include "qft_phase64.cuh"

static const long double kPi = 3.141592653589793238462643383279502884L;

int main() {
    int fails = 0;
    const long double tol_q = 1.5L * std::ldexp(1.0L, -24), tol_p = 2.0L * std::ldexp(1.0L, -24);
    long double worst_s = 0, worst_c = 0;
    const int G = 1 << 21;
    for (int i = -G; i <= G; ++i) {
        const float x = static_cast<float>(0.25L * i / G);
        float s, c;
        qft::sincospi_quarter(x, s, c);
        const long double es = std::fabs(s - std::sin(kPi * x)), ec = std::fabs(c - std::cos(kPi * x));
        if (es > worst_s) worst_s = es;
        if (ec > worst_c) worst_c = ec;
    }
    if (worst_s > tol_q || worst_c > tol_q) {
        std::printf("FAIL sincospi_quarter: max |err| sin %.3Le cos %.3Le > %.3Le\n", worst_s, worst_c, tol_q);
        ++fails;
    }
    std::printf("sincospi_quarter: max |err| sin %.3Le cos %.3Le (bound %.3Le)\n", worst_s, worst_c, tol_q);

    std::mt19937_64 rng(7);
    long double worst = 0;
    auto check = [&](uint64_t ph) {
        float c, s;
        qft::phase64_f32(ph, c, s);
        const long double turns = static_cast<long double>(ph) / 18446744073709551616.0L;  // exact
        const long double ec = std::fabs(c - std::cos(2 * kPi * turns)), es = std::fabs(s - std::sin(2 * kPi * turns));
        const long double e = ec > es ? ec : es;
        if (e > worst) worst = e;
        if (e > tol_p) {
            if (fails < 10) std::printf("FAIL phase64_f32(%llu): err %.3Le\n", static_cast<unsigned long long>(ph), e);
            ++fails;
        }
    };
    for (int i = 0; i < 2000000; ++i) check(rng());
    const uint64_t Q = uint64_t(1) << 62;
    const uint64_t edges[] = {0, 1, Q - 1, Q, Q + 1, 2 * Q - 1, 2 * Q, 2 * Q + 1, 3 * Q, 3 * Q + 1,
                              ~uint64_t(0), Q / 2, Q / 2 - 1, Q / 2 + 1, 3 * Q + Q / 2, 7 * (Q / 4)};
    for (uint64_t e : edges) check(e);
    // exact quarter turns give exact values
    for (int q = 0; q < 4; ++q) {
        float c, s;
        qft::phase64_f32(uint64_t(q) * Q, c, s);
        const float wc[4] = {1, 0, -1, 0}, ws[4] = {0, 1, 0, -1};
        if (c != wc[q] || s != ws[q]) {
            std::printf("FAIL quarter turn %d: (%g, %g)\n", q, c, s);
            ++fails;
        }
    }
    std::printf("phase64_f32: max |err| %.3Le (bound %.3Le)\n", worst, tol_p);
    if (fails) {
        std::printf("%d failures\n", fails);
        return 1;
    }
    std::printf("ALL OK\n");
    return 0;
}
