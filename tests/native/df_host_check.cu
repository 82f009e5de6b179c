// Host-side check of the double-float arithmetic and FP64 <-> df conversions
// of the complex128 pass kernel (paper_2606_18981_gb300/csrc/qft_df.cuh):
// the same __host__ __device__ functions the kernel runs, evaluated on the
// CPU against long double arithmetic.  Prints one line per check and
// "ALL OK" when every bound holds; exit status 1 otherwise.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <random>

#include "qft_df.cuh"

using qft::dfloat;

static int g_fail = 0;
static void check(bool ok, const char* what, double worst, double bound) {
    std::printf("%-44s worst %.3e bound %.3e %s\n", what, worst, bound, ok ? "ok" : "FAIL");
    if (!ok) ++g_fail;
}

static long double val(dfloat a) { return (long double)a.hi + (long double)a.lo; }

int main() {
    std::mt19937_64 rng(20261204);
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    std::uniform_int_distribution<int> ex(-60, 60);

    // 1. FP64 -> df split with exponent shift k: relative error <= 2^-46 for
    //    scaled magnitudes >= 2^-74; below that the low part is dropped
    //    (absolute error < 2^-23 of the value, i.e. < 2^-97).
    {
        double worst = 0, worst_small = 0;
        for (int i = 0; i < 200000; ++i) {
            const int k = ex(rng) * 10;            // shifts of up to +-600
            const double d = std::ldexp(u(rng), ex(rng) + k);
            const dfloat a = qft::df_from_double_shift(d, k);
            const long double ref = std::ldexp((long double)d, -k);
            if (ref == 0) continue;
            const double err = (double)(std::fabs(val(a) - ref) / std::fabs(ref));
            if (std::fabs(ref) >= std::ldexp(1.0L, -74)) worst = std::fmax(worst, err);
            else worst_small = std::fmax(worst_small, err);
        }
        check(worst <= std::ldexp(1.0, -46), "from_double_shift relative error", worst, std::ldexp(1.0, -46));
        check(worst_small <= std::ldexp(1.0, -23), "from_double_shift below 2^-74", worst_small, std::ldexp(1.0, -23));
    }
    // 2. the split's high part is exact: hi is d * 2^-k truncated to 24 bits
    {
        int bad = 0;
        for (int i = 0; i < 100000; ++i) {
            const double d = std::ldexp(u(rng), ex(rng));
            const dfloat a = qft::df_from_double_shift(d, 0);
            if (std::fabs((double)a.hi) > std::fabs(d) || std::fabs(d - (double)a.hi) >= std::ldexp(std::fabs(d), -22)) ++bad;
        }
        check(bad == 0, "from_double_shift high part is truncation", bad, 0);
    }
    // 3. zero, subnormal and values scaled below 2^-126 become 0
    {
        const double cases[] = {0.0, -0.0, 4.9e-324, -2.2e-310};
        bool ok = true;
        for (double d : cases) {
            const dfloat a = qft::df_from_double_shift(d, -1022);
            ok = ok && a.hi == 0.f && a.lo == 0.f;
        }
        const dfloat b = qft::df_from_double_shift(std::ldexp(1.0, -200), 0);
        ok = ok && b.hi == 0.f && b.lo == 0.f;
        check(ok, "zero / subnormal / underflow -> 0", ok ? 0 : 1, 0);
    }
    // 4. df -> FP64 with exponent shift: within one FP64 ulp (truncation of lo)
    {
        double worst = 0;
        for (int i = 0; i < 200000; ++i) {
            const int k = ex(rng) * 10;
            const float h = (float)std::ldexp(u(rng), ex(rng) / 2);
            const float l = (float)(std::ldexp(u(rng), -25) * h);
            const dfloat a = qft::fast_two_sum(h, l);
            const double r = qft::df_to_double_shift(a, k);
            const long double ref = std::ldexp(val(a), k);
            if (ref == 0) continue;
            const double err = (double)(std::fabs((long double)r - ref) / std::fabs(ref));
            if (err > worst) worst = err;
        }
        check(worst <= std::ldexp(1.0, -52), "to_double_shift relative error", worst, std::ldexp(1.0, -52));
    }
    // 4b. the kernel's conversion equals the general one bit for bit: pairs
    //     normalised by fast_two_sum (random, powers of two with a negative low
    //     part, zero / subnormal low parts, shifts that overflow or underflow)
    //     and pairs that are not normalised (the general path)
    {
        long bad = 0, total = 0;
        auto same = [&](dfloat a, int k) {
            const double r = qft::df_to_double_shift(a, k), g = qft::df_to_double_shift_general(a, k);
            ++total;
            if (qft::d2u(r) != qft::d2u(g)) ++bad;
        };
        std::uniform_int_distribution<int> kk(-1200, 1200);
        for (int i = 0; i < 400000; ++i) {
            const int k = (i & 3) ? ex(rng) * 10 : kk(rng);
            const float h = (float)std::ldexp(u(rng), ex(rng) * 2);
            const float l = (float)(std::ldexp(u(rng), -(i % 40)) * h);
            same(qft::fast_two_sum(h, l), k);                       // normalised
            same(dfloat(h, l), k);                                  // as it comes
            const float p2 = std::ldexp(1.0f, ex(rng));
            same(qft::fast_two_sum(p2, -std::ldexp(p2, -25 - (i % 8))), k);  // borrow below a power of two
            same(dfloat(h, 0.f), k);
            same(dfloat(h, std::ldexp(1.0f, -140)), k);             // subnormal low part
            same(dfloat(0.f, l), k);
        }
        check(bad == 0, "to_double_shift equals the general form", (double)bad, 0);
        std::printf("  (%ld pairs)\n", total);
    }
    // 4c. df_turns40: (cos, sin) of 2 pi m / 2^40 for |m| <= 2^37 from the
    //     129-entry table, against long double, relative to |z| = 1
    {
        qft::dcomplex tab[129];
        for (int k = 0; k <= 128; ++k) {
            const long double a = 2.0L * 3.14159265358979323846264338327950288L * k / 1024.0L;
            const double c = (double)std::cos(a), s = (double)std::sin(a);
            tab[k] = qft::dc_make(dfloat(c), dfloat(s));
        }
        std::uniform_int_distribution<int64_t> um(-(int64_t(1) << 37), int64_t(1) << 37);
        double worst = 0;
        auto one = [&](int64_t m) {
            const qft::dcomplex z = qft::df_turns40(m, tab);
            const long double a = 2.0L * 3.14159265358979323846264338327950288L * (long double)m / 1099511627776.0L;
            const long double ec = std::fabs(val(z.re()) - std::cos(a)), es = std::fabs(val(z.im()) - std::sin(a));
            worst = std::fmax(worst, (double)std::fmax(ec, es));
        };
        for (int i = 0; i < 400000; ++i) one(um(rng));
        const int64_t edges[] = {0, 1, -1, int64_t(1) << 37, -(int64_t(1) << 37), (int64_t(1) << 29), -(int64_t(1) << 29),
                                 (int64_t(1) << 29) - 1, (int64_t(3) << 29), (int64_t(3) << 29) - 1, 12345678901LL};
        for (int64_t m : edges) one(m);
        check(worst <= std::ldexp(1.0, -47), "turns40 (cos, sin) error", worst, std::ldexp(1.0, -47));
    }
    // 5. round trip FP64 -> df -> FP64
    {
        double worst = 0;
        for (int i = 0; i < 200000; ++i) {
            const int k = ex(rng) * 10;
            const double d = std::ldexp(u(rng), ex(rng) + k);
            const double r = qft::df_to_double_shift(qft::df_norm(qft::df_from_double_shift(d, k)), k);
            if (std::fabs(d) < std::ldexp(1.0, k - 74)) continue;
            const double err = std::fabs(r - d) / std::fabs(d);
            if (err > worst) worst = err;
        }
        check(worst <= std::ldexp(1.0, -46), "round trip relative error", worst, std::ldexp(1.0, -46));
    }
    // 6. df_add / df_sub (unnormalised): error <= 2^-46 (|a| + |b|)
    // 7. df_dot2: a b - c d with error <= 2^-45 (|a b| + |c d|)
    {
        double wa = 0, wd = 0, wm = 0;
        for (int i = 0; i < 200000; ++i) {
            auto rnd = [&]() {
                const double d = std::ldexp(u(rng), ex(rng) / 4);
                return qft::df_norm(qft::df_from_double_shift(d, 0));
            };
            const dfloat a = rnd(), b = rnd(), c = rnd(), d = rnd();
            const long double s = val(a) + val(b), t = val(a) - val(b);
            const long double scale = std::fabs(val(a)) + std::fabs(val(b));
            wa = std::fmax(wa, (double)(std::fabs(val(qft::df_add(a, b)) - s) / scale));
            wa = std::fmax(wa, (double)(std::fabs(val(qft::df_sub(a, b)) - t) / scale));
            const long double p = val(a) * val(b) - val(c) * val(d);
            const long double ps = std::fabs(val(a) * val(b)) + std::fabs(val(c) * val(d));
            wd = std::fmax(wd, (double)(std::fabs(val(qft::df_dot2(a, b, c, d)) - p) / ps));
            wm = std::fmax(wm, (double)(std::fabs(val(qft::df_mul(a, b)) - val(a) * val(b)) / std::fabs(val(a) * val(b))));
        }
        check(wa <= std::ldexp(1.0, -46), "df_add / df_sub error / (|a|+|b|)", wa, std::ldexp(1.0, -46));
        check(wd <= std::ldexp(1.0, -45), "df_dot2 error / (|ab|+|cd|)", wd, std::ldexp(1.0, -45));
        check(wm <= std::ldexp(1.0, -45), "df_mul relative error", wm, std::ldexp(1.0, -45));
    }
    // 8. dc_mul (complex product v w, each component a df_dot2p): error of a
    //    component <= 2^-45 times the sum of its two products' magnitudes
    {
        double wc = 0;
        for (int i = 0; i < 200000; ++i) {
            auto rnd = [&]() {
                const double d = std::ldexp(u(rng), ex(rng) / 4);
                return qft::df_norm(qft::df_from_double_shift(d, 0));
            };
            const qft::dcomplex v = qft::dc_make(rnd(), rnd()), w = qft::dc_make(rnd(), rnd());
            const long double vr = val(v.re()), vi = val(v.im()), wr = val(w.re()), wi = val(w.im());
            const qft::dcomplex z = qft::dc_mul(v, w);
            const long double re = wr * vr - wi * vi, im = wr * vi + wi * vr;
            const long double sre = std::fabs(wr * vr) + std::fabs(wi * vi), sim = std::fabs(wr * vi) + std::fabs(wi * vr);
            wc = std::fmax(wc, (double)(std::fabs(val(z.re()) - re) / sre));
            wc = std::fmax(wc, (double)(std::fabs(val(z.im()) - im) / sim));
        }
        check(wc <= std::ldexp(1.0, -45), "dc_mul component error / (sum |products|)", wc, std::ldexp(1.0, -45));
    }
    std::printf(g_fail ? "FAILED %d\n" : "ALL OK\n", g_fail);
    return g_fail ? 1 : 0;
}
