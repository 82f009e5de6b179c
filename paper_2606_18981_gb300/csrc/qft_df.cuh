// qft_df.cuh -- double-float ("df") arithmetic for the complex128 pass kernel.
//
// GB300 executes FP64 at 1/64 of its FP32 rate, so a complex128 transform
// whose butterflies and twiddles run on the FP64 pipe is bound by that pipe
// at a few percent of the HBM roofline.  The df path keeps every amplitude as
// an unevaluated sum hi + lo of two FP32 numbers (about 48 significant bits)
// and runs all arithmetic on the FP32 pipe with error-free transformations:
//
//   two_sum(a, b)   s + e = a + b exactly            (Knuth; 6 FP32 adds)
//   two_prod(a, b)  p + e = a * b exactly            (p = a*b, e = fma(a, b, -p))
//   fast_two_sum    renormalisation when |s| >= |e|  (Dekker; 3 adds)
//
// Sums inside the butterfly network are left unnormalised (hi, lo) pairs;
// products and every value written to shared or global memory are
// renormalised.  The relative error of one operation is a few units of 2^-48,
// so an n-wire transform stays far inside the complex128 tolerance 1e-13 n.
//
// Range: FP32 exponents.  The transform is linear, so before the first pass a
// reduction finds the largest binary exponent of the input and the first pass
// scales the input by 2^-k (an integer exponent shift, exact) so that its
// largest component lies in [1, 2); the last pass multiplies by 2^k while it
// converts back to FP64.  Intermediates then stay below 2^(n/2 + 1) and every
// component that matters at the 2^-48 level of the largest one is a normal
// FP32 pair.
//
// Conversions between FP64 and df use integer bit manipulation only (no FP64
// instruction): the FP64 -> df split truncates the 53-bit significand into
// 24 + 29 bits (the low part rounded to 24 bits), and df -> FP64 adds the two
// significands in a 64-bit integer.  Both are __host__ __device__ so the host
// test harness can check them bit for bit against long double arithmetic.
#pragma once
#include <cstdint>
#include <cstring>
#include <cmath>
#include <cuda_runtime.h>

namespace qft {

struct dfloat {
    float hi, lo;
    __host__ __device__ constexpr dfloat() : hi(0.f), lo(0.f) {}
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dfloat(int v) : hi(static_cast<float>(v)), lo(0.f) {}
    // Nearest pair to d (host: table set-up, device: once per CTA or tile).
    __host__ __device__ explicit dfloat(double d)
        : hi(static_cast<float>(d)), lo(static_cast<float>(d - static_cast<double>(static_cast<float>(d)))) {}
};

// A complex amplitude: the high parts of the real and imaginary components in
// one FP32 pair and the low parts in another, so that a complex add or
// subtract is a packed FP32x2 two-sum (one instruction for both components).
// In memory (shared and the workspace between passes): re.hi, im.hi, re.lo,
// im.lo -- 16 bytes, the size of a complex128 amplitude.
struct __align__(16) dcomplex {
    float2 hi;  // (re.hi, im.hi)
    float2 lo;  // (re.lo, im.lo)
    __host__ __device__ dfloat re() const { return dfloat(hi.x, lo.x); }
    __host__ __device__ dfloat im() const { return dfloat(hi.y, lo.y); }
};

__host__ __device__ __forceinline__ dcomplex dc_make(dfloat re, dfloat im) {
    dcomplex r;
    r.hi = make_float2(re.hi, im.hi);
    r.lo = make_float2(re.lo, im.lo);
    return r;
}

// ------------------------------------------------------------ bit helpers

__host__ __device__ __forceinline__ uint32_t f2u(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    std::memcpy(&f, &u, 4);
    return f;
#endif
}
__host__ __device__ __forceinline__ uint64_t d2u(double d) {
#ifdef __CUDA_ARCH__
    return static_cast<uint64_t>(__double_as_longlong(d));
#else
    uint64_t u;
    std::memcpy(&u, &d, 8);
    return u;
#endif
}
__host__ __device__ __forceinline__ double u2d(uint64_t u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double(static_cast<long long>(u));
#else
    double d;
    std::memcpy(&d, &u, 8);
    return d;
#endif
}
__host__ __device__ __forceinline__ float fma_f(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fma(a, b, c);
#endif
}

// ------------------------------------------------- error-free transforms

__host__ __device__ __forceinline__ dfloat two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return dfloat(s, e);
}

__host__ __device__ __forceinline__ dfloat fast_two_sum(float s, float e) {
    const float h = s + e;
    return dfloat(h, e - (h - s));
}

__host__ __device__ __forceinline__ dfloat df_norm(dfloat a) { return fast_two_sum(a.hi, a.lo); }

// a + b and a - b, left unnormalised: the exact sum of the high parts plus the
// rounded sum of the low parts and its error term.
__host__ __device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    dfloat s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return s;
}
__host__ __device__ __forceinline__ dfloat df_sub(dfloat a, dfloat b) {
    dfloat s = two_sum(a.hi, -b.hi);
    s.lo += a.lo - b.lo;
    return s;
}
__host__ __device__ __forceinline__ dfloat df_neg(dfloat a) { return dfloat(-a.hi, -a.lo); }

// a * b (renormalised): the exact product of the high parts plus the cross terms.
__host__ __device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
    const float p = a.hi * b.hi;
    float e = fma_f(a.hi, b.hi, -p);
    e = fma_f(a.hi, b.lo, e);
    e = fma_f(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

// a.hi*b.hi - c.hi*d.hi as an exact two_sum of the exact products, plus every
// cross term: one component of a complex product (renormalised).
__host__ __device__ __forceinline__ dfloat df_dot2(dfloat a, dfloat b, dfloat c, dfloat d) {
    const float p1 = a.hi * b.hi;
    const float e1 = fma_f(a.hi, b.hi, -p1);
    const float p2 = c.hi * d.hi;
    const float e2 = fma_f(c.hi, d.hi, -p2);
    dfloat s = two_sum(p1, -p2);
    float t = s.lo + (e1 - e2);
    t = fma_f(a.hi, b.lo, t);
    t = fma_f(a.lo, b.hi, t);
    t = fma_f(-c.hi, d.lo, t);
    t = fma_f(-c.lo, d.hi, t);
    return fast_two_sum(s.hi, t);
}

#ifdef __CUDA_ARCH__
// Lane-wise FP32 pair arithmetic (add/sub.rn.f32x2, sm_100 and later): the
// same IEEE results as two scalar operations.
__device__ __forceinline__ float2 pk_add(float2 a, float2 b) {
    uint64_t pa, pb, d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(pa) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(pb) : "f"(b.x), "f"(b.y));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pa), "l"(pb));
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(d));
    return r;
}
__device__ __forceinline__ float2 pk_sub(float2 a, float2 b) {
    uint64_t pa, pb, d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(pa) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(pb) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pa), "l"(pb));
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(d));
    return r;
}
#endif

// a + b: df_add on both components -- on the device as one packed two-sum
// (8 FP32x2 instructions for the complex add, the same values lane by lane).
__host__ __device__ __forceinline__ dcomplex dc_add(dcomplex a, dcomplex b) {
#ifdef __CUDA_ARCH__
    dcomplex r;
    const float2 s = pk_add(a.hi, b.hi);
    const float2 bb = pk_sub(s, a.hi);
    const float2 e = pk_add(pk_sub(a.hi, pk_sub(s, bb)), pk_sub(b.hi, bb));
    r.hi = s;
    r.lo = pk_add(pk_add(a.lo, b.lo), e);
    return r;
#else
    return dc_make(df_add(a.re(), b.re()), df_add(a.im(), b.im()));
#endif
}
// a - b: df_sub on both components, packed on the device
__host__ __device__ __forceinline__ dcomplex dc_sub(dcomplex a, dcomplex b) {
#ifdef __CUDA_ARCH__
    dcomplex r;
    const float2 s = pk_sub(a.hi, b.hi);
    const float2 bb = pk_sub(s, a.hi);
    const float2 e = pk_sub(pk_sub(a.hi, pk_sub(s, bb)), pk_add(b.hi, bb));
    r.hi = s;
    r.lo = pk_add(pk_sub(a.lo, b.lo), e);
    return r;
#else
    return dc_make(df_sub(a.re(), b.re()), df_sub(a.im(), b.im()));
#endif
}
// (ar + i ai)(br + i bi) = (ar br - ai bi) + i (ar bi + ai br)
__host__ __device__ __forceinline__ dcomplex dc_mul(dcomplex a, dcomplex b) {
    const dfloat ar = a.re(), ai = a.im(), br = b.re(), bi = b.im();
    return dc_make(df_dot2(ar, br, ai, bi), df_dot2(ar, bi, df_neg(ai), br));
}
// renormalise both components (fast two-sum), packed on the device
__host__ __device__ __forceinline__ dcomplex dc_norm(dcomplex a) {
#ifdef __CUDA_ARCH__
    dcomplex r;
    r.hi = pk_add(a.hi, a.lo);
    r.lo = pk_sub(a.lo, pk_sub(r.hi, a.hi));
    return r;
#else
    return dc_make(df_norm(a.re()), df_norm(a.im()));
#endif
}

// ------------------------------------------- twiddles without FP64 work

// (cos, sin) of 2 pi m / 2^40 as double-float pairs, for |m| <= 2^37 (at most
// an eighth of a turn), with FP32 operations only: m = 2^30 k + r with k the
// nearest integer to m / 2^30 (|k| <= 128) and |r| <= 2^29; the angle 2 pi k
// / 2^10 comes from a table (tab[|k|] = (cos, sin) of 2 pi |k| / 2^10, k >= 0;
// sin is odd), the rest t = 2 pi r / 2^40 (|t| < 3.1e-3) from the Taylor
// series at 0 -- cos t = 1 - t^2/2 + t^4/24 and sin t = t (1 - t^2/6 +
// t^4/120), the omitted terms below 2^-58 -- with t^2 as a pair and the
// quartic terms in FP32 (they are below 4e-12).  The two rotations are then
// combined as base + base (cos t - 1 + i sin t), so that the complex
// product's rounding error scales with |t| < 3.1e-3.  Error a few units of
// 2^-48.
__host__ __device__ __forceinline__ dcomplex df_turns40(int64_t m, const dcomplex* tab) {
    const int k = static_cast<int>((m + (int64_t(1) << 29)) >> 30);
    const int64_t r = m - (static_cast<int64_t>(k) << 30);
    // 2 pi / 2^40 as a pair
    const dfloat c40(0x1.921fb6p-38f, -0x1.777a5cp-63f);
    const float rh = static_cast<float>(r);
    const dfloat rr(rh, static_cast<float>(r - static_cast<int64_t>(rh)));
    const dfloat t = df_mul(rr, c40);
    const dfloat t2 = df_mul(t, t);
    const float q = t2.hi * t2.hi;
    // 1 - t^2/6 + t^4/120 and 1 - t^2/2 + t^4/24
    const dfloat sixth(0x1.555556p-3f, -0x1.555556p-28f);
    const dfloat b = df_mul(t2, sixth);
    dfloat ps = two_sum(1.0f, -b.hi);
    ps.lo += q * (1.0f / 120.0f) - b.lo;
    const dfloat sn = df_mul(t, fast_two_sum(ps.hi, ps.lo));
    // cos t - 1 = -t^2/2 + t^4/24 (|.| < 5e-6)
    const dfloat cm1 = fast_two_sum(-0.5f * t2.hi, q * (1.0f / 24.0f) - 0.5f * t2.lo);
    dcomplex base = tab[k < 0 ? -k : k];
    if (k < 0) base = dc_make(base.re(), df_neg(base.im()));
    // base (cos t + i sin t) = base + base (cos t - 1 + i sin t): the product's
    // rounding error is relative to its own small size
    return dc_norm(dc_add(base, dc_mul(base, dc_make(cm1, sn))));
}

// ------------------------------------------------ FP64 <-> df conversions

// FP64 value d times 2^-k as a df pair, by integer operations only.  The
// significand is split into its top 24 bits (hi, exact) and the remaining 29
// bits (lo, rounded to 24 bits).  Zero and subnormal FP64 inputs, and values
// whose scaled magnitude is below 2^-126, become 0, and the low part of
// values below 2^-74 is dropped; with k
// chosen so that the largest component lies in [1, 2), both only touch
// components 2^-74 below the largest, far under the df precision.  k must
// keep the scaled largest component below 2^128 (it does: it is at most 2).
__host__ __device__ __forceinline__ dfloat df_from_double_shift(double d, int k) {
    const uint64_t b = d2u(d);
    const uint32_t hw = static_cast<uint32_t>(b >> 32), lw = static_cast<uint32_t>(b);
    const int Eraw = static_cast<int>((hw >> 20) & 0x7FFu);
    const int E = Eraw - k;  // biased FP64 exponent of d * 2^-k
    const uint32_t sign = hw & 0x80000000u;
    dfloat r;
    if (Eraw != 0 && E >= 897) {  // d normal, and d * 2^-k normal as FP32 (biased exponent E - 896 >= 1)
        r.hi = u2f(sign | (static_cast<uint32_t>(E - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
        const uint32_t m = lw & 0x1FFFFFFFu;                  // low 29 significand bits
        const float scale = E >= 949 ? u2f(static_cast<uint32_t>(E - 948) << 23) : 0.f;  // 2^(E - 1075)
        r.lo = u2f(f2u(static_cast<float>(m) * scale) | sign);
    } else {
        r.hi = 0.f;
        r.lo = 0.f;
    }
    return r;
}

// (a.hi + a.lo) * 2^k as FP64, for any pair whose high part dominates.  The
// two significands are added in a 64-bit integer (lo's bits below the 53-bit
// significand are truncated); a result whose exponent leaves the FP64 normal
// range becomes 0 (underflow) or infinity.
__host__ __device__ __forceinline__ double df_to_double_shift_general(dfloat a, int k) {
    const uint32_t hb = f2u(a.hi);
    const int Eh = static_cast<int>((hb >> 23) & 0xFFu);
    if (Eh == 0) return 0.0;  // hi is zero (or subnormal, below any value that matters)
    const uint64_t sh = static_cast<uint64_t>(hb >> 31);
    uint64_t M = static_cast<uint64_t>((hb & 0x7FFFFFu) | 0x800000u) << 29;  // 53-bit significand, ulp 2^(Eh-179)
    const uint32_t lb = f2u(a.lo);
    const int El = static_cast<int>((lb >> 23) & 0xFFu);
    if (El != 0) {
        const uint64_t Ml = (lb & 0x7FFFFFu) | 0x800000u;
        const int sa = El - Eh + 29;  // lo = Ml * 2^(El-150) = Ml * 2^sa ulps
        uint64_t add = 0;
        if (sa >= 0) add = sa < 40 ? (Ml << sa) : 0;
        else if (sa > -25) add = Ml >> (-sa);
        if ((lb >> 31) == sh) M += add;
        else M -= add;
    }
    int Ed = Eh + 896 + k;  // biased FP64 exponent
    if (M >= (uint64_t(1) << 53)) {
        M >>= 1;
        ++Ed;
    } else if (M < (uint64_t(1) << 52)) {
        M <<= 1;
        --Ed;
    }
    if (Ed <= 0) return sh ? -0.0 : 0.0;
    if (Ed >= 2047) return u2d((sh << 63) | (uint64_t(0x7FF) << 52));
    return u2d((sh << 63) | (static_cast<uint64_t>(Ed) << 52) | (M & ((uint64_t(1) << 52) - 1)));
}

// The same conversion, bit for bit, written for the pairs the kernel stores
// (normalised by fast_two_sum, so |lo| <= ulp(hi) / 2): lo's significand then
// sits at most 5 bits above the 29 bits below hi's, its aligned value is
// below 2^29 and fits a 32-bit word, and the 53-bit sum lies in
// (2^52 - 2^29, 2^53), so it needs at most one left shift.  Every step is a
// select on 32-bit words plus one 64-bit add; other pairs take the general
// path above.
__host__ __device__ __forceinline__ double df_to_double_shift(dfloat a, int k) {
    const uint32_t hb = f2u(a.hi), lb = f2u(a.lo);
    const int Eh = static_cast<int>((hb >> 23) & 0xFFu);
    const int El = static_cast<int>((lb >> 23) & 0xFFu);
    const int sa = El - Eh + 29;
    if (sa > 5) return df_to_double_shift_general(a, k);
    const uint32_t Ml = El ? ((lb & 0x7FFFFFu) | 0x800000u) : 0u;
    const int rs = -sa < 31 ? -sa : 31;
    const uint32_t add = sa >= 0 ? (Ml << sa) : (Ml >> rs);
    const uint32_t sh = hb >> 31;
    const int64_t sadd = ((lb >> 31) == sh) ? static_cast<int64_t>(add) : -static_cast<int64_t>(add);
    uint64_t M = (static_cast<uint64_t>((hb & 0x7FFFFFu) | 0x800000u) << 29) + static_cast<uint64_t>(sadd);
    const bool low = M < (uint64_t(1) << 52);
    M = low ? (M << 1) : M;
    const int Ed = Eh + 896 + k - (low ? 1 : 0);
    const uint32_t mhi = static_cast<uint32_t>(M >> 32) & 0xFFFFFu;
    uint32_t whi = (sh << 31) | (static_cast<uint32_t>(Ed) << 20) | mhi;
    uint32_t wlo = static_cast<uint32_t>(M);
    const bool zero = Ed <= 0;
    const bool inf = Ed >= 2047;
    whi = zero ? (sh << 31) : (inf ? ((sh << 31) | 0x7FF00000u) : whi);
    wlo = (zero || inf) ? 0u : wlo;
    whi = Eh == 0 ? 0u : whi;
    wlo = Eh == 0 ? 0u : wlo;
    return u2d((static_cast<uint64_t>(whi) << 32) | wlo);
}

}  // namespace qft
