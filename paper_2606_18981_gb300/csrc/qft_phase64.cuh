// qft_phase64.cuh -- exp(2 pi i phase / 2^64) for 64-bit fixed-point phases
// (one turn = 2^64), as the phase-estimation sweep uses them (the sum of the
// controlled evolutions' phases, exact mod 2^64).  Host and device, so that
// the host checks run the same code.
#pragma once

#include <cmath>
#include <cstdint>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace qft {

// sin(pi x) and cos(pi x) for |x| <= 1/4 in FP32 from their Taylor series at
// 0 (t = pi x, |t| <= pi/4; the first omitted terms, t^11/11! and t^12/12!,
// are below 2e-9 and 2e-10), by Horner's rule: within 1.5 units of 2^-24 of
// the exact values over the whole interval.  No range reduction: the caller
// has reduced the phase exactly in integers.
__host__ __device__ inline void sincospi_quarter(float x, float& s, float& c) {
    const float t = x * 3.14159265358979f;
    const float t2 = t * t;
    float ps = fmaf(t2, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = fmaf(ps, t2, 1.0f / 120.0f);
    ps = fmaf(ps, t2, -1.0f / 6.0f);
    s = fmaf(ps * t2, t, t);
    float pc = fmaf(t2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    pc = fmaf(pc, t2, -1.0f / 720.0f);
    pc = fmaf(pc, t2, 1.0f / 24.0f);
    pc = fmaf(pc, t2, -0.5f);
    c = fmaf(pc, t2, 1.0f);
}

// The phase as the nearest quarter turn q4 (exact, in integers) and the rest,
// rem = phase - q4 2^62 with |rem| <= 2^61, i.e. |rem / 2^63| <= 1/4 half-turn.
__host__ __device__ inline uint64_t phase64_quarter(uint64_t phase, int64_t& rem) {
    const uint64_t q4 = (phase + (uint64_t(1) << 61)) >> 62;  // 0..4
    rem = static_cast<int64_t>(phase - (q4 << 62));
    return q4;
}

// (c, s) = (cos, sin) of q4 quarter turns plus the angle whose (cos, sin) are
// (cs, sn): (cs, sn), (-sn, cs), (-cs, -sn), (sn, -cs) for q4 mod 4 = 0..3,
// written as selects (a switch on a per-thread quarter made the warps branch).
template <typename T>
__host__ __device__ inline void rotate_quarters(uint64_t q4, T cs, T sn, T& c, T& s) {
    const unsigned q = static_cast<unsigned>(q4 & 3u);
    const T tc = (q & 1u) ? sn : cs;
    const T ts = (q & 1u) ? cs : sn;
    c = ((q + 1u) & 2u) ? -tc : tc;
    s = (q & 2u) ? -ts : ts;
}

// complex64: exp(2 pi i phase / 2^64) with the rest of the reduction taken
// from its top 32 bits, rounded (the dropped part is below 2^-32 of pi, far
// under FP32's resolution here).
__host__ __device__ inline void phase64_f32(uint64_t phase, float& c, float& s) {
    int64_t rem;
    const uint64_t q4 = phase64_quarter(phase, rem);
    const int32_t hi = static_cast<int32_t>((rem + (int64_t(1) << 31)) >> 32);
    float sn, cs;
    sincospi_quarter(static_cast<float>(hi) * (1.0f / 2147483648.0f), sn, cs);
    rotate_quarters(q4, cs, sn, c, s);
}

}  // namespace qft
