// qft_pair.cuh -- paired register stages of complex64 passes (packed FP32).
//
// In a paired pass, tile bit 0 -- always a batch wire, never a wire of one of
// the pass's blocks -- becomes a SIMD lane: each thread runs the two groups
// that differ only in that bit through one instruction stream, and every FP32
// operation is a packed f32x2 instruction (add/sub/mul/fma.rn.f32x2, sm_100
// and later).  The two amplitudes of a pair are held planar in registers,
//   re = (a0.re, a1.re),  im = (a0.im, a1.im),
// so a complex product or butterfly needs no exchange between the two
// halves of a register pair.  Buffer B holds 16-byte pair units in that planar
// form; only the TMA-loaded tile (interleaved complex64) and the HBM stores
// are repacked.  The arithmetic per amplitude is that of the unpaired stage
// (same butterflies, the same rotation constants, the same exact-phase
// twiddles), so results agree with it to FP32 rounding.
//
// The two amplitudes of a pair see the same block circuit; their cross
// twiddles differ by the pair wire's own phase (when that wire lies above the
// block), which the lane part of the group tables carries per lane.
#pragma once
#include "qft_device.cuh"

namespace qft {

struct P2 {
    uint64_t re, im;  // bits 0..31: amplitude with pair bit 0; bits 32..63: pair bit 1
};

// Packed FP32 pairs.  The asm statements are not volatile, so the compiler
// may merge or drop them like ordinary arithmetic.
__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// exact sign flip of both halves (multiplication by -1 is exact)
__device__ __forceinline__ uint64_t f2_neg(uint64_t a) { return f2_mul(a, f2_pack(-1.f, -1.f)); }

__device__ __forceinline__ P2 p_bcast(float re, float im) { return {f2_pack(re, re), f2_pack(im, im)}; }
__device__ __forceinline__ P2 p_add(P2 a, P2 b) { return {f2_add(a.re, b.re), f2_add(a.im, b.im)}; }
__device__ __forceinline__ P2 p_sub(P2 a, P2 b) { return {f2_sub(a.re, b.re), f2_sub(a.im, b.im)}; }
// lane-wise complex product a * w
__device__ __forceinline__ P2 p_mul(P2 a, P2 w) {
    P2 r;
    r.re = f2_fma(a.im, f2_neg(w.im), f2_mul(a.re, w.re));
    r.im = f2_fma(a.re, w.im, f2_mul(a.im, w.re));
    return r;
}

// z *= exp(DIR * 2 pi i m / 32) in both lanes (m a compile-time constant after
// unrolling; +-i and -1 reduce to moves and exact sign flips).
template <int DIR>
__device__ __forceinline__ void rot32p(P2& z, int m) {
    m &= 31;
    if (m == 0) return;
    const bool neg = m >= 16;
    const int mm = m & 15;
    if (mm == 8) {
        const uint64_t t = z.re;
        if (DIR > 0) { z.re = f2_neg(z.im); z.im = t; } else { z.re = z.im; z.im = f2_neg(t); }
    } else if (mm != 0) {
        const float c = static_cast<float>(kW32c[mm]);
        const float s = static_cast<float>(DIR > 0 ? kW32s[mm] : -kW32s[mm]);
        const uint64_t re = f2_fma(z.im, f2_pack(-s, -s), f2_mul(z.re, f2_pack(c, c)));
        z.im = f2_fma(z.im, f2_pack(c, c), f2_mul(z.re, f2_pack(s, s)));
        z.re = re;
    }
    if (neg) { z.re = f2_neg(z.re); z.im = f2_neg(z.im); }
}

// The block sub-circuit of block_circuit (Sec. 2, Fig. 1 order) on pairs.
template <int DIR, int R>
__device__ __forceinline__ void block_circuit_p(P2 (&v)[1 << R], int kk) {
    constexpr int NJ = 1 << R;
#pragma unroll
    for (int t = R - 1; t >= 0; --t) {
        const int bit = 1 << t;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            if (!(j & bit)) {
                const P2 a = v[j], b = v[j | bit];
                v[j] = p_add(a, b);
                v[j | bit] = p_sub(a, b);
            }
        }
        if (kk >= R - 1) {
#pragma unroll
            for (int j = 0; j < NJ; ++j)
                if (j & bit) rot32p<DIR>(v[j], (j & (bit - 1)) << (4 - t));
        } else {
            int lo = t - kk;
            if (lo < 0) lo = 0;
            const int mask = (bit - 1) & ~((1 << lo) - 1);
#pragma unroll
            for (int j = 0; j < NJ; ++j)
                if (j & bit) rot32p<DIR>(v[j], (j & mask) << (4 - t));
        }
    }
}

// Group tables of a paired stage: as GroupTab, with the twiddle planes held
// as pairs.  Lane entries carry (factor, factor * pair-wire factor); high
// entries carry the same factor in both lanes.
struct GroupTabP {
    uint32_t* pb;
    int64_t* ob;
    P2* tw;  // [e][entry]
    int ntab;
};

template <int DIR>
__device__ __forceinline__ void compute_tile_twiddles_p(const PassParams& P, int64_t tile, P2* Ubuf) {
    const int i = threadIdx.x;
    if (i >= P.nU || tile >= P.num_tiles) return;
    int s = 0;
    while (s + 1 < P.nstages && P.st[s + 1].uoff <= i) ++s;
    const StageDesc& S = P.st[s];
    const int e = i - S.uoff;
    uint64_t I_tile;
    int64_t dummy;
    tile_coords(P, tile, I_tile, dummy);
    const uint64_t beta = cross_phase(I_tile, P.n, S.wlo + S.r - 1, S.wlo + e, P.kk);
    const float2 w = phase_turns<float, DIR>(beta, P.n);
    Ubuf[i] = p_bcast(w.x, w.y);
}

template <int DIR, int NT>
__device__ __forceinline__ void build_group_tables_p(const PassParams& P, GroupTabP& tab) {
    const int tid = threadIdx.x;
    const int ntab = tab.ntab;
    const uint64_t pair_wire = 1ull << P.p_wire[0];
    for (int s = 0; s < P.nstages; ++s) {
        const StageDesc& S = P.st[s];
        const int ng = 1 << S.ngbits;
        const int nhi = ng > 32 ? ng >> 5 : 1;
        for (int i = tid; i < 32 + nhi; i += NT) {
            const int g = i < 32 ? (i < ng ? i : 0) : ((i - 32) << 5);
            uint32_t pb = 0;
            uint64_t iw = 0;
            int64_t ob = 0;
            for (int b = 0; b < S.ngbits; ++b) {
                if ((g >> b) & 1) {
                    const int p = S.gpos[b];
                    pb |= 1u << p;
                    iw |= 1ull << P.p_wire[p];
                    ob += int64_t(1) << P.p_out[p];
                }
            }
            const int idx = P.tab_off[s] + i;
            tab.pb[idx] = pb;
            tab.ob[idx] = ob;
            const int hi = S.wlo + S.r - 1;
            for (int e = 0; e < P.ntw; ++e) {
                float2 w0 = make_float2(1.f, 0.f), w1 = w0;
                if (S.cross && e < S.r) {
                    w0 = phase_turns<float, DIR>(cross_phase(iw, P.n, hi, S.wlo + e, P.kk), P.n);
                    w1 = i < 32 ? phase_turns<float, DIR>(cross_phase(iw | pair_wire, P.n, hi, S.wlo + e, P.kk), P.n)
                                : w0;
                }
                tab.tw[e * ntab + idx] = {f2_pack(w0.x, w1.x), f2_pack(w0.y, w1.y)};
            }
        }
    }
}

// One paired register stage (stage kinds as in qft_pass.cu's run_stage).
// A: the TMA tile (interleaved complex64, dense tile order); Bb: buffer B in
// 16-byte pair units, XOR-swizzled on the unit index.
template <int DIR, int R, int KIND, int NT>
__device__ __forceinline__ void run_stage_p(const PassParams& P, const StageDesc& S, const GroupTabP& tab, int toff,
                                            const float2* __restrict__ A, P2* __restrict__ Bb, int64_t out_tile,
                                            float scale, const P2* __restrict__ U, bool acc_norm, double& norm_acc) {
    constexpr int NJ = 1 << R;
    constexpr bool kFromA = (KIND == 0 || KIND == 3);
    constexpr bool kToGlobal = (KIND == 2 || KIND == 3);
    const int ng = 1 << S.ngbits;
    const uint32_t q = static_cast<uint32_t>(S.q);
    uint32_t soff[NJ];
    soff[0] = 0;
#pragma unroll
    for (int j = 1; j < NJ; ++j) soff[j] = soff[j & (j - 1)] ^ static_cast<uint32_t>(S.img[low_bit(j)]);
    const bool cross = S.cross != 0;
    const bool use_u = cross && S.tile_above;
    P2 u[R];
#pragma unroll
    for (int e = 0; e < R; ++e) u[e] = use_u ? U[e] : p_bcast(1.f, 0.f);
    int64_t oo[R];
    if (kToGlobal) {
#pragma unroll
        for (int e = 0; e < R; ++e) oo[e] = int64_t(1) << P.p_out[q + e];
    }
    const bool adjacent = P.p_out[0] == 0;  // the pair is one 16-byte unit in the output too
    const int64_t d1 = int64_t(1) << P.p_out[0];
    const uint64_t sc2 = f2_pack(scale, scale);
    for (int g = threadIdx.x; g < ng; g += NT) {
        const int lo5 = toff + (g & 31), hi5 = toff + 32 + (g >> 5);
        const uint32_t pb = tab.pb[lo5] | tab.pb[hi5];
        P2 v[NJ];
        if (kFromA) {
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const float4 t = *reinterpret_cast<const float4*>(A + (pb + (uint32_t(j) << q)));
                v[j].re = f2_pack(t.x, t.z);
                v[j].im = f2_pack(t.y, t.w);
            }
        } else {
            const uint32_t base = swz<3>(pb >> 1);
#pragma unroll
            for (int j = 0; j < NJ; ++j) v[j] = Bb[base ^ soff[j]];
        }
        if (kFromA && acc_norm) {
            uint64_t a = f2_pack(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                a = f2_fma(v[j].re, v[j].re, a);
                a = f2_fma(v[j].im, v[j].im, a);
            }
            float a0, a1;
            f2_unpack(a, a0, a1);
            norm_acc += static_cast<double>(a0) + static_cast<double>(a1);
        }
        if (cross) {
            P2 tau[R];
#pragma unroll
            for (int e = 0; e < R; ++e) {
                if (S.lo_tw && S.hi_tw) tau[e] = p_mul(tab.tw[e * tab.ntab + lo5], tab.tw[e * tab.ntab + hi5]);
                else if (S.lo_tw) tau[e] = tab.tw[e * tab.ntab + lo5];
                else tau[e] = tab.tw[e * tab.ntab + hi5];
                if (use_u) tau[e] = p_mul(tau[e], u[e]);
            }
            constexpr int LB = R < 2 ? R : 2;
            constexpr int HB = R - LB;
            P2 tl[1 << LB], th[1 << HB];
#pragma unroll
            for (int a = 1; a < (1 << LB); ++a)
                tl[a] = (a & (a - 1)) ? p_mul(tl[a & (a - 1)], tau[low_bit(a)]) : tau[low_bit(a)];
#pragma unroll
            for (int b = 1; b < (1 << HB); ++b)
                th[b] = (b & (b - 1)) ? p_mul(th[b & (b - 1)], tau[LB + low_bit(b)]) : tau[LB + low_bit(b)];
#pragma unroll
            for (int j = 1; j < NJ; ++j) {
                const int a = j & ((1 << LB) - 1), b = j >> LB;
                if (a) v[j] = p_mul(v[j], tl[a]);
                if (b) v[j] = p_mul(v[j], th[b]);
            }
        }
        block_circuit_p<DIR, R>(v, P.kk);
        if (kToGlobal) {
            float2* __restrict__ out = static_cast<float2*>(P.out) + (out_tile + tab.ob[lo5] + tab.ob[hi5]);
            if (adjacent) {
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    int64_t o = 0;
#pragma unroll
                    for (int e = 0; e < R; ++e)
                        if (j & (1 << e)) o += oo[e];
                    float r0, r1, i0, i1;
                    f2_unpack(f2_mul(v[j].re, sc2), r0, r1);
                    f2_unpack(f2_mul(v[j].im, sc2), i0, i1);
                    *reinterpret_cast<float4*>(out + o) = make_float4(r0, i0, r1, i1);
                }
            } else {
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    int64_t o = 0;
#pragma unroll
                    for (int e = 0; e < R; ++e)
                        if (j & (1 << e)) o += oo[e];
                    float r0, r1, i0, i1;
                    f2_unpack(f2_mul(v[j].re, sc2), r0, r1);
                    f2_unpack(f2_mul(v[j].im, sc2), i0, i1);
                    out[o] = make_float2(r0, i0);
                    out[o + d1] = make_float2(r1, i1);
                }
            }
        } else {
            const uint32_t base = swz<3>(pb >> 1);
#pragma unroll
            for (int j = 0; j < NJ; ++j) Bb[base ^ soff[j]] = v[j];
        }
    }
}

template <int DIR, int KIND, int NT, int MAXR>
__device__ __forceinline__ void dispatch_r_p(const PassParams& P, int s, const GroupTabP& tab, const float2* A,
                                             P2* Bb, int64_t out_tile, float scale, const P2* U, bool acc_norm,
                                             double& norm_acc) {
    const StageDesc& S = P.st[s];
    const int toff = P.tab_off[s];
    switch (S.r) {
        case 1: run_stage_p<DIR, 1, KIND, NT>(P, S, tab, toff, A, Bb, out_tile, scale, U, acc_norm, norm_acc); break;
        case 2: run_stage_p<DIR, 2, KIND, NT>(P, S, tab, toff, A, Bb, out_tile, scale, U, acc_norm, norm_acc); break;
        case 3: run_stage_p<DIR, 3, KIND, NT>(P, S, tab, toff, A, Bb, out_tile, scale, U, acc_norm, norm_acc); break;
        default:
            if constexpr (MAXR >= 4)
                run_stage_p<DIR, 4, KIND, NT>(P, S, tab, toff, A, Bb, out_tile, scale, U, acc_norm, norm_acc);
            break;
    }
}

template <int DIR, int NT, int MAXR>
__device__ __forceinline__ void dispatch_stage_p(const PassParams& P, int s, const GroupTabP& tab, const float2* A,
                                                 P2* Bb, int64_t out_tile, float scale, const P2* U, bool acc_norm,
                                                 double& norm_acc) {
    const bool first = (s == 0), last = (s == P.nstages - 1);
    if (first && last) dispatch_r_p<DIR, 3, NT, MAXR>(P, s, tab, A, Bb, out_tile, scale, U, acc_norm, norm_acc);
    else if (first) dispatch_r_p<DIR, 0, NT, MAXR>(P, s, tab, A, Bb, out_tile, scale, U, acc_norm, norm_acc);
    else if (last) dispatch_r_p<DIR, 2, NT, MAXR>(P, s, tab, A, Bb, out_tile, scale, U, acc_norm, norm_acc);
    else dispatch_r_p<DIR, 1, NT, MAXR>(P, s, tab, A, Bb, out_tile, scale, U, acc_norm, norm_acc);
}

}  // namespace qft
