// qft_device.cuh -- device helpers shared by the pass, batch and tensor-core
// kernels: mbarrier / TMA wrappers, complex arithmetic, exact-phase twiddles,
// the buffer-B swizzle, the block sub-circuit, group tables and tile
// coordinates.  Internal to libqftfft.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "plan.hpp"

namespace qft {

// ------------------------------------------------------------------ helpers

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after limit_ns (the caller reports QFT_ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, const int32_t c[5],
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]),
        "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Index of the lowest set bit of j (j > 0).  Written as plain arithmetic so
// that, with j a constant of an unrolled loop, it folds to a constant and the
// register arrays it indexes stay in registers (an opaque intrinsic there
// would force those arrays into local memory).
__host__ __device__ constexpr int low_bit(int j) {
    return (j & 1) ? 0 : (j & 2) ? 1 : (j & 4) ? 2 : (j & 8) ? 3 : (j & 16) ? 4 : (j & 32) ? 5 : 6;
}

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// exp(2 pi i m / 32) for m = 0..15 (cos, sin): the rotations of controlled
// phases between wires at distance <= 4 inside one register block
// (R_2 .. R_5 and their products).
__device__ constexpr double kW32c[16] = {
    1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
    0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173, 0.19509032201612826785,
    0.0, -0.19509032201612826785, -0.38268343236508977173, -0.55557023301960222474,
    -0.70710678118654752440, -0.83146961230254523708, -0.92387953251128675613, -0.98078528040323044913};
__device__ constexpr double kW32s[16] = {
    0.0, 0.19509032201612826785, 0.38268343236508977173, 0.55557023301960222474,
    0.70710678118654752440, 0.83146961230254523708, 0.92387953251128675613, 0.98078528040323044913,
    1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
    0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173, 0.19509032201612826785};

// z *= exp(DIR * 2 pi i m / 32).  With m a compile-time constant after loop
// unrolling the trivial rotations (1, +-i, -1) reduce to moves and negations.
template <int DIR, typename V>
__device__ __forceinline__ void rot32(V& z, int m) {
    using T = decltype(z.x);
    m &= 31;
    if (m == 0) return;
    const bool neg = m >= 16;
    const int mm = m & 15;
    if (mm == 8) {  // multiply by DIR * i
        const T t = z.x;
        if (DIR > 0) { z.x = -z.y; z.y = t; } else { z.x = z.y; z.y = -t; }
    } else if (mm != 0) {
        const T c = static_cast<T>(kW32c[mm]);
        const T s = static_cast<T>(DIR > 0 ? kW32s[mm] : -kW32s[mm]);
        const T re = z.x * c - z.y * s;
        z.y = z.x * s + z.y * c;
        z.x = re;
    }
    if (neg) { z.x = -z.x; z.y = -z.y; }
}

__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }

// exp(DIR * 2 pi i beta / 2^n) for an exact integer phase beta (any 64-bit
// value; only beta mod 2^n matters), n <= 40.  The phase is reduced exactly
// in fixed point (2^40 = one turn) to the nearest quarter turn, so the
// floating-point sine/cosine only sees |x| <= 1/4 (in units of pi).
template <typename T, int DIR>
__device__ __forceinline__ typename Vec2<T>::type phase_turns(uint64_t beta, int n) {
    const uint64_t b = (beta << (64 - n)) >> 24;            // beta mod 2^n, scaled to 2^40 per turn
    const uint64_t q4 = (b + (1ull << 37)) >> 38;            // nearest quarter turn, 0..4
    const int64_t rem = static_cast<int64_t>(b) - static_cast<int64_t>(q4 << 38);  // |rem| <= 2^37
    const T x = static_cast<T>(rem) * static_cast<T>(1.0 / 549755813888.0);      // rem / 2^39
    T s, c;
    sincospi_t(x, &s, &c);
    typename Vec2<T>::type r;
    switch (q4 & 3) {
        case 0: r.x = c; r.y = s; break;
        case 1: r.x = -s; r.y = c; break;
        case 2: r.x = -c; r.y = -s; break;
        default: r.x = s; r.y = -c; break;
    }
    if (DIR < 0) r.y = -r.y;
    return r;
}

// XOR swizzle of buffer B: the low SW bits of a tile index are XORed with the
// XOR-fold of its higher SW-bit groups.  A bank-conflict-free access needs the
// lanes of one SMEM wavefront (16 lanes x 8 bytes, or 8 lanes x 16 bytes) to
// hit distinct SW-bit slots; with this map that holds whenever those lanes'
// tile bits have distinct residues mod SW, which the planner arranges.
template <int SW>
__device__ __forceinline__ uint32_t swz(uint32_t x) {
    uint32_t y = x >> SW;
    uint32_t f = 0;
#pragma unroll
    for (int i = 0; i < 16 / SW + 1; ++i) { f ^= y; y >>= SW; }
    return x ^ (f & ((1u << SW) - 1));
}

// The r-wire sub-circuit of one block, in registers (Sec. 2, Fig. 1): for the
// block's wires from the top down, the (unnormalised) butterfly H then the
// controlled phases from the lower wires of the block within distance kk.
// v[j]: bit e of j is wire wlo + e.  The 1/sqrt(2) of every H is folded into
// the pass's final scale.
template <int DIR, int R, typename V>
__device__ __forceinline__ void block_circuit(V (&v)[1 << R], int kk) {
    constexpr int NJ = 1 << R;
#pragma unroll
    for (int t = R - 1; t >= 0; --t) {
        const int bit = 1 << t;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            if (!(j & bit)) {
                const V a = v[j], b = v[j | bit];
                v[j] = cadd(a, b);
                v[j | bit] = csub(a, b);
            }
        }
        if (kk >= R - 1) {
#pragma unroll
            for (int j = 0; j < NJ; ++j)
                if (j & bit) rot32<DIR>(v[j], (j & (bit - 1)) << (4 - t));
        } else {
            int lo = t - kk;
            if (lo < 0) lo = 0;
            const int mask = (bit - 1) & ~((1 << lo) - 1);
#pragma unroll
            for (int j = 0; j < NJ; ++j)
                if (j & bit) rot32<DIR>(v[j], (j & mask) << (4 - t));
        }
    }
}

// Per-stage group tables.  A group g (the 2^r amplitudes one thread holds in a
// stage) splits as g = (g & 31) | (g >> 5) << 5 into a lane part and a high
// part whose tile bits are disjoint, so every per-group quantity that is
// additive over disjoint bits is the combination of one lane entry (index
// g & 31) and one high entry (index 32 + (g >> 5)):
//   pb  tile index bits (OR),  ob  output address offset (sum),
//   V   the cross-twiddle factors exp(s 2 pi i beta_e / 2^n) of the group's
//       tile wires above the block, one per block wire e (product).
// The tile coordinate's share of the cross twiddle, U_e, is computed once per
// tile.  beta_e is additive over disjoint wire sets, so the full cross twiddle
// of block wire e is U_e * V_e(lane entry) * V_e(high entry).
template <typename V>
struct GroupTab {
    uint32_t* pb;
    int64_t* ob;
    V* tw;  // [e][entry], e < ntw: plane e holds factor e of every entry (lane reads are consecutive)
    int ntab;
};

// Integer phase beta_e of block wire c = wlo + e for the logical bits I (only
// wires above hi = wlo + r - 1 matter): the controlled phases CP(c, t) with
// t > hi, t - c <= kk, in units of 2^-n turns (Eq. 5 / Sec. 2).
__device__ __forceinline__ uint64_t cross_phase(uint64_t I, int n, int hi, int c, int kk) {
    const uint64_t rh = (__brevll(I) >> (64 - n)) & ((1ull << (n - 1 - hi)) - 1ull);
    uint64_t m = rh;
    const int lowcut = n - 1 - c - kk;  // keep targets t <= c + kk
    if (lowcut > 0) m &= ~((1ull << lowcut) - 1ull);
    return m << c;
}

// Deterministic CTA-wide sum (fixed shuffle tree, then warps in order).
template <int NT>
__device__ __forceinline__ double block_sum(double x, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = x;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < NT / 32; ++i) t += red[i];
    __syncthreads();
    return t;
}

// Output factor of the decode step (Sec. 3 step 4) times the folded 2^{-n/2}.
__device__ __forceinline__ double output_factor(const PassParams& P, double scale_in) {
    switch (P.scale_mode) {
        case 0: return scale_in > 0.0 ? P.inv_root_n / scale_in : 0.0;  // state
        case 1: return P.inv_root_n;                                     // unitary
        case 2: return 1.0;                                              // unnormalised
        default: return P.inv_root_n * P.inv_root_n;                     // 1/N
    }
}

__device__ __forceinline__ void issue_tile_load(const PassParams& P, const CUtensorMap* map, int64_t tile,
                                                void* dstA, uint64_t* bar, uint32_t bytes) {
    mbar_arrive_expect_tx(bar, bytes);
    if (P.load_mode == 1) {
        const char* src = static_cast<const char*>(P.in) + static_cast<int64_t>(bytes) * tile;
        bulk_load_1d(dstA, src, bytes, bar);
    } else {
        int32_t c[5];
#pragma unroll
        for (int d = 0; d < 5; ++d) {
            const int len = P.dim_len[d];
            c[d] = len ? static_cast<int32_t>((tile >> P.dim_src[d]) & ((int64_t(1) << len) - 1)) : 0;
        }
        tma_load_5d(dstA, map, c, bar);
    }
}

// Logical bits of the tile coordinate and its output address offset.
__device__ __forceinline__ void tile_coords(const PassParams& P, int64_t tile, uint64_t& I_tile, int64_t& out_tile) {
    I_tile = 0;
    out_tile = 0;
    for (int sg = 0; sg < P.nseg; ++sg) {
        const TileSeg& G = P.seg[sg];
        const uint64_t v = (static_cast<uint64_t>(tile) >> G.src) & ((1ull << G.len) - 1ull);
        I_tile |= v << G.wire;
        if (G.out_rev)
            out_tile += static_cast<int64_t>((__brevll(v) >> (64 - G.len)) << (G.out - G.len + 1));
        else
            out_tile += static_cast<int64_t>(v << G.out);
    }
}

// U_e for every stage of one tile: thread i < nU computes entry i.
template <typename T, int DIR>
__device__ __forceinline__ void compute_tile_twiddles(const PassParams& P, int64_t tile,
                                                      typename Vec2<T>::type* Ubuf) {
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
    Ubuf[i] = phase_turns<T, DIR>(beta, P.n);
}

// Build the group tables (pb, ob, cross-twiddle factors of the group's tile
// wires) of every stage of pass P into shared memory.
template <typename T, int DIR, int NT>
__device__ __forceinline__ void build_group_tables(const PassParams& P, GroupTab<typename Vec2<T>::type>& tab) {
    using V = typename Vec2<T>::type;
    const int tid = threadIdx.x;
    const int ntab = tab.ntab;
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
            for (int e = 0; e < P.ntw; ++e) {
                V w;
                w.x = T(1);
                w.y = T(0);
                if (S.cross && e < S.r) w = phase_turns<T, DIR>(cross_phase(iw, P.n, S.wlo + S.r - 1, S.wlo + e, P.kk), P.n);
                tab.tw[e * ntab + idx] = w;
            }
        }
    }
}

}  // namespace qft
