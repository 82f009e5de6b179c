// qft_wide.cuh -- the wide pass kernel (complex64): one HBM sweep with
// tiles of 2^14 amplitudes, so a transform of n <= 10 P wires needs only P
// passes (Sec. 2 Eq. 2 / Eq. 5 and Sec. 3.1: fusing more gates per sweep is
// what cuts the memory traffic).
//
// A tile is 4 coalescing batch bits (the 4 lowest input addresses, 128-byte
// HBM runs) plus two register stages of 5 tile bits each.  In the tile's bit
// order x:
//   x0..x3    batch bits (the 4 lowest input addresses)
//   x4..x8    stage 1, the pass's low block: E1 = 5 - R1 extra batch wires,
//             then its R1 wires ascending
//   x9..x13   stage 0, the pass's top block: E0 = 5 - R0 extra batch wires,
//             then its R0 wires ascending
// The planner orders the TMA box dimensions so that the tile lands in shared
// memory in exactly this order (with the hardware's 128-byte swizzle).
//
// 512 threads; each thread holds 32 amplitudes in registers in both stages
// (the whole tile lives in the register file between the stages):
//   stage 0: thread t owns the x bits 0..8 given by wide_x0(t) and the 32
//            values of x9..x13 (register index j = x >> 9);
//   stage 1: thread t owns the x bits {0..3, 9..13} given by wide_x1(t) and
//            the 32 values of x4..x8 (j = (x >> 4) & 31).
// Per tile:
//   1. wait for the TMA load of the tile into buffer T (issued one tile ahead);
//   2. stage 0: read T, cross twiddle of the controlled phases from wires
//      above the block (Eq. 5, exact integer phases), the block's Hadamards
//      and controlled phases in registers (Sec. 2, Fig. 1 order);
//   3. barrier: T is consumed, thread 0 issues the next tile's load into T,
//      so it streams in during the exchange, stage 1 and the stores;
//   4. exchange through buffer Z in two rounds (x bit 3, which is warp bit 0
//      in both thread maps, so a round is whole warps): the even warps write
//      their stage-0 results, sync among themselves, read their stage-1
//      inputs and go straight on to stage 1, while the odd warps, released by
//      a named barrier once Z is free, do the same -- one half's exchange
//      overlaps the other half's arithmetic;
//   5. stage 1 (cross twiddle + block circuit) and the store straight from
//      registers through the pass's output address map (the qubit-reversal
//      layout adapter and, in the last pass, the decode scale).
// Shared memory: T = 128 KiB, Z = 82 KiB (a 64 KiB half tile, padded so that
// every access pattern is bank-conflict free and every address is a thread
// base plus a compile-time offset).  One CTA per SM.
//
// Group mode (GROUP = true; batches of same-plan transforms): one launch runs
// the pass for G transforms at their own addresses.  Global tile s is local
// tile s mod 2^lt_bits of transform s >> lt_bits: the TMA load takes that
// transform's tensor map from a device array, the stores its output base.
// The norm is kept per transform: the first pass writes each tile's squared
// sum (a fixed-order CTA reduction in double-float arithmetic on the FP32
// pipe), and the last pass, before its first tile, sums each of its tiles'
// transform's tile sums in a fixed order and keeps the decode scale in shared
// memory, so every tile of a transform applies the same scale (Sec. 3 step 4).
// (FP64 runs at a small fraction of the FP32 rate on this GPU, so no FP64
// arithmetic is done per tile.)
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "plan.hpp"
#include "qft_device.cuh"
#include "qft_df.cuh"

namespace qft {

constexpr int kWideThreads = 512;
constexpr int kWideTileBits = 14;

// ------------------------------------------------------------ index maps
// (host + device, so the CPU tests check them exhaustively)

// Exchange-buffer index of tile index x: x without its bit 3 (the round bit).
__host__ __device__ constexpr uint32_t wide_compress(uint32_t x) { return (x & 7u) | ((x >> 4) << 3); }
// Padded exchange-buffer address of index z (monotone, hence injective).
__host__ __device__ constexpr uint32_t wide_zpad(uint32_t z) { return z + 8u * (z >> 5) + 8u * (z >> 8) + (z >> 9); }
constexpr uint32_t kWideZElems = wide_zpad(8191u) + 1u;
constexpr size_t kWideTileBytes = (size_t(1) << kWideTileBits) * 8;
constexpr size_t kWideSmemBytes = kWideTileBytes + size_t(kWideZElems) * 8;

// Physical element of tile index x in buffer T under the 128-byte TMA swizzle
// (16-byte chunk index = element bits 1..3, XORed with the 128-byte row bits
// 0..2 = element bits 4..6).
__host__ __device__ constexpr uint32_t wide_swz128(uint32_t x) { return x ^ (((x >> 4) & 7u) << 1); }

__host__ __device__ constexpr uint32_t wide_brev5(uint32_t v) {
    return ((v & 1u) << 4) | ((v & 2u) << 2) | (v & 4u) | ((v & 8u) >> 2) | ((v & 16u) >> 4);
}
// Stage-0 thread -> its x bits 0..8: lanes 0..4 -> x0, x1, x2, x6, x7;
// warps 0..3 -> x3, x4, x5, x8.
__host__ __device__ constexpr uint32_t wide_x0(uint32_t tid) {
    return (tid & 7u) | (((tid >> 3) & 1u) << 6) | (((tid >> 4) & 1u) << 7) | (((tid >> 5) & 1u) << 3) |
           (((tid >> 6) & 1u) << 4) | (((tid >> 7) & 1u) << 5) | (((tid >> 8) & 1u) << 8);
}
// Stage-1 thread -> its x bits {0..3, 9..13}.
//   top = false (middle and last passes): lanes 0..4 -> x0, x1, x2, x9, x10;
//     warps 0..3 -> x3, x11, x12, x13.  Stores run along output bits 0..2.
//   top = true (first pass of a natural-order plan, whose output puts the top
//     wires x13..x10 at output addresses 0..3): lanes 0..4 -> x13, x12, x11,
//     x10, x9; warps 0..3 -> x3, x0, x1, x2.  Stores run along output bits 0..3.
__host__ __device__ constexpr uint32_t wide_x1(uint32_t tid, bool top) {
    return top ? ((wide_brev5(tid & 31u) << 9) | (((tid >> 5) & 1u) << 3) | ((tid >> 6) & 7u))
               : ((tid & 7u) | (((tid >> 3) & 3u) << 9) | (((tid >> 5) & 1u) << 3) | ((tid >> 6) << 11));
}
// Exchange addresses: stage-0 thread t writes register j at wide_a0(t) + wide_k0(j)
// (tile index wide_x0(t) | j << 9); stage-1 thread t reads register j at
// wide_a1(t) + wide_k1(j) (tile index wide_x1(t) | j << 4).
__host__ __device__ constexpr uint32_t wide_k0(uint32_t j) { return 328u * j + (j >> 1); }
__host__ __device__ constexpr uint32_t wide_k1(uint32_t j) { return 8u * j + 8u * (j >> 2); }
__host__ __device__ constexpr uint32_t wide_a0(uint32_t tid) { return wide_zpad(wide_compress(wide_x0(tid))); }
__host__ __device__ constexpr uint32_t wide_a1(uint32_t tid, bool top) {
    return (wide_x1(tid, top) & 7u) + 328u * (wide_x1(tid, top) >> 9) + ((wide_x1(tid, top) >> 9) >> 1);
}

// ------------------------------------------------------------ device code

__device__ __forceinline__ void tma_prefetch_l2_5d(const CUtensorMap* map, const int32_t c[5]) {
    asm volatile("cp.async.bulk.prefetch.tensor.5d.L2.global.tile [%0, {%1, %2, %3, %4, %5}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4])
                 : "memory");
}

// Named CTA barriers (barrier 0 is __syncthreads): bar.arrive signals without
// waiting (with release semantics for the thread's earlier shared-memory
// accesses), bar.sync waits for `count` arrivals.
__device__ __forceinline__ void bar_sync_n(uint32_t id, uint32_t count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive_n(uint32_t id, uint32_t count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
constexpr uint32_t kBarEvenWrote = 2; // the even warps' exchange writes are done
constexpr uint32_t kBarZFree = 3;     // the even warps have read the exchange buffer
constexpr uint32_t kBarOddWrote = 4;  // the odd warps' exchange writes are done

// 8-byte asynchronous global -> shared copy (no register holds the value in flight).
__device__ __forceinline__ void cp_async_8(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Local tile of global tile s (group mode: the tile within its transform).
template <bool GROUP>
__device__ __forceinline__ int64_t wide_local(const WideParams& P, int64_t s) {
    if constexpr (GROUP) return s & ((int64_t(1) << P.lt_bits) - 1);
    else return s;
}

// Decode factor of the last pass from scale_in (Sec. 3 step 4; scale modes as qft_execute).
__device__ __forceinline__ float wide_decode_factor(const WideParams& P, double scale_in) {
    double f;
    switch (P.scale_mode) {
        case 0: f = scale_in > 0.0 ? P.inv_root_n / scale_in : 0.0; break;
        case 1: f = P.inv_root_n; break;
        case 2: f = 1.0; break;
        default: f = P.inv_root_n * P.inv_root_n; break;
    }
    return static_cast<float>(f);
}

__device__ __forceinline__ void wide_coords(const WideParams& P, int64_t tile, int32_t c[5]) {
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        const int len = P.dim_len[d];
        c[d] = len ? static_cast<int32_t>((tile >> P.dim_src[d]) & ((int64_t(1) << len) - 1)) : 0;
    }
}

__device__ __forceinline__ void wide_tile_coords(const WideParams& P, int64_t tile, uint64_t& I_tile,
                                                 int64_t& out_tile) {
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

// Per-tile cross-twiddle tables.  The cross phase of a block wire is a sum of
// independent contributions of the wires above it (Eq. 5), so for a thread it
// splits exactly into (tile coordinates + the 4 batch bits x0..x3) and (the
// thread's other 5 fixed bits).  UA holds the first part for every value a of
// x0..x3: entry (i * 16 + a), i < R0 for stage-0 wire wlo0 + i, i = R0 + e for
// stage-1 wire wlo1 + e.  Threads 0 .. 16 (R0 + R1) - 1 build one entry each.
template <int DIR, int R0, int R1, bool GROUP>
__device__ __forceinline__ void wide_tile_twiddles(const WideParams& P, int64_t tile, float2* UA, int kk) {
    const int t = threadIdx.x;
    if (t >= 16 * (R0 + R1) || tile >= P.num_tiles) return;
    const int i = t >> 4, a = t & 15;
    uint64_t I;
    int64_t dummy;
    wide_tile_coords(P, wide_local<GROUP>(P, tile), I, dummy);
#pragma unroll
    for (int b = 0; b < 4; ++b)
        if ((a >> b) & 1) I |= 1ull << P.p_wire[b];
    const int s = i < R0 ? 0 : 1;
    const int e = s ? i - R0 : i;
    const int wlo = s ? P.wlo1 : P.wlo0;
    const int hi = wlo + (s ? R1 : R0) - 1;
    UA[t] = phase_turns<float, DIR>(cross_phase(I, P.n, hi, wlo + e, kk), P.n);
}

// Diagonal prod_e tau_e^{j_e} on the 2^R amplitudes of one group: the low two
// bits' products first, then each high-bit product built right before use
// (few twiddles live at a time).
template <int R>
__device__ __forceinline__ void wide_apply_cross(float2 (&g)[1 << R], const float2 (&tau)[R]) {
    constexpr int LB = R < 2 ? R : 2;
    constexpr int HB = R - LB;
    float2 t01 = tau[0];
    if (LB == 2) t01 = cmul(tau[0], tau[1]);
#pragma unroll
    for (int j = 1; j < (1 << R); ++j) {
        const int a = j & ((1 << LB) - 1);
        if (a == 1) g[j] = cmul(g[j], tau[0]);
        else if (a == 2) g[j] = cmul(g[j], tau[1]);
        else if (a == 3) g[j] = cmul(g[j], t01);
    }
#pragma unroll
    for (int b = 1; b < (1 << HB); ++b) {
        float2 th = tau[LB + low_bit(b)];
#pragma unroll
        for (int e = low_bit(b) + 1; e < HB; ++e)
            if ((b >> e) & 1) th = cmul(th, tau[LB + e]);
#pragma unroll
        for (int a = 0; a < (1 << LB); ++a) g[(b << LB) | a] = cmul(g[(b << LB) | a], th);
    }
}

// One register stage on the thread's 32 values: 2^E groups (the extra batch
// bits, register bits 0..E-1) of 2^R block amplitudes (register bits E..4).
// uv: the group-independent cross twiddle of each block wire; W: the extra
// bits' factor per group ([js][e], js >= 1).
template <int DIR, int R>
__device__ __forceinline__ void wide_stage(float2 (&v)[32], const float2 (&uv)[R], const float2* __restrict__ W,
                                           bool cross, int kk) {
    constexpr int E = 5 - R;
#pragma unroll
    for (int js = 0; js < (1 << E); ++js) {
        float2 g[1 << R];
#pragma unroll
        for (int jb = 0; jb < (1 << R); ++jb) g[jb] = v[js + (jb << E)];
        if (cross) {
            float2 tau[R];
#pragma unroll
            for (int e = 0; e < R; ++e) tau[e] = js ? cmul(uv[e], W[js * R + e]) : uv[e];
            wide_apply_cross<R>(g, tau);
        }
        block_circuit<DIR, R>(g, kk);
#pragma unroll
        for (int jb = 0; jb < (1 << R); ++jb) v[js + (jb << E)] = g[jb];
    }
}

template <int DIR, int R0, int R1, bool TOP, bool GROUP>
__global__ void __launch_bounds__(kWideThreads, 1)
    qft_wide_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ WideParams P) {
    constexpr int E0 = 5 - R0, E1 = 5 - R1;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2* const T = reinterpret_cast<float2*>(smem_raw);
    float2* const Z = reinterpret_cast<float2*>(smem_raw + kWideTileBytes);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(16) float2 UA[2][16 * (R0 + R1)];  // per tile: tile coordinates + batch bits x0..x3
    __shared__ __align__(16) float2 VB[32 * (R0 + R1)];     // per kernel: the thread's other fixed bits
    __shared__ __align__(16) float2 W0[(1 << E0) * R0];
    __shared__ __align__(16) float2 W1[(1 << E1) * R1];
    __shared__ double red[kWideThreads / 32];
    __shared__ float2 redt[GROUP ? 2 : 1][kWideThreads / 32];  // group mode: per-tile warp sums (hi, lo), double-buffered
    __shared__ float s_scale[GROUP ? kWideGroupTilesPerCta : 1];  // group mode, last pass: decode scale of the k-th tile
    __shared__ void* s_outp[2];  // group mode: the output base of the k-th tile's transform, fetched a tile ahead
    __shared__ int64_t s_othr[kWideThreads];  // each thread's output offset (kept out of registers)

    const uint32_t tid = threadIdx.x;
    const uint32_t x0 = wide_x0(tid), x1 = wide_x1(tid, TOP);
    const uint32_t pT = wide_swz128(x0);
    const uint32_t a0 = wide_a0(tid), a1 = wide_a1(tid, TOP);
    const bool round1 = ((tid >> 5) & 1u) != 0;
    const int hi0 = P.wlo0 + R0 - 1, hi1 = P.wlo1 + R1 - 1;
    const bool cross0 = hi0 < P.n - 1;  // stage 1 always has the stage-0 wires above it

    // The thread's output offset, and the indices of its fixed bits in the
    // cross-twiddle tables: x0..x3 (UA) and the other five (VB: stage 0
    // x4..x8, stage 1 x9..x13).
    {
        int64_t othr = 0;
        for (int b = 0; b < kWideTileBits; ++b)
            if ((x1 >> b) & 1u) othr += int64_t(1) << P.p_out[b];
        s_othr[tid] = othr;
    }
    const uint32_t ia0 = x0 & 15u, ib0 = (x0 >> 4) & 31u;
    const uint32_t ia1 = x1 & 15u, ib1 = x1 >> 9;
    // The cutoff k of global tile s's transform (group mode: from the sorted
    // cutoff runs; else the plan's).
    auto kk_of = [&](int64_t s) -> int {
        if constexpr (GROUP) {
            const int64_t ti = s >> P.lt_bits;
            int v = P.gk_val[0];
#pragma unroll
            for (int i = 1; i < kWideGroupMaxK; ++i)
                if (i < P.gk_n && ti >= P.gk_end[i - 1]) v = P.gk_val[i];
            return v;
        } else {
            return P.kk;
        }
    };
    // The kernel-wide cross-twiddle tables for cutoff kk.
    auto build_tables = [&](int kk) {
        // VB: entry (i * 32 + b), i as in UA; bits x4 + k (stage 0) or x9 + k (stage 1) = bit k of b
        for (int t = tid; t < 32 * (R0 + R1); t += kWideThreads) {
            const int i = t >> 5, b = t & 31;
            const int s = i < R0 ? 0 : 1;
            const int e = s ? i - R0 : i;
            const int wlo = s ? P.wlo1 : P.wlo0;
            const int hi = wlo + (s ? R1 : R0) - 1;
            uint64_t I = 0;
            for (int k = 0; k < 5; ++k)
                if ((b >> k) & 1) I |= 1ull << P.p_wire[(s ? 9 : 4) + k];
            VB[t] = (s || cross0) ? phase_turns<float, DIR>(cross_phase(I, P.n, hi, wlo + e, kk), P.n) : cunit<float2>();
        }
        // the extra batch bits' factors, per group of the thread's registers
        if (tid < (1 << E0) * R0) {
            const int js = tid / R0, e = tid % R0;
            uint64_t I = 0;
            for (int i = 0; i < E0; ++i)
                if ((js >> i) & 1) I |= 1ull << P.p_wire[9 + i];
            W0[tid] = cross0 ? phase_turns<float, DIR>(cross_phase(I, P.n, hi0, P.wlo0 + e, kk), P.n) : cunit<float2>();
        }
        if (tid >= 64 && tid < 64 + (1 << E1) * R1) {
            const int w = tid - 64, js = w / R1, e = w % R1;
            uint64_t I = 0;
            for (int i = 0; i < E1; ++i)
                if ((js >> i) & 1) I |= 1ull << P.p_wire[4 + i];
            W1[w] = phase_turns<float, DIR>(cross_phase(I, P.n, hi1, P.wlo1 + e, kk), P.n);
        }
    };
    int64_t tile = blockIdx.x;
    int kk_tab = kk_of(tile);  // the cutoff the tables hold
    build_tables(kk_tab);
    if (tid == 0) mbar_init(&mbar, 1);
    if constexpr (GROUP) {
        if (tid == 0 && tile < P.num_tiles) s_outp[0] = P.outs[tile >> P.lt_bits];
    }
    wide_tile_twiddles<DIR, R0, R1, GROUP>(P, tile, UA[0], kk_tab);
    if constexpr (GROUP) {
        // Last pass: the decode scale of each of this CTA's tiles (the host keeps
        // them <= kWideGroupTilesPerCta): warp w takes tiles w, w + 16, ...; its
        // lanes sum the transform's tile sums in a fixed xor-butterfly order.
        if (P.last) {
            const int64_t mine = (P.num_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
            const int lane = tid & 31, tpt = 1 << P.lt_bits;
            for (int64_t j = tid >> 5; j < mine; j += kWideThreads / 32) {
                const int64_t s = blockIdx.x + j * gridDim.x;
                const int64_t ti = s >> P.lt_bits;
                const double* tp = P.tpart + (ti << P.lt_bits);
                double a = lane < tpt ? tp[lane] : 0.0;
                if (lane + 32 < tpt) a += tp[lane + 32];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0) {
                    const double scale_in = sqrt(a);
                    s_scale[j] = wide_decode_factor(P, scale_in);
                    if ((s & (tpt - 1)) == 0 && P.gscale) {
                        double* g = P.gscale[ti];
                        if (g) *g = scale_in;
                    }
                }
            }
        }
    }
    __syncthreads();

    // Last pass: scale_in from the first pass's per-CTA partial sums (group
    // mode: per tile, below).
    float scale = 1.f;
    if (!GROUP && P.last) {
        double s = 0.0;
        for (int i = tid; i < P.npartials; i += kWideThreads) s += P.partials[i];
        const double scale_in = sqrt(block_sum<kWideThreads>(s, red));
        scale = wide_decode_factor(P, scale_in);
        if (blockIdx.x == 0 && tid == 0) {
            P.meta[0] = scale_in;
            if (P.user_scale) *P.user_scale = scale_in;
        }
    }

    // the input tensor map of global tile s
    auto map_of = [&](int64_t s) -> const CUtensorMap* {
        if constexpr (GROUP) return static_cast<const CUtensorMap*>(P.maps) + (s >> P.lt_bits);
        else return &tmap;
    };
    auto issue = [&](int64_t s) {  // thread 0: load tile s into T
        int32_t c[5];
        wide_coords(P, wide_local<GROUP>(P, s), c);
        mbar_arrive_expect_tx(&mbar, static_cast<uint32_t>(kWideTileBytes));
        tma_load_5d(T, map_of(s), c, &mbar);
        if (P.l2_prefetch && s + gridDim.x < P.num_tiles) {
            wide_coords(P, wide_local<GROUP>(P, s + gridDim.x), c);
            tma_prefetch_l2_5d(map_of(s + gridDim.x), c);
        }
    };
    if (tid == 0 && !P.test_skip_first_load && tile < P.num_tiles) issue(tile);

    double norm_acc = 0.0;
    uint32_t parity = 0u;
    bool aborted = false, ok = true;
    for (int k = 0; tile < P.num_tiles; tile += gridDim.x, ++k) {
        const int kk = kk_of(tile);
        if constexpr (GROUP) {
            if (P.last) scale = s_scale[k];
            if (kk != kk_tab) {  // the next transform run: every thread is done with the tables
                __syncthreads();
                build_tables(kk);
                __syncthreads();
                kk_tab = kk;
            }
        }
        ok = mbar_wait_bounded(&mbar, parity, P.wait_limit_ns);
        parity ^= 1u;
        const float2* Ucur = UA[k & 1];
        float2 v[32];
        float tile_norm = 0.f;  // group mode: the thread's share of this tile's squared norm
        if (ok) {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = T[pT + (uint32_t(j) << 9)];
            if (P.first) {
                float2 s0 = make_float2(0.f, 0.f), s1 = s0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    s0 = cfma2(v[j], v[j], s0);
                    s1 = cfma2(v[j + 16], v[j + 16], s1);
                }
                const float ts = (s0.x + s0.y) + (s1.x + s1.y);
                if constexpr (GROUP) tile_norm = ts;
                else norm_acc += static_cast<double>(ts);
            }
            float2 uv[R0];
#pragma unroll
            for (int e = 0; e < R0; ++e) uv[e] = cmul(Ucur[e * 16 + ia0], VB[e * 32 + ib0]);
            wide_stage<DIR, R0>(v, uv, W0, cross0, kk);
        }
        if constexpr (GROUP) {
            if (P.first) {  // the warp's sum in double-float (two-sum is exact, so every lane ends equal)
                dfloat t(tile_norm, 0.f);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    t = df_add(t, dfloat(__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o)));
                if ((tid & 31) == 0) redt[k & 1][tid >> 5] = make_float2(t.hi, t.lo);
            }
        }
        if constexpr (GROUP) {
            if (tid == 0) cp_async_wait_all();  // this tile's output base has landed in s_outp
        }
        // every thread is past the previous tile's exchange: Z may be written
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        if constexpr (GROUP) {
            if (P.first && tid == 32) {  // the tile's sum, warps in order (the next write to this half is two tiles on)
                dfloat t(redt[k & 1][0].x, redt[k & 1][0].y);
#pragma unroll
                for (int w = 1; w < kWideThreads / 32; ++w) t = df_add(t, dfloat(redt[k & 1][w].x, redt[k & 1][w].y));
                t = df_norm(t);
                P.tpart[tile] = static_cast<double>(t.hi) + static_cast<double>(t.lo);
            }
        }
        // T has been read: the next tile streams into it during the rest of this one.
        if (tid == 0 && tile + gridDim.x < P.num_tiles) {
            fence_proxy_async_smem();
            issue(tile + gridDim.x);
            if constexpr (GROUP) cp_async_8(&s_outp[(k + 1) & 1], P.outs + ((tile + gridDim.x) >> P.lt_bits));
        }
        wide_tile_twiddles<DIR, R0, R1, GROUP>(P, tile + gridDim.x, UA[(k + 1) & 1], kk_of(tile + gridDim.x));
        if (!round1) {  // even warps: x bit 3 = 0
#pragma unroll
            for (int j = 0; j < 32; ++j) Z[a0 + wide_k0(j)] = v[j];
            bar_sync_n(kBarEvenWrote, kWideThreads / 2);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = Z[a1 + wide_k1(j)];
            bar_arrive_n(kBarZFree, kWideThreads);
        } else {  // odd warps: x bit 3 = 1, once the even warps have read Z
            bar_sync_n(kBarZFree, kWideThreads);
#pragma unroll
            for (int j = 0; j < 32; ++j) Z[a0 + wide_k0(j)] = v[j];
            bar_sync_n(kBarOddWrote, kWideThreads / 2);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = Z[a1 + wide_k1(j)];
        }
        if (P.last) {  // the decode scale (stage 1 is linear, so it may come first)
            const float2 sc = make_float2(scale, scale);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = cmul2(v[j], sc);
        }
        {
            float2 uv[R1];
#pragma unroll
            for (int e = 0; e < R1; ++e) uv[e] = cmul(Ucur[(R0 + e) * 16 + ia1], VB[(R0 + e) * 32 + ib1]);
            wide_stage<DIR, R1>(v, uv, W1, true, kk);
        }
        uint64_t I_tile;
        int64_t out_tile;
        wide_tile_coords(P, wide_local<GROUP>(P, tile), I_tile, out_tile);
        float2* base;
        if constexpr (GROUP) base = static_cast<float2*>(s_outp[k & 1]);
        else base = static_cast<float2*>(P.out);
        float2* __restrict__ outp = base + (out_tile + s_othr[tid]);
#pragma unroll
        for (int j = 0; j < 32; ++j) outp[P.oj[j]] = v[j];
    }

    if (aborted) {
        if (tid == 0) {
            atomicExch(P.status, -5);  // QFT_ERR_TIMEOUT
            // let this tile's copy land before the CTA's shared memory is released
            // (the next tile's is issued only after the check)
            if (!ok) mbar_wait_bounded(&mbar, parity ^ 1u, P.wait_limit_ns);
            if constexpr (GROUP) cp_async_wait_all();
        }
        return;
    }
    if (!GROUP && P.first) {
        const double tot = block_sum<kWideThreads>(norm_acc, red);
        if (tid == 0) P.partials[blockIdx.x] = tot;
    }
}

template <int DIR, int R0, int R1, bool TOP, bool GROUP>
inline cudaError_t launch_wide_t(const CUtensorMap& map, const WideParams& P, int grid, cudaStream_t stream) {
    auto kern = qft_wide_kernel<DIR, R0, R1, TOP, GROUP>;
    const cudaError_t e = ensure_dynamic_smem(kern, kWideSmemBytes);
    if (e != cudaSuccess) return e;
    kern<<<grid, kWideThreads, kWideSmemBytes, stream>>>(map, P);
    return cudaGetLastError();
}

// Dispatch over the block splits (R0, R1) in {4, 5} x {3, 4, 5} and the
// first-pass store map, for one direction and mode (one translation unit each,
// so that they compile in parallel).
template <int DIR, bool GROUP>
inline cudaError_t launch_wide_dir(int r0, int r1, int top, const CUtensorMap& map, const WideParams& P, int grid,
                                   cudaStream_t st) {
#define QFT_WIDE_CASE(A, B)                                                        \
    if (r0 == A && r1 == B)                                                        \
        return top ? launch_wide_t<DIR, A, B, true, GROUP>(map, P, grid, st)       \
                   : launch_wide_t<DIR, A, B, false, GROUP>(map, P, grid, st);
    QFT_WIDE_CASE(5, 5)
    QFT_WIDE_CASE(5, 4)
    QFT_WIDE_CASE(5, 3)
    QFT_WIDE_CASE(4, 5)
    QFT_WIDE_CASE(4, 4)
    QFT_WIDE_CASE(4, 3)
#undef QFT_WIDE_CASE
    return cudaErrorInvalidValue;
}

}  // namespace qft
