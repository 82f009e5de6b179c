// qft_batch_kernel.cuh -- the batched persistent kernel: one launch over a
// work list of tile items drawn from many transforms, running the pass
// kernel's stage code (qft_pass_kernels.cuh) per item.  Its instantiations are
// in qft_batch_f32.cu, qft_batch_f64.cu and qft_batch_df.cu; the host side
// (work list, queue order, layout) is qft_batch.cpp.
#pragma once

#include "qft_pass_kernels.cuh"

namespace qft {

// ------------------------------------------------------------ batched launch
//
// One persistent launch over a list of tile work items drawn from many
// transforms of different sizes and plans.  Each CTA claims items in order
// from an atomic counter; an item is one tile of one pass of one transform.
// A later-pass item waits (bounded) until every tile of its transform's
// previous pass has signalled completion.  The host queues the items as a
// wavefront over blocks of transforms (batch_order.hpp), so a later pass sits
// about a block of other items behind its predecessor: its producers have
// usually finished when it is claimed.  Loads are double-buffered (when two
// load buffers fit in shared memory): while a CTA computes its current item
// it has already claimed the next one and, if that item's producers are
// done, its tile is on the way into the other buffer; otherwise (or with one
// buffer) the load is issued after the current item, once the producers are
// done.  The pass descriptors are staged in shared memory one item ahead.
// Every item depends only on items earlier in the queue, claimed by running
// CTAs, and the earliest unfinished item is always some CTA's current item
// with its producers done, so the waits always end.

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Thread 0 of a batch CTA: wait until the producers of item `it` are done
// (bounded by wait_ns; a single check when `poll`), then issue its tile load
// into `dst`.  Returns 1 if the load was issued, 0 if `poll` found the
// producers still running, -1 if the wait gave up.
template <typename V>
__device__ __forceinline__ int batch_issue(const BatchItem& it, const PassParams* descs, const CUtensorMap* maps,
                                           const int* counters, V* dst, uint64_t* bar, bool poll,
                                           uint64_t wait_ns) {
    if (it.wait_ctr >= 0) {
        if (ld_acquire_gpu(counters + it.wait_ctr) < it.wait_target) {
            if (poll) return 0;
            const uint64_t t0 = global_timer_ns();
            while (ld_acquire_gpu(counters + it.wait_ctr) < it.wait_target)
                if (global_timer_ns() - t0 > wait_ns) return -1;
        }
        fence_proxy_async_global();  // the producers' stores before this item's TMA reads
    }
    const PassParams& P = descs[it.desc];
    const uint32_t bytes = (1u << P.tb) * static_cast<uint32_t>(sizeof(V));
    issue_tile_load(P, maps + (it.map >= 0 ? it.map : 0), it.tile, dst, bar, bytes);
    return 1;
}

// Completion signal of a stored item (every thread of the CTA calls it): the
// CTA's stores are made visible, then the pass's counter is incremented once.
// The CTA that completes a first pass sums the per-warp norms of all its
// tiles (lane j takes every 32nd partial, then a fixed shuffle tree:
// deterministic), publishes scale_in and increments once more, so the next
// pass waits for num_tiles + 1.
template <typename T, int NT>
__device__ __forceinline__ void batch_signal(const BatchItem& it, const PassParams& P, int* counters) {
    constexpr int kW = NT / 32;
    __threadfence();
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    int fin = 0;
    if (lane == 0) {
        const int old = atomicAdd(counters + it.signal_ctr, 1);
        fin = P.first && old == static_cast<int>(P.num_tiles) - 1;
    }
    if (__shfl_sync(0xffffffffu, fin, 0)) {
        __threadfence();
        const int np = static_cast<int>(P.num_tiles) * kW;
        double t = 0.0;
        for (int i = lane; i < np; i += 32) t += __ldcg(P.partials + (i / kW) * kBatchNormSlots + i % kW);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) {
            double scale_in = sqrt(t);
            if constexpr (AmpTraits<T>::kDF) scale_in = ldexp(scale_in, df_shift_from_meta(P.meta));
            P.meta[0] = scale_in;
            if (P.user_scale) *P.user_scale = scale_in;
            __threadfence();
            atomicAdd(counters + it.signal_ctr, 1);
        }
    }
}

template <typename T, int DIR, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    qft_batch_kernel(const BatchItem* __restrict__ items, int nitems, const PassParams* __restrict__ descs,
                     const CUtensorMap* __restrict__ maps, int* counters, int* next, int* status,
                     uint64_t wait_ns, BatchLayout lay) {
    using V = typename Vec2<T>::type;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ double red[NT / 32];
    __shared__ __align__(16) typename Vec2<T>::type Ubuf_raw[kMaxR * kMaxStages];
    // double-float: the table of the FP32-only per-tile factors (phase_turns_df)
    __shared__ __align__(16) V t40[AmpTraits<T>::kDF ? 129 : 1];
    __shared__ int s_first, s_next, s_pref, s_ok;
    __shared__ __align__(16) PassParams s_prm[2];  // this item's pass descriptor and the next one's
    __shared__ int s_nxdesc;
    static_assert(sizeof(PassParams) % 8 == 0, "descriptor copied in 8-byte words");

    const int tid = threadIdx.x;
    using Tr = AmpTraits<T>;
    // widest register block: as for the pass kernel of the same CTA shape
    constexpr int kBatchMaxR = NT > 256 ? (Tr::kDF ? 3 : 4) : ((MINB == 1 && !Tr::kDF) ? 5 : 4);
    const uint32_t max_elems = 1u << lay.max_tb;
    const uint32_t other = lay.nbuf == 2 ? max_elems : 0u;  // offset of the other load buffer (0: one buffer)
    V* B = reinterpret_cast<V*>(smem_raw);
    V* A0 = B + max_elems;  // load buffers A0 and, with two, A0 + max_elems
    V* Ubuf = Ubuf_raw;
    // group tables: twiddle planes (lay.tw_stride bytes per entry), output offsets, tile bits
    unsigned char* tab_raw = smem_raw + (1 + lay.nbuf) * static_cast<size_t>(max_elems) * sizeof(V);
    const size_t ntab = static_cast<size_t>(lay.max_ntab);
    GroupTab<V> tab;
    tab.ntab = lay.max_ntab;
    tab.tw = reinterpret_cast<V*>(tab_raw);
    tab.ob = reinterpret_cast<int64_t*>(tab_raw + static_cast<size_t>(lay.tw_stride) * ntab);
    tab.pb = reinterpret_cast<uint32_t*>(tab_raw + (static_cast<size_t>(lay.tw_stride) + 8) * ntab);
    tab.sb = tab.pb + ntab;
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
    }
    if constexpr (Tr::kDF) build_turns40_table<NT>(t40);
    __syncthreads();
    uint32_t parity = 0;    // phase bit per load buffer (every thread)
    uint32_t inflight = 0;  // buffers with a load issued and not yet waited for (thread 0)
    int cached_shape = -1;
    if (tid == 0) {
        const int c0 = atomicAdd(next, 1);
        int ok = 1;
        // (test hook: a transform whose plan asks for it leaves the CTA's first
        // tile load unissued, so the bounded wait on it expires)
        if (c0 < nitems && !descs[items[c0].desc].test_skip_first_load) {
            ok = batch_issue(items[c0], descs, maps, counters, A0, &mbar[0], false, wait_ns) > 0;
            if (ok) inflight |= 1u;
        }
        s_first = c0;
        s_ok = ok;
    }
    __syncthreads();
    int item = s_first;
    bool cur_ok = s_ok != 0;
    constexpr int kWords = static_cast<int>(sizeof(PassParams) / 8);
    static_assert(kWords <= NT, "one descriptor word per thread");
    if (item < nitems && tid < kWords)
        reinterpret_cast<uint64_t*>(&s_prm[0])[tid] = reinterpret_cast<const uint64_t*>(&descs[items[item].desc])[tid];
    __syncthreads();
    int buf = 0;
    int pb = 0;  // which s_prm holds this item's descriptor
    bool aborted = false;
    while (item < nitems) {
        if (!cur_ok) {  // the wait for this item's producers gave up (same value in every thread)
            aborted = true;
            break;
        }
        const int bnext = buf ^ (lay.nbuf - 1);  // the next item's buffer (the same one with one buffer)
        V* const A = A0 + (buf ? other : 0u);
        V* const Anext = A0 + (bnext ? other : 0u);
        if (tid == 0) {
            const int nx = atomicAdd(next, 1);
            int pref = 0;
            if (nx < nitems && bnext != buf) {  // with one buffer the load waits for this item's stages
                pref = batch_issue(items[nx], descs, maps, counters, Anext, &mbar[bnext], true, wait_ns);
                if (pref > 0) inflight |= 1u << bnext;
            }
            s_next = nx;
            s_pref = pref;
            s_nxdesc = nx < nitems ? items[nx].desc : 0;
        }
        const BatchItem it = items[item];
        // the pass descriptor, copied into shared memory during the previous item
        const PassParams& P = s_prm[pb];
        if (it.shape != cached_shape) {
            build_group_tables_wide<T, DIR, NT>(P, tab);
            cached_shape = it.shape;
        }
        if constexpr (Tr::kDF) compute_tile_twiddles_df<DIR>(P, it.tile, Ubuf, t40);
        else compute_tile_twiddles<T, DIR>(P, it.tile, Ubuf);
        __syncthreads();  // tables, twiddles, s_next, s_pref and s_nxdesc
        const int nx = s_next;
        const int pref = s_pref;
        // Each thread waits for the tile on its own; whether any wait gave up
        // is decided CTA-wide at the first barrier that follows.  A thread
        // whose wait gave up skips its stage work, and keeps the phase bit
        // (and thread 0 the in-flight mark) for the wait on exit.
        const bool okw = mbar_wait_bounded(&mbar[buf], (parity >> buf) & 1u, wait_ns);
        if (okw) {
            parity ^= 1u << buf;
            if (tid == 0) inflight &= ~(1u << buf);
        }
        uint64_t I_tile;
        int64_t out_tile;
        tile_coords(P, it.tile, I_tile, out_tile);
        // amplitude I/O of this item's transform (double-float: its own exponent shift)
        AmpIO io{0, 0, 0, 0};
        if constexpr (Tr::kDF) {
            io.raw_in = P.first;
            io.raw_out = P.last;
            io.shift_in = df_shift_from_meta(P.meta);
        }
        T scale = T(1);
        bool checked = false;  // the tile wait's CTA-wide check is done
        if (P.first && P.last) {
            if (__syncthreads_or(!okw)) {
                aborted = true;
                break;
            }
            checked = true;
            double s = 0.0;
            for (uint32_t i = tid; i < (1u << P.tb); i += NT) s += Tr::norm2_at(A, i, io);
            const double tot = block_sum<NT>(s, red);
            const double scale_in = Tr::kDF ? ldexp(sqrt(tot), io.shift_in) : sqrt(tot);
            Tr::out_scale(output_factor(P, scale_in), scale, io.shift_out, io.shift_in);
            if (tid == 0) {
                P.meta[0] = scale_in;
                if (P.user_scale) *P.user_scale = scale_in;
            }
        } else if (P.last) {
            // scale_in was published by the first pass's finalising CTA before
            // the counters this item waited on (read past L1: written in this launch)
            const double scale_in = __ldcg(P.meta);
            Tr::out_scale(output_factor(P, scale_in), scale, io.shift_out, io.shift_in);
        }
        double norm_acc = 0.0;
        for (int s = 0; s < P.nstages; ++s) {
            if (okw)
                dispatch_stage<T, DIR, NT, kBatchMaxR>(P, s, tab, A, B, out_tile, scale, Ubuf + P.st[s].uoff,
                                                       P.first && !P.last, norm_acc, io);
            if (!checked) {
                checked = true;
                if (__syncthreads_or(!okw)) {
                    aborted = true;
                    break;
                }
            } else {
                __syncthreads();
            }
        }
        if (aborted) break;
        // the next item's descriptor: loaded now, stored into the other
        // s_prm after this item's completion signal (its latency overlaps it)
        uint64_t nd = 0;
        const bool has_nd = nx < nitems && tid < kWords;
        if (has_nd) nd = reinterpret_cast<const uint64_t*>(&descs[s_nxdesc])[tid];
        if (P.first && !P.last) {
            // one partial norm per warp of each first-pass tile (no CTA-wide reduction)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) norm_acc += __shfl_down_sync(0xffffffffu, norm_acc, o);
            if ((tid & 31) == 0) P.partials[it.tile * kBatchNormSlots + (tid >> 5)] = norm_acc;
        }
        if (it.signal_ctr >= 0) batch_signal<T, NT>(it, P, counters);
        if (has_nd) reinterpret_cast<uint64_t*>(&s_prm[pb ^ 1])[tid] = nd;
        fence_proxy_async_smem();  // this item's shared-memory reads before later TMA writes
        // the next item's load, if its producers were still running above
        if (tid == 0) {
            int ok = 1;
            if (nx < nitems && pref == 0) {
                ok = batch_issue(items[nx], descs, maps, counters, Anext, &mbar[bnext], false, wait_ns) > 0;
                if (ok) inflight |= 1u << bnext;
            }
            s_ok = ok;
        }
        __syncthreads();
        cur_ok = s_ok != 0;
        item = nx;
        buf = bnext;
        pb ^= 1;
    }
    if (aborted) {
        if (tid == 0) {
            atomicExch(status, -5);  // QFT_ERR_TIMEOUT
            // let in-flight copies land before the CTA's shared memory is released
            for (int b = 0; b < 2; ++b)
                if ((inflight >> b) & 1u) mbar_wait_bounded(&mbar[b], (parity >> b) & 1u, wait_ns);
        }
    }
}

template <typename T, int DIR, int NT, int MINB>
inline cudaError_t launch_batch_t(const BatchItem* items, int nitems, const PassParams* descs,
                                  const CUtensorMap* maps, int* counters, int* next, int* status, uint64_t wait_ns,
                                  BatchLayout lay, int grid, size_t smem, cudaStream_t stream) {
    auto kern = qft_batch_kernel<T, DIR, NT, MINB>;
    {
        const cudaError_t e = ensure_dynamic_smem(kern, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, NT, smem, stream>>>(items, nitems, descs, maps, counters, next, status, wait_ns, lay);
    return cudaGetLastError();
}

}  // namespace qft
