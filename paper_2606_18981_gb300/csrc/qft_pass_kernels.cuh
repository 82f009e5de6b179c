// qft_pass_kernels.cuh -- the SMEM-staged pass kernel of the QFT->FFT hot path
// (sm_103a) and its stage code, as templates (the batched persistent kernel
// that reuses the stages is in qft_batch_kernel.cuh).  Each dtype's
// instantiations live in their own translation unit (qft_pass_f32.cu,
// qft_pass_f64.cu, qft_pass_df.cu) so they compile in parallel; qft_pass.cu
// holds the host-side dispatch.
//
// One launch = one HBM sweep over the state.  A persistent CTA loops over
// tiles: a tile (2^tb amplitudes, the pass's wire group plus batch wires) is
// fetched by TMA into buffer A (cp.async.bulk.tensor, or a 1D cp.async.bulk
// for contiguous tiles), completion tracked by an mbarrier; then the pass's
// register stages run:
//
//   stage s: every thread takes the 2^r amplitudes that differ only in the
//   stage's r wires (one fused block of the circuit), multiplies them by the
//   cross twiddle of the controlled phases whose target wire lies above the
//   block (Eq. 5 / Sec. 2: diagonal two-level updates, folded into one phase
//   per amplitude computed from exact integer phases), then applies the
//   block's own Hadamards and controlled phases in registers (Sec. 2,
//   Fig. 1 order), and writes the amplitudes back to buffer B (XOR-swizzled
//   so that every stage reads and writes without bank conflicts).
//
// The last stage of a pass stores straight from registers to HBM with the
// output wire->address map of the pass (this is where the qubit-reversal
// swaps and the decode scale of Sec. 3 step 4 are folded in).  While stages
// 1.. run on buffer B, the TMA engine already fetches the next tile into A.
//
// The first pass also accumulates ||x||^2 (Sec. 3 step 1) from the raw
// amplitudes it reads; the last pass turns the per-CTA partial sums into
// scale_in and applies 1/scale_in together with the folded 2^{-n/2} of the
// n unnormalised butterflies.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "plan.hpp"
#include "qft_device.cuh"

namespace qft {

// Stage kinds: where a stage reads its amplitudes and where it writes them.
enum StageKind { K_FIRST = 0, K_MID = 1, K_LAST = 2, K_ONLY = 3 };
//   K_FIRST  TMA buffer A (dense tile order) -> swizzled buffer B
//   K_MID    B -> B
//   K_LAST   B -> HBM through the pass's output address map (with the output scale)
//   K_ONLY   A -> HBM (a pass of a single stage)

template <typename T, int DIR, int R, int KIND, int NT>
__device__ __forceinline__ void run_stage(const PassParams& P, const StageDesc& S,
                                          const GroupTab<typename Vec2<T>::type>& tab, int toff,
                                          const typename Vec2<T>::type* __restrict__ A,
                                          typename Vec2<T>::type* __restrict__ Bb, int64_t out_tile, T scale,
                                          const typename Vec2<T>::type* __restrict__ U, bool acc_norm,
                                          double& norm_acc, const AmpIO& io) {
    using V = typename Vec2<T>::type;
    using Tr = AmpTraits<T>;
    constexpr int NJ = 1 << R;
    constexpr bool kFromA = (KIND == K_FIRST || KIND == K_ONLY);
    constexpr bool kToGlobal = (KIND == K_LAST || KIND == K_ONLY);
    const int ng = 1 << S.ngbits;
    const uint32_t q = static_cast<uint32_t>(S.q);
    // swizzled offsets of the register bits (the swizzle is XOR-linear), by Gray steps
    uint32_t soff[NJ];
    soff[0] = 0;
#pragma unroll
    for (int j = 1; j < NJ; ++j) soff[j] = soff[j & (j - 1)] ^ static_cast<uint32_t>(S.img[low_bit(j)]);
    const bool cross = S.cross != 0;
    const bool use_u = cross && S.tile_above;
    V u[R];
#pragma unroll
    for (int e = 0; e < R; ++e) {
        u[e] = cunit<V>();
    }
    if (use_u) {
#pragma unroll
        for (int e = 0; e < R; ++e) u[e] = U[e];
    }
    int64_t oo[R];
    if (kToGlobal) {
#pragma unroll
        for (int e = 0; e < R; ++e) oo[e] = int64_t(1) << P.p_out[q + e];
    }
    for (int g = threadIdx.x; g < ng; g += NT) {
        const int lo5 = toff + (g & 31), hi5 = toff + 32 + (g >> 5);
        V v[NJ];
        if (kFromA) {
            const uint32_t pb = tab.pb[lo5] | tab.pb[hi5];
#pragma unroll
            for (int j = 0; j < NJ; ++j) v[j] = Tr::load(A, pb + (uint32_t(j) << q), io);
        } else {
            const uint32_t base = tab.sb[lo5] ^ tab.sb[hi5];
#pragma unroll
            for (int j = 0; j < NJ; ++j) v[j] = Bb[base ^ soff[j]];
        }
        if (kFromA && acc_norm) {
            typename Tr::NormAcc a{};
#pragma unroll
            for (int j = 0; j < NJ; ++j) Tr::norm_add(a, v[j]);
            norm_acc += Tr::norm_done(a);
        }
        if (cross) {
            // tau_e for each block wire, then the diagonal prod_e tau_e^{j_e}
            // applied as (low 2 bits) x (high bits) products.
            V tau[R];
#pragma unroll
            for (int e = 0; e < R; ++e) {
                // lane / high table factors that are identically 1 are skipped
                if (S.lo_tw && S.hi_tw) tau[e] = cmul(tab.tw[e * tab.ntab + lo5], tab.tw[e * tab.ntab + hi5]);
                else if (S.lo_tw) tau[e] = tab.tw[e * tab.ntab + lo5];
                else tau[e] = tab.tw[e * tab.ntab + hi5];
                if (use_u) tau[e] = cmul(tau[e], u[e]);
            }
            constexpr int LB = R < 2 ? R : 2;
            constexpr int HB = R - LB;
            V tl[1 << LB], th[1 << HB];
#pragma unroll
            for (int a = 1; a < (1 << LB); ++a)
                tl[a] = (a & (a - 1)) ? cmul(tl[a & (a - 1)], tau[low_bit(a)]) : tau[low_bit(a)];
#pragma unroll
            for (int b = 1; b < (1 << HB); ++b)
                th[b] = (b & (b - 1)) ? cmul(th[b & (b - 1)], tau[LB + low_bit(b)]) : tau[LB + low_bit(b)];
#pragma unroll
            for (int j = 1; j < NJ; ++j) {
                const int a = j & ((1 << LB) - 1), b = j >> LB;
                if (a) v[j] = cmul(v[j], tl[a]);
                if (b) v[j] = cmul(v[j], th[b]);
            }
        }
        block_circuit<DIR, R>(v, P.kk);
        if (kToGlobal) {
            V* __restrict__ out = static_cast<V*>(P.out) + (out_tile + tab.ob[lo5] + tab.ob[hi5]);
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                int64_t o = 0;
#pragma unroll
                for (int e = 0; e < R; ++e)
                    if (j & (1 << e)) o += oo[e];
                Tr::store(out, o, v[j], scale, io);
            }
        } else {
            const uint32_t base = tab.sb[lo5] ^ tab.sb[hi5];
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                Tr::settle(v[j]);
                Bb[base ^ soff[j]] = v[j];
            }
        }
    }
}

template <typename T, int DIR, int KIND, int NT, int MAXR>
__device__ __forceinline__ void dispatch_r(const PassParams& P, int s, const GroupTab<typename Vec2<T>::type>& tab,
                                           const typename Vec2<T>::type* A, typename Vec2<T>::type* Bb,
                                           int64_t out_tile, T scale, const typename Vec2<T>::type* U,
                                           bool acc_norm, double& norm_acc, const AmpIO& io) {
    const StageDesc& S = P.st[s];
    const int toff = P.tab_off[s];
    switch (S.r) {
        case 1: run_stage<T, DIR, 1, KIND, NT>(P, S, tab, toff, A, Bb, out_tile, scale, U, acc_norm, norm_acc, io); break;
        case 2: run_stage<T, DIR, 2, KIND, NT>(P, S, tab, toff, A, Bb, out_tile, scale, U, acc_norm, norm_acc, io); break;
        case 3: run_stage<T, DIR, 3, KIND, NT>(P, S, tab, toff, A, Bb, out_tile, scale, U, acc_norm, norm_acc, io); break;
        case 4:
            if constexpr (MAXR >= 4)
                run_stage<T, DIR, 4, KIND, NT>(P, S, tab, toff, A, Bb, out_tile, scale, U, acc_norm, norm_acc, io);
            break;
        default:
            if constexpr (MAXR >= 5)
                run_stage<T, DIR, 5, KIND, NT>(P, S, tab, toff, A, Bb, out_tile, scale, U, acc_norm, norm_acc, io);
            break;
    }
}

template <typename T, int DIR, int NT, int MAXR>
__device__ __forceinline__ void dispatch_stage(const PassParams& P, int s, const GroupTab<typename Vec2<T>::type>& tab,
                                               const typename Vec2<T>::type* A, typename Vec2<T>::type* Bb,
                                               int64_t out_tile, T scale, const typename Vec2<T>::type* U,
                                               bool acc_norm, double& norm_acc, const AmpIO& io) {
    const bool first = (s == 0), last = (s == P.nstages - 1);
    if (first && last) dispatch_r<T, DIR, K_ONLY, NT, MAXR>(P, s, tab, A, Bb, out_tile, scale, U, acc_norm, norm_acc, io);
    else if (first) dispatch_r<T, DIR, K_FIRST, NT, MAXR>(P, s, tab, A, Bb, out_tile, scale, U, acc_norm, norm_acc, io);
    else if (last) dispatch_r<T, DIR, K_LAST, NT, MAXR>(P, s, tab, A, Bb, out_tile, scale, U, acc_norm, norm_acc, io);
    else dispatch_r<T, DIR, K_MID, NT, MAXR>(P, s, tab, A, Bb, out_tile, scale, U, acc_norm, norm_acc, io);
}

// Widest register stage a kernel shape compiles: 5 wires for complex64 with
// 256 threads and one CTA per SM; 3 where the registers are capped at 128
// per thread with pair-of-pairs amplitudes (double-float with 512 threads, or
// two CTAs per SM) or with 512 threads and two CTAs per SM; 4 otherwise.
template <bool DF, int NT, int MINB>
inline constexpr int kMaxStageWires =
    (NT <= 256 && MINB == 1 && !DF) ? 5 : ((DF && (NT > 256 || MINB == 2)) || (MINB == 2 && NT > 256)) ? 3 : 4;

// MINB = CTAs per SM the launch is built for: 2 caps registers at 65536 / (2 NT)
// and is used only for passes whose stages hold <= 4 wires and whose buffers
// fit twice in shared memory (tiles of <= 2^12 complex64 amplitudes).
template <typename T, int DIR, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    qft_pass_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ PassParams P) {
    using V = typename Vec2<T>::type;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ double red[NT / 32];
    __shared__ __align__(16) V Ubuf[2][kMaxR * kMaxStages];
    using Tr = AmpTraits<T>;
    // double-float: the table of the FP32-only per-tile factors (phase_turns_df)
    __shared__ __align__(16) V t40[Tr::kDF ? 129 : 1];

    const int tid = threadIdx.x;
    const uint32_t tile_elems = 1u << P.tb;
    const uint32_t tile_bytes = tile_elems * static_cast<uint32_t>(sizeof(V));
    // buffer B first, then the two TMA load buffers, then the group tables
    V* B = reinterpret_cast<V*>(smem_raw);
    V* const A0 = B + tile_elems;  // load buffer k & 1 is A0 + (k & 1) * tile_elems
    unsigned char* tab_raw = smem_raw + 3 * static_cast<size_t>(tile_bytes);
    const int ntab = P.ntab;
    GroupTab<V> tab;
    tab.ntab = ntab;
    tab.tw = reinterpret_cast<V*>(tab_raw);
    tab.ob = reinterpret_cast<int64_t*>(tab_raw + P.ntw * sizeof(V) * static_cast<size_t>(ntab));
    tab.pb = reinterpret_cast<uint32_t*>(tab_raw + (P.ntw * sizeof(V) + 8) * static_cast<size_t>(ntab));
    tab.sb = tab.pb + ntab;

    build_group_tables<T, DIR, NT>(P, tab);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
    }
    int64_t tile = blockIdx.x;
    if constexpr (Tr::kDF) {
        build_turns40_table<NT>(t40);
        __syncthreads();
        compute_tile_twiddles_df<DIR>(P, tile, Ubuf[0], t40);
    } else {
        compute_tile_twiddles<T, DIR>(P, tile, Ubuf[0]);
    }
    __syncthreads();

    // Amplitude I/O: the double-float kernel converts the caller's FP64 data
    // in the first pass and back in the last, with its exponent shift.
    AmpIO io{0, 0, 0, 0};
    if constexpr (Tr::kDF) {
        io.raw_in = P.first;
        io.raw_out = P.last;
        io.shift_in = df_shift_from_meta(P.meta);
    }

    // Last pass of a multi-pass plan: scale_in from the first pass's partials
    // (sums of |x 2^-shift|^2 for the double-float kernel).
    T scale = T(1);
    if (P.last && !P.first) {
        double s = 0.0;
        for (int i = tid; i < P.npartials; i += NT) s += P.partials[i];
        const double tot = block_sum<NT>(s, red);
        const double scale_in = Tr::kDF ? ldexp(sqrt(tot), io.shift_in) : sqrt(tot);
        Tr::out_scale(output_factor(P, scale_in), scale, io.shift_out, io.shift_in);
        if (blockIdx.x == 0 && tid == 0) {
            P.meta[0] = scale_in;
            if (P.user_scale) *P.user_scale = scale_in;
        }
    }

    double norm_acc = 0.0;
    uint32_t parity = 0u;  // bit b: phase parity of mbar[b]
    bool aborted = false;
    if (tid == 0 && !P.test_skip_first_load) {
        if (tile < P.num_tiles) issue_tile_load(P, &tmap, tile, A0, &mbar[0], tile_bytes);
        if (tile + gridDim.x < P.num_tiles)
            issue_tile_load(P, &tmap, tile + gridDim.x, A0 + tile_elems, &mbar[1], tile_bytes);
    }

    for (int k = 0; tile < P.num_tiles; tile += gridDim.x, ++k) {
        const int buf = k & 1;
        V* const Ab = A0 + (buf ? tile_elems : 0u);
        uint64_t I_tile;
        int64_t out_tile;
        tile_coords(P, tile, I_tile, out_tile);
        // Each thread waits for the tile on its own; whether any wait gave up is
        // decided CTA-wide at the barrier after the first stage (a thread whose
        // wait failed skips its stage work), which saves one barrier per tile.
        const bool ok = mbar_wait_bounded(&mbar[buf], (parity >> buf) & 1u, P.wait_limit_ns);
        parity ^= 1u << buf;
        if (P.first && P.last) {
            // Single-pass transform (the whole state is this tile): norm first.
            double s = 0.0;
            for (uint32_t i = tid; i < tile_elems; i += NT) s += Tr::norm2_at(Ab, i, io);
            const double tot = block_sum<NT>(s, red);
            const double scale_in = Tr::kDF ? ldexp(sqrt(tot), io.shift_in) : sqrt(tot);
            Tr::out_scale(output_factor(P, scale_in), scale, io.shift_out, io.shift_in);
            if (tid == 0) {
                P.meta[0] = scale_in;
                if (P.user_scale) *P.user_scale = scale_in;
            }
        }
        const V* Ucur = Ubuf[buf];
        for (int s = 0; s < P.nstages; ++s) {
            const bool last_stage = (s == P.nstages - 1);
            const bool from_A = (s == 0);
            if (ok)
                dispatch_stage<T, DIR, NT,
                               kMaxStageWires<Tr::kDF, NT, MINB>>(
                    P, s, tab, Ab, B, out_tile, scale, Ucur + P.st[s].uoff, P.first && !P.last, norm_acc, io);
            if (last_stage) {
                if constexpr (Tr::kDF) compute_tile_twiddles_df<DIR>(P, tile + gridDim.x, Ubuf[buf ^ 1], t40);
                else compute_tile_twiddles<T, DIR>(P, tile + gridDim.x, Ubuf[buf ^ 1]);
            }
            if (from_A) {
                if (__syncthreads_or(!ok)) {
                    aborted = true;
                    parity ^= 1u << buf;  // this tile's phase may not have completed: wait on it again below
                    break;
                }
                // A[buf] is consumed: fetch the tile after next into it.
                const int64_t nt = tile + 2 * static_cast<int64_t>(gridDim.x);
                if (tid == 0 && nt < P.num_tiles) {
                    fence_proxy_async_smem();
                    issue_tile_load(P, &tmap, nt, Ab, &mbar[buf], tile_bytes);
                }
            } else {
                __syncthreads();
            }
        }
        if (aborted) break;
    }

    if (aborted) {
        if (tid == 0) {
            atomicExch(P.status, -5);  // QFT_ERR_TIMEOUT
            // let in-flight copies land before the CTA's shared memory is released
            for (int b = 0; b < 2; ++b) mbar_wait_bounded(&mbar[b], (parity >> b) & 1u, P.wait_limit_ns);
        }
        return;
    }
    if (P.first && !P.last) {
        const double tot = block_sum<NT>(norm_acc, red);
        if (tid == 0) P.partials[blockIdx.x] = tot;
    }
}

template <typename T, int DIR, int NT, int MINB>
inline cudaError_t launch_pass_t(const CUtensorMap& map, const PassParams& P, int grid, size_t smem,
                                 cudaStream_t stream) {
    auto kern = qft_pass_kernel<T, DIR, NT, MINB>;
    {
        const cudaError_t e = ensure_dynamic_smem(kern, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, NT, smem, stream>>>(map, P);
    return cudaGetLastError();
}

}  // namespace qft
