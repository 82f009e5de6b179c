// qft_pair.cu -- the paired pass kernel for complex64 (see qft_pair.cuh).
//
// Same pipeline as qft_pass_kernel (qft_pass.cu): a persistent CTA per SM,
// tiles fetched by TMA into two alternating load buffers, register stages
// through the swizzled buffer B, the last stage storing straight to HBM with
// the pass's output map and output scale.  What differs is the stage: every
// thread runs two groups (tile bit 0 = 0 and 1) with packed f32x2 arithmetic,
// so a 2^tb-amplitude tile is 2^(tb-1) pair units and the planner limits
// blocks to four wires (16 pairs = 64 registers of amplitudes per thread).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "plan.hpp"
#include "qft_pair.cuh"

namespace qft {

// MINB = 2: two CTAs per SM (registers capped at 128, blocks of <= 3 wires).
template <int DIR, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    qft_pass_p_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ PassParams P) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ double red[NT / 32];
    __shared__ __align__(16) P2 Ubuf[2][kMaxR * kMaxStages];

    const int tid = threadIdx.x;
    const uint32_t tile_elems = 1u << P.tb;
    const uint32_t tile_bytes = tile_elems * static_cast<uint32_t>(sizeof(float2));
    // buffer B (pair units) first, then the two TMA load buffers, then the group tables
    P2* B = reinterpret_cast<P2*>(smem_raw);
    float2* const A0 = reinterpret_cast<float2*>(smem_raw + tile_bytes);
    unsigned char* tab_raw = smem_raw + 3 * static_cast<size_t>(tile_bytes);
    const int ntab = P.ntab;
    GroupTabP tab;
    tab.ntab = ntab;
    tab.tw = reinterpret_cast<P2*>(tab_raw);
    tab.ob = reinterpret_cast<int64_t*>(tab_raw + P.ntw * sizeof(P2) * static_cast<size_t>(ntab));
    tab.pb = reinterpret_cast<uint32_t*>(tab_raw + (P.ntw * sizeof(P2) + 8) * static_cast<size_t>(ntab));
    build_group_tables_p<DIR, NT>(P, tab);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
    }
    int64_t tile = blockIdx.x;
    compute_tile_twiddles_p<DIR>(P, tile, Ubuf[0]);
    __syncthreads();

    float scale = 1.f;
    if (P.last) {  // a paired pass never is the only pass: scale_in comes from the first pass's partials
        double s = 0.0;
        for (int i = tid; i < P.npartials; i += NT) s += P.partials[i];
        const double tot = block_sum<NT>(s, red);
        const double scale_in = sqrt(tot);
        scale = static_cast<float>(output_factor(P, scale_in));
        if (blockIdx.x == 0 && tid == 0) {
            P.meta[0] = scale_in;
            if (P.user_scale) *P.user_scale = scale_in;
        }
    }

    double norm_acc = 0.0;
    uint32_t parity = 0u;
    bool aborted = false;
    if (tid == 0 && !P.test_skip_first_load) {
        if (tile < P.num_tiles) issue_tile_load(P, &tmap, tile, A0, &mbar[0], tile_bytes);
        if (tile + gridDim.x < P.num_tiles)
            issue_tile_load(P, &tmap, tile + gridDim.x, A0 + tile_elems, &mbar[1], tile_bytes);
    }

    for (int k = 0; tile < P.num_tiles; tile += gridDim.x, ++k) {
        const int buf = k & 1;
        float2* const Ab = A0 + (buf ? tile_elems : 0u);
        uint64_t I_tile;
        int64_t out_tile;
        tile_coords(P, tile, I_tile, out_tile);
        const bool ok = mbar_wait_bounded(&mbar[buf], (parity >> buf) & 1u, P.wait_limit_ns);
        parity ^= 1u << buf;
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        const P2* Ucur = Ubuf[buf];
        for (int s = 0; s < P.nstages; ++s) {
            const bool last_stage = (s == P.nstages - 1);
            dispatch_stage_p<DIR, NT, MINB == 1 ? 4 : 3>(P, s, tab, Ab, B, out_tile, scale, Ucur + P.st[s].uoff,
                                                         P.first != 0, norm_acc);
            if (last_stage) compute_tile_twiddles_p<DIR>(P, tile + gridDim.x, Ubuf[buf ^ 1]);
            __syncthreads();
            if (s == 0) {
                const int64_t nt = tile + 2 * static_cast<int64_t>(gridDim.x);
                if (tid == 0 && nt < P.num_tiles) {
                    fence_proxy_async_smem();
                    issue_tile_load(P, &tmap, nt, Ab, &mbar[buf], tile_bytes);
                }
            }
        }
    }

    if (aborted) {
        if (tid == 0) {
            atomicExch(P.status, -5);  // QFT_ERR_TIMEOUT
            for (int b = 0; b < 2; ++b) mbar_wait_bounded(&mbar[b], (parity >> b) & 1u, P.wait_limit_ns);
        }
        return;
    }
    if (P.first) {
        const double tot = block_sum<NT>(norm_acc, red);
        if (tid == 0) P.partials[blockIdx.x] = tot;
    }
}

template <int DIR, int MINB>
static cudaError_t launch_pass_p_t(const CUtensorMap& map, const PassParams& P, int grid, size_t smem,
                                   cudaStream_t stream) {
    auto kern = qft_pass_p_kernel<DIR, 256, MINB>;
    {
        const cudaError_t e = ensure_dynamic_smem(kern, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, 256, smem, stream>>>(map, P);
    return cudaGetLastError();
}

cudaError_t launch_pass_p(int dir, int minb, const CUtensorMap& map, const PassParams& P, int grid, size_t smem,
                          cudaStream_t stream) {
    if (minb == 2)
        return dir < 0 ? launch_pass_p_t<-1, 2>(map, P, grid, smem, stream)
                       : launch_pass_p_t<+1, 2>(map, P, grid, smem, stream);
    return dir < 0 ? launch_pass_p_t<-1, 1>(map, P, grid, smem, stream)
                   : launch_pass_p_t<+1, 1>(map, P, grid, smem, stream);
}

}  // namespace qft
