// qft_pass_df.cu -- the double-float complex128 pass kernel (qft_pass_kernels.cuh
// instantiated with T = dfloat, arithmetic in qft_df.cuh) and the
// maximum-exponent pre-pass of its range normalisation (single transforms and
// batches; the batch kernel itself is instantiated in qft_batch_df.cu).
//
// A complex128 transform on this path reads the caller's FP64 state in its
// first pass, converts each component to an FP32 pair scaled by 2^-k, keeps
// 16-byte pairs in the workspace between passes (the same footprint as
// double2), and converts back to FP64 times 2^k in its last pass.  k is the
// largest binary exponent of the input, found by qft_df_maxexp_kernel before
// the first pass and left in the workspace metadata (int at byte 16).
#include "qft_pass_kernels.cuh"

namespace qft {

// Largest biased FP64 exponent over the real and imaginary parts of n2
// doubles, atomically max-combined into *out (which the caller zeroes).
__global__ void __launch_bounds__(256) qft_df_maxexp_kernel(const uint4* __restrict__ x, size_t n16, int* out) {
    uint32_t m = 0;
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n16; i += size_t(gridDim.x) * blockDim.x) {
        const uint4 v = x[i];  // two doubles: high words in .y and .w
        m = max(m, max((v.y >> 20) & 0x7FFu, (v.w >> 20) & 0x7FFu));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, static_cast<int>(m));
}

cudaError_t launch_df_maxexp(const void* state, size_t n_amps, int* out, int num_sms, cudaStream_t stream) {
    const size_t n16 = n_amps * 2 / 2;  // one 16-byte load per complex128 amplitude
    size_t blocks = (n16 + 255) / 256;
    const size_t cap = size_t(num_sms) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    qft_df_maxexp_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(static_cast<const uint4*>(state), n16, out);
    return cudaGetLastError();
}

cudaError_t launch_pass_df_minb2(int dir, const CUtensorMap& map, const PassParams& P, int grid, size_t smem,
                                 cudaStream_t stream);

// 256 threads: blocks of <= 4 wires, up to 255 registers, 8 warps per SM; or
// (minb = 2) blocks of <= 3 wires within 128 registers, two CTAs per SM.
// 512 threads: blocks of <= 3 wires within 128 registers, 16 warps per SM.
cudaError_t launch_pass_df(int dir, int threads, int minb, const CUtensorMap& map, const PassParams& P, int grid,
                           size_t smem, cudaStream_t stream) {
    if (threads == 256 && minb == 2) return launch_pass_df_minb2(dir, map, P, grid, smem, stream);
    if (threads == 512)
        return dir < 0 ? launch_pass_t<dfloat, -1, 512, 1>(map, P, grid, smem, stream)
                       : launch_pass_t<dfloat, +1, 512, 1>(map, P, grid, smem, stream);
    return dir < 0 ? launch_pass_t<dfloat, -1, 256, 1>(map, P, grid, smem, stream)
                   : launch_pass_t<dfloat, +1, 256, 1>(map, P, grid, smem, stream);
}

// Batches of double-float transforms: zero each transform's maximum-exponent
// word, then take every transform's maximum in one launch (grid.y = transform).
__global__ void qft_df_zero_list_kernel(int* const* __restrict__ outs, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) *outs[i] = 0;
}

__global__ void __launch_bounds__(256) qft_df_maxexp_list_kernel(const uint4* const* __restrict__ states,
                                                               const uint64_t* __restrict__ n16,
                                                               int* const* __restrict__ outs) {
    const int t = blockIdx.y;
    const uint4* x = states[t];
    const uint64_t n = n16[t];
    uint32_t m = 0;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < n; i += uint64_t(gridDim.x) * blockDim.x) {
        const uint4 v = x[i];
        m = max(m, max((v.y >> 20) & 0x7FFu, (v.w >> 20) & 0x7FFu));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(outs[t], static_cast<int>(m));
}

cudaError_t launch_df_maxexp_list(const void* const* d_states, const uint64_t* d_n16, int* const* d_outs, int count,
                                  uint64_t max_n16, int num_sms, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    qft_df_zero_list_kernel<<<(count + 255) / 256, 256, 0, stream>>>(d_outs, count);
    uint64_t bx = (max_n16 + 255) / 256;
    const uint64_t cap = (uint64_t(num_sms) * 8 + count - 1) / count;  // about 8 blocks per SM in all
    if (bx > cap) bx = cap;
    if (bx < 1) bx = 1;
    dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(count));
    qft_df_maxexp_list_kernel<<<grid, 256, 0, stream>>>(reinterpret_cast<const uint4* const*>(d_states), d_n16,
                                                         d_outs);
    return cudaGetLastError();
}

}  // namespace qft
