// qft_pass.cu -- host-side dispatch of the pass and batch kernels to their
// per-dtype instantiations, and the shared-memory sizes of both kernels.
// The kernels themselves are templates in qft_pass_kernels.cuh.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "plan.hpp"

namespace qft {

cudaError_t launch_pass_f32(int dir, int threads, int minb, const CUtensorMap& map, const PassParams& P, int grid, size_t smem, cudaStream_t stream);
cudaError_t launch_pass_f64(int dir, int threads, const CUtensorMap& map, const PassParams& P, int grid, size_t smem, cudaStream_t stream);
cudaError_t launch_batch_f32(int dir, int minb, const BatchItem* items, int nitems, const PassParams* descs, const CUtensorMap* maps, int* counters,
                             int* next, int* status, uint64_t wait_ns, BatchLayout lay, int grid, size_t smem,
                             cudaStream_t stream);
cudaError_t launch_batch_f64(int dir, const BatchItem* items, int nitems, const PassParams* descs, const CUtensorMap* maps, int* counters,
                             int* next, int* status, uint64_t wait_ns, BatchLayout lay, int grid, size_t smem,
                             cudaStream_t stream);

// minb = 2: complex64 batches whose tiles are <= 2^12 amplitudes and whose
// blocks have <= 4 wires run two CTAs per SM (one CTA's load overlaps the
// other's stages).
cudaError_t launch_batch(int dtype, int dir, int minb, const BatchItem* items, int nitems, const PassParams* descs, const CUtensorMap* maps, int* counters,
                             int* next, int* status, uint64_t wait_ns, BatchLayout lay, int grid, size_t smem,
                             cudaStream_t stream) {
    if (dtype == 0) return launch_batch_f32(dir, minb, items, nitems, descs, maps, counters, next, status, wait_ns, lay, grid, smem, stream);
    return launch_batch_f64(dir, items, nitems, descs, maps, counters, next, status, wait_ns, lay, grid, smem, stream);
}

// Dynamic shared memory of one batch CTA: buffer B, the load buffers of the
// largest tile, and the group tables (twiddle planes, output offset, tile bits
// and their swizzled buffer-B offset per entry).
size_t batch_smem_bytes(BatchLayout lay, size_t elem_bytes) {
    return (1 + size_t(lay.nbuf)) * (size_t(1) << lay.max_tb) * elem_bytes +
           size_t(lay.max_ntab) * (size_t(lay.tw_stride) + 8 + 4 + 4);
}

cudaError_t launch_pass(int dtype, int dir, int threads, int minb, const CUtensorMap& map, const PassParams& P, int grid, size_t smem, cudaStream_t stream) {
    if (dtype == 0) return launch_pass_f32(dir, threads, minb, map, P, grid, smem, stream);
    return launch_pass_f64(dir, threads, map, P, grid, smem, stream);
}

// Dynamic shared memory of one CTA: buffer B, the two TMA load buffers and
// the group tables (ntw twiddle factors + output offset + tile bits + their
// swizzled buffer-B offset per entry).
size_t pass_smem_bytes(const PassParams& P, size_t elem_bytes) {
    return 3 * (size_t(1) << P.tb) * elem_bytes + size_t(P.ntab) * (P.ntw * elem_bytes + 8 + 4 + 4);
}

}  // namespace qft

namespace qft {

cudaError_t launch_wide_fwd(int r0, int r1, int top, const CUtensorMap& map, const WideParams& P, int grid,
                            cudaStream_t st);
cudaError_t launch_wide_inv(int r0, int r1, int top, const CUtensorMap& map, const WideParams& P, int grid,
                            cudaStream_t st);
cudaError_t launch_wide_group_fwd(int r0, int r1, int top, const CUtensorMap& map, const WideParams& P, int grid,
                                  cudaStream_t st);
cudaError_t launch_wide_group_inv(int r0, int r1, int top, const CUtensorMap& map, const WideParams& P, int grid,
                                  cudaStream_t st);

// The wide pass kernel (qft_wide.cuh) for one direction and block split.
cudaError_t launch_pass_wide(int dir, int r0, int r1, int top, const CUtensorMap& map, const WideParams& P, int grid,
                             cudaStream_t stream) {
    return dir < 0 ? launch_wide_fwd(r0, r1, top, map, P, grid, stream)
                   : launch_wide_inv(r0, r1, top, map, P, grid, stream);
}

// The same in group mode (P.maps, P.outs, P.tpart set; map unused).
cudaError_t launch_pass_wide_group(int dir, int r0, int r1, int top, const WideParams& P, int grid,
                                   cudaStream_t stream) {
    static const CUtensorMap unused{};
    return dir < 0 ? launch_wide_group_fwd(r0, r1, top, unused, P, grid, stream)
                   : launch_wide_group_inv(r0, r1, top, unused, P, grid, stream);
}

}  // namespace qft
