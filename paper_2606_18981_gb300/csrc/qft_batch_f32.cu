// qft_batch_f32.cu -- complex64 instantiations of the batched persistent
// kernel (qft_batch_kernel.cuh): 256 threads with one or two CTAs per SM, or
// 512 threads with one, both directions.
#include "qft_batch_kernel.cuh"

namespace qft {

cudaError_t launch_batch_f32(int dir, int minb, const BatchItem* items, int nitems, const PassParams* descs, const CUtensorMap* maps, int* counters,
                             int* next, int* status, uint64_t wait_ns, BatchLayout lay, int grid, size_t smem,
                             cudaStream_t stream) {
    if (minb == 2)
        return dir < 0 ? launch_batch_t<float, -1, 256, 2>(items, nitems, descs, maps, counters, next, status, wait_ns, lay, grid, smem, stream)
                       : launch_batch_t<float, +1, 256, 2>(items, nitems, descs, maps, counters, next, status, wait_ns, lay, grid, smem, stream);
    if (lay.threads == 512)
        return dir < 0 ? launch_batch_t<float, -1, 512, 1>(items, nitems, descs, maps, counters, next, status, wait_ns, lay, grid, smem, stream)
                       : launch_batch_t<float, +1, 512, 1>(items, nitems, descs, maps, counters, next, status, wait_ns, lay, grid, smem, stream);
    return dir < 0 ? launch_batch_t<float, -1, 256, 1>(items, nitems, descs, maps, counters, next, status, wait_ns, lay, grid, smem, stream)
                   : launch_batch_t<float, +1, 256, 1>(items, nitems, descs, maps, counters, next, status, wait_ns, lay, grid, smem, stream);
}

}  // namespace qft
