// qft_batch_f64.cu -- complex128 instantiations of the batched persistent
// kernel (qft_batch_kernel.cuh): one CTA per SM, both directions.
#include "qft_batch_kernel.cuh"

namespace qft {

cudaError_t launch_batch_f64(int dir, const BatchItem* items, int nitems, const PassParams* descs, const CUtensorMap* maps, int* counters,
                             int* next, int* status, uint64_t wait_ns, BatchLayout lay, int grid, size_t smem,
                             cudaStream_t stream) {
    return dir < 0 ? launch_batch_t<double, -1, 256, 1>(items, nitems, descs, maps, counters, next, status, wait_ns, lay, grid, smem, stream)
                   : launch_batch_t<double, +1, 256, 1>(items, nitems, descs, maps, counters, next, status, wait_ns, lay, grid, smem, stream);
}

}  // namespace qft
