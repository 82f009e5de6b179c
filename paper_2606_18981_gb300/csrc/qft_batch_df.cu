// qft_batch_df.cu -- double-float complex128 instantiations of the batched
// persistent kernel (qft_batch_kernel.cuh): one CTA per SM of 256 or 512
// threads, both directions.
// The maximum-exponent pre-pass over the batch's transforms is in
// qft_pass_df.cu.
#include "qft_batch_kernel.cuh"

namespace qft {

cudaError_t launch_batch_df(int dir, const BatchItem* items, int nitems, const PassParams* descs,
                            const CUtensorMap* maps, int* counters, int* next, int* status, uint64_t wait_ns,
                            BatchLayout lay, int grid, size_t smem, cudaStream_t stream) {
    if (lay.threads == 512)
        return dir < 0 ? launch_batch_t<dfloat, -1, 512, 1>(items, nitems, descs, maps, counters, next, status,
                                                            wait_ns, lay, grid, smem, stream)
                       : launch_batch_t<dfloat, +1, 512, 1>(items, nitems, descs, maps, counters, next, status,
                                                            wait_ns, lay, grid, smem, stream);
    return dir < 0 ? launch_batch_t<dfloat, -1, 256, 1>(items, nitems, descs, maps, counters, next, status, wait_ns,
                                                        lay, grid, smem, stream)
                   : launch_batch_t<dfloat, +1, 256, 1>(items, nitems, descs, maps, counters, next, status, wait_ns,
                                                        lay, grid, smem, stream);
}

}  // namespace qft
