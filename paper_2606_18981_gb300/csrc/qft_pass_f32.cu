// qft_pass_f32.cu -- complex64 instantiations of the pass kernel
// (qft_pass_kernels.cuh): 256 threads with one or two CTAs per SM, or 512
// threads with one, for both directions.
#include "qft_pass_kernels.cuh"

namespace qft {

cudaError_t launch_pass_f32(int dir, int threads, int minb, const CUtensorMap& map, const PassParams& P, int grid, size_t smem, cudaStream_t stream) {
    if (minb == 2 && threads == 256)
        return dir < 0 ? launch_pass_t<float, -1, 256, 2>(map, P, grid, smem, stream)
                       : launch_pass_t<float, +1, 256, 2>(map, P, grid, smem, stream);
    if (threads == 512)
        return dir < 0 ? launch_pass_t<float, -1, 512, 1>(map, P, grid, smem, stream)
                       : launch_pass_t<float, +1, 512, 1>(map, P, grid, smem, stream);
    return dir < 0 ? launch_pass_t<float, -1, 256, 1>(map, P, grid, smem, stream)
                   : launch_pass_t<float, +1, 256, 1>(map, P, grid, smem, stream);
}

}  // namespace qft
