// qft_pass_f64.cu -- complex128 instantiations of the pass kernel
// (qft_pass_kernels.cuh): 256 or 512 threads, one CTA per SM, both directions.
#include "qft_pass_kernels.cuh"

namespace qft {

cudaError_t launch_pass_f64(int dir, int threads, const CUtensorMap& map, const PassParams& P, int grid, size_t smem, cudaStream_t stream) {
    if (threads == 512)
        return dir < 0 ? launch_pass_t<double, -1, 512, 1>(map, P, grid, smem, stream)
                       : launch_pass_t<double, +1, 512, 1>(map, P, grid, smem, stream);
    return dir < 0 ? launch_pass_t<double, -1, 256, 1>(map, P, grid, smem, stream)
                   : launch_pass_t<double, +1, 256, 1>(map, P, grid, smem, stream);
}

}  // namespace qft
