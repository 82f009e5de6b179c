// qft_pass_df2.cu -- the double-float pass kernel in its two-CTAs-per-SM
// shape (256 threads, blocks of <= 3 wires within 128 registers, tiles whose
// three buffers fit twice into an SM's shared memory); its own translation
// unit so that it compiles beside the other instantiations.
#include "qft_pass_kernels.cuh"

namespace qft {

cudaError_t launch_pass_df_minb2(int dir, const CUtensorMap& map, const PassParams& P, int grid, size_t smem,
                                 cudaStream_t stream) {
    return dir < 0 ? launch_pass_t<dfloat, -1, 256, 2>(map, P, grid, smem, stream)
                   : launch_pass_t<dfloat, +1, 256, 2>(map, P, grid, smem, stream);
}

}  // namespace qft
