// qft_tc_fwd.cu -- the precision tier's kernels for the forward direction
// (templates in qft_tc.cuh), in a translation unit of their own.
#include "qft_tc.cuh"

namespace qft {
template cudaError_t launch_tc_dir<-1>(int, const CUtensorMap&, const PassParams&, const TcParams&, int, size_t,
                                        cudaStream_t);
}  // namespace qft
