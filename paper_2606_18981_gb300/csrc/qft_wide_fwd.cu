// qft_wide_fwd.cu -- forward (DIR = -1) instantiations of the wide pass kernel
// (qft_wide.cuh): top block of R0 in {4, 5} wires, low block of R1 in
// {3, 4, 5} wires, with or without the first-pass store map.  Each direction
// and mode is its own translation unit so that they compile in parallel.
#include "qft_wide.cuh"

#include "plan_host.hpp"

namespace qft {

static_assert(kWideSmem == kWideSmemBytes, "planner and kernel disagree on the wide kernel's shared memory");

cudaError_t launch_wide_fwd(int r0, int r1, int top, const CUtensorMap& map, const WideParams& P, int grid,
                           cudaStream_t st) {
    return launch_wide_dir<-1, false>(r0, r1, top, map, P, grid, st);
}

}  // namespace qft
