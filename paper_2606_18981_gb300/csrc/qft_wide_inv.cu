// qft_wide_inv.cu -- inverse (DIR = +1) instantiations of the wide pass kernel
// (qft_wide.cuh): top block of R0 in {4, 5} wires, low block of R1 in
// {3, 4, 5} wires, with or without the first-pass store map.  The two
// directions are separate translation units so that they compile in parallel.
#include "qft_wide.cuh"

namespace qft {

cudaError_t launch_wide_inv(int r0, int r1, int top, const CUtensorMap& map, const WideParams& P, int grid,
                           cudaStream_t st) {
    constexpr int D = +1;
#define QFT_WIDE_CASE(A, B)                                                                              \
    if (r0 == A && r1 == B)                                                                              \
        return top ? launch_wide_t<D, A, B, true>(map, P, grid, st) : launch_wide_t<D, A, B, false>(map, P, grid, st);
    QFT_WIDE_CASE(5, 5)
    QFT_WIDE_CASE(5, 4)
    QFT_WIDE_CASE(5, 3)
    QFT_WIDE_CASE(4, 5)
    QFT_WIDE_CASE(4, 4)
    QFT_WIDE_CASE(4, 3)
#undef QFT_WIDE_CASE
    return cudaErrorInvalidValue;
}

}  // namespace qft
