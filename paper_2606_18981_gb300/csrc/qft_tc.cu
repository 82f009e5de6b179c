// qft_tc.cu -- host side of the precision tier (kernels in qft_tc.cuh): the
// fast-path test, shared-memory sizes, the launch dispatch (the kernels of
// each direction are instantiated in qft_tc_fwd.cu / qft_tc_inv.cu) and the
// rounding of the block matrices into the operand formats.
#include "qft_tc.cuh"

namespace qft {

bool tc_fast_pass(const PassParams& P) { return tc_fast_ok(P); }

size_t tc_smem_bytes(const PassParams& P, int prec, int kpad, int ncols) {
    if (tc_fast_ok(P)) {
        switch (prec) {
            case TC_TF32: return tc_fast_smem<TC_TF32>(P);
            case TC_BF16: return tc_fast_smem<TC_BF16>(P);
            case TC_BF16X3: return tc_fast_smem<TC_BF16X3>(P);
            case TC_FP16: return tc_fast_smem<TC_FP16>(P);
            default: return tc_fast_smem<TC_FP16X3>(P);
        }
    }
    const int eb = prec == TC_TF32 ? 4 : 2;
    const bool split = prec == TC_BF16X3 || prec == TC_FP16X3;
    const size_t tile = (size_t(1) << P.tb) * 8;
    const size_t dst = size_t(2) * (size_t(1) << P.st[0].r) * ncols * 4;
    const size_t stage = tile > dst ? tile : dst;
    const size_t a = size_t(128) * kpad * eb * (split ? 2 : 1);
    const size_t b = size_t(ncols) * kpad * eb * (split ? 2 : 1);
    return stage + a + b + 4 * 256 + size_t(P.ntab) * (kMaxR * 8 + 8 + 4 + 4);
}

cudaError_t launch_tc_pass(int dir, int prec, const CUtensorMap& map, const PassParams& P, const void* a_hi,
                           const void* a_lo, int kpad, int ncols, int grid, size_t smem, cudaStream_t st) {
    TcParams Q;
    Q.a_hi = a_hi;
    Q.a_lo = a_lo;
    Q.kpad = kpad;
    Q.ncols = ncols;
    return dir < 0 ? launch_tc_dir<-1>(prec, map, P, Q, grid, smem, st) : launch_tc_dir<+1>(prec, map, P, Q, grid, smem, st);
}

// Round the FP64 real block matrix (128 x kpad, row-major) into the operand
// format, split into hi and lo, in the shared-memory operand layout.
template <int PREC>
__global__ void tc_prepare_a_kernel(const double* src, unsigned char* hi, unsigned char* lo, int kpad) {
    constexpr int EB = TcOp<PREC>::bytes;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 128 * kpad; i += gridDim.x * blockDim.x) {
        const int row = i / kpad, k = i % kpad;
        const double x = src[i];
        const float h = store_op<PREC>(hi + op_offset<EB>(row, k, kpad), static_cast<float>(x));
        store_op<PREC>(lo + op_offset<EB>(row, k, kpad), static_cast<float>(x - static_cast<double>(h)));
    }
}

cudaError_t tc_prepare_a(int prec, const double* d_src, void* d_hi, void* d_lo, int kpad, cudaStream_t st) {
    unsigned char* hi = static_cast<unsigned char*>(d_hi);
    unsigned char* lo = static_cast<unsigned char*>(d_lo);
    switch (prec) {
        case TC_TF32: tc_prepare_a_kernel<TC_TF32><<<64, 256, 0, st>>>(d_src, hi, lo, kpad); break;
        case TC_BF16: tc_prepare_a_kernel<TC_BF16><<<64, 256, 0, st>>>(d_src, hi, lo, kpad); break;
        case TC_BF16X3: tc_prepare_a_kernel<TC_BF16X3><<<64, 256, 0, st>>>(d_src, hi, lo, kpad); break;
        case TC_FP16: tc_prepare_a_kernel<TC_FP16><<<64, 256, 0, st>>>(d_src, hi, lo, kpad); break;
        default: tc_prepare_a_kernel<TC_FP16X3><<<64, 256, 0, st>>>(d_src, hi, lo, kpad); break;
    }
    return cudaGetLastError();
}

}  // namespace qft
