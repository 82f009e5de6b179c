// plan_host.hpp -- host-side plan structures shared by the C ABI files
// (qftfft_api.cpp, qft_batch.cpp).  Internal to libqftfft.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "plan.hpp"

namespace qft {

cudaError_t launch_pass(int dtype, int dir, int threads, int minb, const CUtensorMap& map, const PassParams& P,
                        int grid, size_t smem, cudaStream_t stream);
size_t pass_smem_bytes(const PassParams& P, size_t elem_bytes);
cudaError_t launch_pass_p(int dir, int minb, const CUtensorMap& map, const PassParams& P, int grid, size_t smem,
                          cudaStream_t stream);
cudaError_t launch_pass_wide(int dir, int r0, int r1, int top, const CUtensorMap& map, const WideParams& P, int grid,
                             cudaStream_t stream);
cudaError_t launch_pass_wide_group(int dir, int r0, int r1, int top, const WideParams& P, int grid,
                                   cudaStream_t stream);
constexpr size_t kWideSmem = 215032;  // dynamic shared memory of the wide kernel (checked in qft_wide_fwd.cu)
cudaError_t launch_pass_df(int dir, int threads, int minb, const CUtensorMap& map, const PassParams& P, int grid,
                           size_t smem, cudaStream_t stream);
cudaError_t launch_df_maxexp(const void* state, size_t n_amps, int* out, int num_sms, cudaStream_t stream);
cudaError_t launch_tc_pass(int dir, int prec, const CUtensorMap& map, const PassParams& P, const void* a_hi,
                           const void* a_lo, int kpad, int ncols, int grid, size_t smem, cudaStream_t st);
size_t tc_smem_bytes(const PassParams& P, int prec, int kpad, int ncols);
// true when the pass runs on the fast tensor-core kernel (the only one for 7-wire blocks)
bool tc_fast_pass(const PassParams& P);
cudaError_t tc_prepare_a(int prec, const double* d_src, void* d_hi, void* d_lo, int kpad, cudaStream_t st);

// Workspace layout of one transform: [0, 4096) metadata (scale_in at 0,
// status word at 8, norm partial sums from 64); the ping-pong state buffer
// from 4096.
constexpr size_t kMetaBytes = 4096;
constexpr size_t kStatusOff = 8;
constexpr size_t kMaxExpOff = 16;  // double-float plans: largest biased FP64 exponent of the input (int)
constexpr size_t kPartialOff = 64;
constexpr int kMaxPartials = (kMetaBytes - kPartialOff) / 8;

struct PassHost {
    PassParams prm;
    int in_buf = 0, out_buf = 0;  // 0 = caller's state, 1 = workspace ping-pong buffer
    int grid = 1;
    int minb = 1;  // CTAs per SM the pass kernel is built for (2: tiles <= 2^12, stages <= 4 wires)
    size_t smem = 0;
    // TMA description
    int rank = 5;
    cuuint64_t gdim[5];
    cuuint64_t gstride[4];
    cuuint32_t box[5];
    int wires = 0;
    int run_bits = 0;  // low input address bits inside the tile (log2 amplitudes per HBM run)
    // wide pass (complex64, 2^14-amplitude tiles, qft_wide.cuh): block split and
    // launch parameters; its tensor map uses the 128-byte swizzle
    int wide = 0, wide_r0 = 0, wide_r1 = 0, wide_top = 0;
    WideParams wp{};
    // tensor-core tier: the pass's block matrix in operand format (plan-owned device memory)
    void* tc_a_hi = nullptr;
    void* tc_a_lo = nullptr;
    int tc_kpad = 0, tc_ncols = 0;
};

int set_cuda_error(cudaError_t e);           // records e for qft_last_cuda_error, returns QFT_ERR_CUDA

void set_cuda_error_code(int e);
PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn();

}  // namespace qft

struct qft_plan_s {
    ~qft_plan_s() {
        for (auto& ph : passes) {
            if (ph.tc_a_hi) cudaFree(ph.tc_a_hi);
            if (ph.tc_a_lo) cudaFree(ph.tc_a_lo);
        }
    }
    int precision = 0;  // QFT_PREC_* (tensor-core tiers; QFT_PREC_FP64 is kept in fp64 below)
    bool df = false;    // complex128 in double-float arithmetic (the default for complex128)
    int n = 0, k = -1, kk = 0, dir = -1, dtype = 0, order = 0;
    // Subset plans: the QFT acts on index bits [w0, w0 + n) of an array of
    // 2^n_addr amplitudes, once for every value of the other bits.  Ordinary
    // plans have n_addr = n and w0 = 0.
    int n_addr = 0, w0 = 0;
    size_t esize = 8;
    int TB = 13, cmin = 2, rmax = 4;
    int threads = 256;  // CTA size of the pass kernel (256: stages of <= 5 wires; 512: <= 4)
    int pass_split = 0;    // qft_opts.pass_split
    int wide_tiles = 0;    // complex64 natural order on the wide pass kernel (2^14-amplitude tiles)
    int l2_prefetch = 0;   // wide passes: also prefetch the tile after next into L2
    bool shape_given = false;  // the caller fixed the tile shape (tile_bits, coalesce_bits, threads, max_stage_bits)
    uint64_t wait_limit_ns = 2000000000ull;
    int test_skip_first_load = 0;
    int num_sms = 148;
    long long n_h = 0, n_cp = 0, n_swap = 0;
    std::vector<qft::PassHost> passes;
    size_t ws_bytes = 0;
    // tensor maps for the last (state, workspace) pointer pair
    std::mutex mu;
    const void* map_in = nullptr;
    const void* map_state = nullptr;
    const void* map_work = nullptr;
    std::vector<CUtensorMap> maps;
};

namespace qft {
// True when executing the plan will not allocate device memory: every plan
// except a tensor-core tier plan whose block matrices have not been uploaded
// yet (its first qft_execute does that).
bool plan_device_ready(const qft_plan_s* pl);
}  // namespace qft
