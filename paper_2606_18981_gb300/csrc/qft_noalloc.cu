// qft_noalloc.cu -- qft_execute for callers that cannot allocate device memory.
//
// qft_execute needs a caller-allocated workspace (scale_in, the status word,
// the per-CTA norm partial sums and, for natural-order multi-pass plans, an
// N-amplitude ping-pong buffer).  Some callers cannot provide one: code that
// runs while a CUDA stream is being captured into a graph (cudaMalloc is not
// allowed during capture), host runtimes that own the device heap and expose
// no allocator to libraries, and latency-critical loops that must never enter
// an allocator.  qft_execute_noalloc serves them from a fixed scratch array
// that lives in this library's device image instead.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes
// (32 MiB + 4 KiB): every GPU that loads the library holds it until the
// process exits.  Host code must not use the symbol as a pointer (it is a
// host-side stand-in); its device address is looked up once per device with
// cudaGetSymbolAddress while that device is current, on the first call made
// on that device, and cached.  That first call therefore should come before
// any stream capture.  All calls share the one array and it keeps the last
// call's contents; the execute path clears the status word itself and fully
// rewrites the partial sums before reading them.  Calls whose kernels overlap
// on the GPU (different streams, or different host threads) race on the array.
//
// Tensor-core tier plans upload their block matrices (device memory they
// allocate) on their first qft_execute; until that has happened this entry
// point refuses them (QFT_ERR_UNSUPPORTED) rather than allocate.  A bounded
// wait that expires writes QFT_ERR_TIMEOUT into the scratch's status word,
// which qft_noalloc_status reads back.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "../../include/qftfft.h"
#include "plan_host.hpp"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t(32) << 20) + 4096;
static_assert(qft::kMetaBytes == 4096 && qft::kStatusOff == 8, "scratch layout follows the workspace's");

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per device).
int scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return QFT_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return QFT_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return QFT_OK;
}

}  // namespace

extern "C" {

int qft_execute_noalloc(qft_plan_t plan, void* d_state, double* d_scale_in, int scale_mode, qft_stream_t stream) {
    if (!plan || !d_state) return QFT_ERR_BAD_ARG;
    if (qft_workspace_size(plan) > kNoAllocScratchBytes) return QFT_ERR_SIZE;
    if (!qft::plan_device_ready(plan)) return QFT_ERR_UNSUPPORTED;  // its first execute would allocate
    void* scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc != QFT_OK) return rc;
    return qft_execute(plan, d_state, scratch, d_scale_in, scale_mode, stream);
}

int qft_noalloc_status(qft_stream_t stream) {
    void* scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc != QFT_OK) return rc;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    int32_t status = 0;
    if (e == cudaSuccess)
        e = cudaMemcpy(&status, static_cast<const char*>(scratch) + qft::kStatusOff, sizeof(status),
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return QFT_ERR_CUDA;
    }
    return status;
}

}  // extern "C"
