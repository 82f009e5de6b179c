// qft_batch.cpp -- batched execution: many transforms of different sizes and
// cutoffs in one persistent launch of qft_batch_kernel (see qft_pass.cu).
//
// qft_batch_create binds each transform (a plan and its device state) once:
// it copies the plan's pass descriptors with the transform's buffers filled
// in, encodes a TMA tensor map per strided pass, lays out the per-transform
// workspace (scale_in, norm partial sums, ping-pong buffer) inside the
// caller's batch workspace, and builds the ordered work list (one item per
// tile per pass, transform by transform, with completion counters between a
// transform's passes).  These tables live in device memory owned by the
// batch object.  qft_batch_execute is then two memsets and one kernel launch
// on the caller's stream, so it can be captured into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/qftfft.h"
#include "batch_order.hpp"
#include "plan_host.hpp"

namespace qft {
cudaError_t launch_batch(int dtype, int dir, int minb, const BatchItem* items, int nitems, const PassParams* descs,
                         const CUtensorMap* maps, int* counters, int* next, int* status, uint64_t wait_ns,
                         BatchLayout lay, int grid, size_t smem, cudaStream_t stream);
size_t batch_smem_bytes(BatchLayout lay, size_t elem_bytes);
cudaError_t launch_batch_df(int dir, const BatchItem* items, int nitems, const PassParams* descs,
                            const CUtensorMap* maps, int* counters, int* next, int* status, uint64_t wait_ns,
                            BatchLayout lay, int grid, size_t smem, cudaStream_t stream);
cudaError_t launch_df_maxexp_list(const void* const* d_states, const uint64_t* d_n16, int* const* d_outs, int count,
                                  uint64_t max_n16, int num_sms, cudaStream_t stream);
}  // namespace qft

using namespace qft;

struct qft_batch_s {
    int count = 0, dtype = 0, dir = -1, nitems = 0, grid = 1, minb = 1;
    BatchLayout lay{1, 1, 1, 8, 256};
    size_t smem = 0;
    uint64_t wait_ns = 2000000000ull;
    // device tables owned by the batch
    PassParams* d_descs = nullptr;
    BatchItem* d_items = nullptr;
    CUtensorMap* d_maps = nullptr;
    int* d_counters = nullptr;  // [0] = work-queue head, [1] = status word, then pass-completion counters
    int ncounters = 0;
    // double-float complex128 batches: per transform its state, amplitude count
    // and maximum-exponent word (read by the pre-pass before the batch kernel)
    bool df = false;
    int num_sms = 148;
    const void** d_df_states = nullptr;
    uint64_t* d_df_n16 = nullptr;
    int** d_df_outs = nullptr;
    uint64_t df_max_n16 = 0;
};

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Per-transform workspace inside the batch workspace: meta (scale_in) +
// one partial sum per warp of each first-pass tile, then (natural order,
// > 1 pass) the ping-pong state buffer.
size_t meta_bytes(const qft_plan_s* pl) {
    return align_up(64 + 8 * static_cast<size_t>(kBatchNormSlots) * static_cast<size_t>(pl->passes[0].prm.num_tiles));
}
size_t work_bytes(const qft_plan_s* pl) {
    const bool need = pl->order == QFT_ORDER_NATURAL && pl->passes.size() > 1;
    return need ? align_up((size_t(1) << pl->n_addr) * pl->esize) : 0;
}

void free_batch(qft_batch_s* b) {
    if (!b) return;
    cudaFree(b->d_df_states);
    cudaFree(b->d_df_n16);
    cudaFree(b->d_df_outs);
    cudaFree(b->d_descs);
    cudaFree(b->d_items);
    cudaFree(b->d_maps);
    cudaFree(b->d_counters);
    delete b;
}

}  // namespace

extern "C" {

size_t qft_batch_workspace_size(const qft_plan_t* plans, int count) {
    if (!plans || count <= 0) return 0;
    size_t s = kAlign;  // reserved
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return 0;
        s += meta_bytes(plans[i]) + work_bytes(plans[i]);
    }
    return s;
}

int qft_batch_create(qft_batch_t* out, const qft_plan_t* plans, void* const* d_states, int count, void* d_workspace,
                     size_t workspace_bytes, double* d_scale_in, int scale_mode) {
    if (!out) return QFT_ERR_BAD_ARG;
    *out = nullptr;
    if (!plans || !d_states || count <= 0 || !d_workspace) return QFT_ERR_BAD_ARG;
    if (scale_mode < QFT_SCALE_STATE || scale_mode > QFT_SCALE_INV_N) return QFT_ERR_BAD_ARG;
    if (reinterpret_cast<uintptr_t>(d_workspace) & (kAlign - 1)) return QFT_ERR_BAD_ARG;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !d_states[i] || (reinterpret_cast<uintptr_t>(d_states[i]) & 255)) return QFT_ERR_BAD_ARG;
        if (plans[i]->dtype != plans[0]->dtype || plans[i]->dir != plans[0]->dir) return QFT_ERR_UNSUPPORTED;
        if (plans[i]->precision) return QFT_ERR_UNSUPPORTED;  // tensor-core tier plans run only through qft_execute
        if (plans[i]->n_addr != plans[i]->n) return QFT_ERR_UNSUPPORTED;  // subset plans run only through qft_execute
        if (plans[i]->df != plans[0]->df) return QFT_ERR_UNSUPPORTED;       // one arithmetic per batch
        for (const auto& ph : plans[i]->passes)
            if (ph.wide) return QFT_ERR_UNSUPPORTED;  // wide-tile passes run only through qft_execute
    }
    if (workspace_bytes < qft_batch_workspace_size(plans, count)) return QFT_ERR_SIZE;
    auto fn = get_encode_fn();

    qft_batch_s* b = new (std::nothrow) qft_batch_s();
    if (!b) return QFT_ERR_NOMEM;
    b->count = count;
    b->dtype = plans[0]->dtype;
    b->dir = plans[0]->dir;
    b->wait_ns = plans[0]->wait_limit_ns;
    b->df = plans[0]->df;
    b->num_sms = plans[0]->num_sms;
    std::vector<const void*> df_states;
    std::vector<uint64_t> df_n16;
    std::vector<int*> df_outs;

    // Transforms with the same plan run next to each other (fewer table rebuilds);
    // each transform's items stay contiguous (its second pass follows its first).
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return plans[x] < plans[y]; });

    std::vector<PassParams> descs;
    std::vector<std::vector<std::vector<BatchItem>>> groups(count);  // [transform][pass] -> its tile items
    std::vector<CUtensorMap> maps;
    std::vector<const qft_plan_s*> shapes;
    char* ws = static_cast<char*>(d_workspace);
    size_t off = kAlign;
    int ncounters = 2;  // queue head, status
    int rc = QFT_OK;
    for (int oi = 0; oi < count && rc == QFT_OK; ++oi) {
        const int i = order[oi];
        qft_plan_s* pl = plans[i];
        int shape = static_cast<int>(std::find(shapes.begin(), shapes.end(), pl) - shapes.begin());
        if (shape == static_cast<int>(shapes.size())) shapes.push_back(pl);
        char* meta = ws + off;
        off += meta_bytes(pl);
        if (b->df) {
            df_states.push_back(d_states[i]);
            df_n16.push_back(uint64_t(1) << pl->n);  // one 16-byte load per complex128 amplitude
            df_outs.push_back(reinterpret_cast<int*>(meta + kMaxExpOff));
            b->df_max_n16 = std::max<uint64_t>(b->df_max_n16, uint64_t(1) << pl->n);
        }
        char* work = ws + off;
        off += work_bytes(pl);
        const int P = static_cast<int>(pl->passes.size());
        int prev_ctr = -1;
        int64_t prev_tiles = 0;
        for (int j = 0; j < P; ++j) {
            const PassHost& ph = pl->passes[j];
            PassParams prm = ph.prm;
            prm.scale_mode = scale_mode;
            prm.in = ph.in_buf == 0 ? d_states[i] : work;
            prm.out = ph.out_buf == 0 ? d_states[i] : work;
            prm.meta = reinterpret_cast<double*>(meta);
            prm.partials = reinterpret_cast<double*>(meta + 64);
            prm.user_scale = d_scale_in ? d_scale_in + i : nullptr;
            prm.status = nullptr;  // set below once the counter block exists
            prm.wait_limit_ns = pl->wait_limit_ns;
            prm.test_skip_first_load = pl->test_skip_first_load;
            int map_idx = -1;
            if (prm.load_mode == 0) {
                if (!fn) { rc = set_cuda_error(cudaErrorNotSupported); break; }
                CUtensorMap m;
                const cuuint32_t estride[5] = {1, 1, 1, 1, 1};
                CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<void*>(prm.in), ph.gdim,
                                ph.gstride, ph.box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) { set_cuda_error_code(static_cast<int>(r)); rc = QFT_ERR_CUDA; break; }
                map_idx = static_cast<int>(maps.size());
                maps.push_back(m);
            }
            const int desc_idx = static_cast<int>(descs.size());
            descs.push_back(prm);
            const int sig = (j + 1 < P) ? ncounters++ : -1;
            groups[oi].emplace_back();
            std::vector<BatchItem>& items = groups[oi].back();
            for (int64_t t = 0; t < prm.num_tiles; ++t) {
                BatchItem it;
                it.desc = desc_idx;
                it.shape = shape * kMaxPasses + j;
                it.tile = t;
                it.wait_ctr = prev_ctr;
                it.wait_target = static_cast<int32_t>(prev_tiles);
                it.signal_ctr = sig;
                it.map = map_idx;
                items.push_back(it);
            }
            b->lay.max_tb = std::max(b->lay.max_tb, static_cast<int32_t>(prm.tb));
            b->lay.max_ntab = std::max(b->lay.max_ntab, static_cast<int32_t>(prm.ntab));
            // twiddle planes: complex entries of the element type
            b->lay.tw_stride = std::max(b->lay.tw_stride, static_cast<int32_t>(prm.ntw * static_cast<int>(pl->esize)));
            prev_ctr = sig;
            prev_tiles = prm.num_tiles;
        }
    }
    if (rc != QFT_OK) { free_batch(b); return rc; }
    b->ncounters = ncounters;
    // two load buffers (the next item's tile loads while this one computes)
    // when they fit, else one
    constexpr size_t kSmemLimit = 227 * 1024 - 4096;
    b->lay.nbuf = 2;
    b->smem = batch_smem_bytes(b->lay, plans[0]->esize);
    if (b->smem > kSmemLimit) {
        b->lay.nbuf = 1;
        b->smem = batch_smem_bytes(b->lay, plans[0]->esize);
    }
    if (b->smem > kSmemLimit) { free_batch(b); return QFT_ERR_UNSUPPORTED; }
    // two CTAs per SM when both fit in shared memory (dynamic + the kernel's
    // 4 KB of static shared memory + 1 KB the SM reserves per CTA; the grid is
    // persistent, so both must be resident) and every block has <= 4 wires
    // (the 128-register kernel), for complex64 passes
    bool small = b->dtype == QFT_C64 && b->lay.max_tb <= 12 && 2 * (b->smem + 5 * 1024) <= 228 * 1024;
    for (const auto& d : descs) {
        for (int s = 0; s < d.nstages; ++s)
            if (d.st[s].r > 4) small = false;
    }
    b->minb = small ? 2 : 1;
    // 512-thread CTAs (twice the warps per SM) when every plan asked for them
    // and the batch runs one CTA per SM in complex64 or double-float
    bool t512 = b->minb == 1 && (b->dtype == QFT_C64 || b->df);
    for (int i = 0; i < count; ++i)
        if (plans[i]->threads != 512) t512 = false;
    for (const auto& d : descs) {
        for (int s = 0; s < d.nstages; ++s)
            if (d.st[s].r > (b->df ? 3 : 4)) t512 = false;
    }
    b->lay.threads = t512 ? 512 : 256;

    // Queue order: a wavefront over blocks of about kBlockGrids grids' worth
    // of first-pass items (batch_order.hpp).
    std::vector<BatchItem> items;
    {
        constexpr size_t kBlockGrids = 4;
        const size_t block_items = kBlockGrids * static_cast<size_t>(plans[0]->num_sms) * b->minb;
        std::vector<std::vector<size_t>> sizes(count);
        for (int t = 0; t < count; ++t)
            for (const auto& g : groups[t]) sizes[t].push_back(g.size());
        for (const auto& tj : wavefront_order(sizes, block_items)) {
            const auto& g = groups[tj.first][tj.second];
            items.insert(items.end(), g.begin(), g.end());
        }
    }
    // after a first pass: all its tiles, then the completing CTA's scale_in
    for (auto& it : items)
        if (it.wait_ctr >= 0 && it.shape % kMaxPasses == 1) it.wait_target += 1;
    b->nitems = static_cast<int>(items.size());
    b->grid = std::max(1, std::min(plans[0]->num_sms * b->minb, b->nitems));

    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&b->d_counters), sizeof(int) * ncounters);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_descs), sizeof(PassParams) * descs.size());
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_items), sizeof(BatchItem) * items.size());
    if (e == cudaSuccess && !maps.empty()) e = cudaMalloc(reinterpret_cast<void**>(&b->d_maps), sizeof(CUtensorMap) * maps.size());
    if (e == cudaSuccess && b->df) {
        e = cudaMalloc(reinterpret_cast<void**>(&b->d_df_states), sizeof(void*) * df_states.size());
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_df_n16), sizeof(uint64_t) * df_n16.size());
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_df_outs), sizeof(int*) * df_outs.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_df_states, df_states.data(), sizeof(void*) * df_states.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_df_n16, df_n16.data(), sizeof(uint64_t) * df_n16.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_df_outs, df_outs.data(), sizeof(int*) * df_outs.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) { free_batch(b); cudaGetLastError(); return QFT_ERR_NOMEM; }
    for (auto& d : descs) d.status = b->d_counters + 1;
    e = cudaMemcpy(b->d_descs, descs.data(), sizeof(PassParams) * descs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !maps.empty())
        e = cudaMemcpy(b->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_counters, 0, sizeof(int) * ncounters);
    if (e != cudaSuccess) { free_batch(b); return set_cuda_error(e); }
    *out = b;
    return QFT_OK;
}

int qft_batch_execute(qft_batch_t b, qft_stream_t stream) {
    if (!b) return QFT_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(int) * b->ncounters, st);
    if (e != cudaSuccess) return set_cuda_error(e);
    // counter indices in the items start at 2: [0] queue head, [1] status word
    if (b->df) {
        e = launch_df_maxexp_list(b->d_df_states, b->d_df_n16, b->d_df_outs, b->count, b->df_max_n16, b->num_sms, st);
        if (e != cudaSuccess) return set_cuda_error(e);
        e = launch_batch_df(b->dir, b->d_items, b->nitems, b->d_descs, b->d_maps, b->d_counters, b->d_counters,
                            b->d_counters + 1, b->wait_ns, b->lay, b->grid, b->smem, st);
    } else {
        e = launch_batch(b->dtype, b->dir, b->minb, b->d_items, b->nitems, b->d_descs, b->d_maps, b->d_counters,
                         b->d_counters, b->d_counters + 1, b->wait_ns, b->lay, b->grid, b->smem, st);
    }
    return e == cudaSuccess ? QFT_OK : set_cuda_error(e);
}

int qft_batch_status(qft_batch_t b, qft_stream_t stream) {
    if (!b) return QFT_ERR_BAD_ARG;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_cuda_error(e);
    int s = 0;
    e = cudaMemcpy(&s, b->d_counters + 1, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(e);
    return s;
}

int qft_batch_destroy(qft_batch_t b) {
    free_batch(b);
    return QFT_OK;
}

}  // extern "C"
