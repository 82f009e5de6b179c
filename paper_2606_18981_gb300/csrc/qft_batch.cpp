// qft_batch.cpp -- batched execution: many transforms of different sizes and
// cutoffs in one persistent launch of qft_batch_kernel (see qft_pass.cu).
//
// qft_batch_create binds each transform (a plan and its device state) once
// (batch_build makes the tables, shared with the serving loop's batch slots):
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
#include "batch_host.hpp"
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
    BatchTables T;
    BatchDevice D;  // device tables owned by the batch object
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

void free_device(BatchDevice& D) {
    cudaFree(D.df_states);
    cudaFree(D.df_n16);
    cudaFree(D.df_outs);
    cudaFree(D.descs);
    cudaFree(D.items);
    cudaFree(D.maps);
    cudaFree(D.counters);
    D = BatchDevice{};
}

}  // namespace

namespace qft {

size_t batch_transform_workspace_bytes(const qft_plan_s* pl) { return meta_bytes(pl) + work_bytes(pl); }

size_t batch_workspace_bytes(const qft_plan_t* plans, int count) {
    if (!plans || count <= 0) return 0;
    size_t s = kAlign;  // reserved
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return 0;
        s += meta_bytes(plans[i]) + work_bytes(plans[i]);
    }
    return s;
}

int batch_build(const qft_plan_t* plans, void* const* d_states, int count, void* d_workspace, size_t workspace_bytes,
                double* d_scale_in, int scale_mode, bool fixed_shape, BatchTables& T) {
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
    if (workspace_bytes < batch_workspace_bytes(plans, count)) return QFT_ERR_SIZE;
    auto fn = get_encode_fn();

    T = BatchTables{};
    T.count = count;
    T.dtype = plans[0]->dtype;
    T.dir = plans[0]->dir;
    T.wait_ns = plans[0]->wait_limit_ns;
    T.df = plans[0]->df;
    T.num_sms = plans[0]->num_sms;

    // Transforms with the same plan run next to each other (fewer table rebuilds);
    // each transform's items stay contiguous (its second pass follows its first).
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return plans[x] < plans[y]; });

    std::vector<PassParams>& descs = T.descs;
    std::vector<std::vector<std::vector<BatchItem>>> groups(count);  // [transform][pass] -> its tile items
    std::vector<CUtensorMap>& maps = T.maps;
    std::vector<const qft_plan_s*> shapes;
    char* ws = static_cast<char*>(d_workspace);
    size_t off = kAlign;
    int ncounters = 2;  // queue head, status
    for (int oi = 0; oi < count; ++oi) {
        const int i = order[oi];
        qft_plan_s* pl = plans[i];
        int shape = static_cast<int>(std::find(shapes.begin(), shapes.end(), pl) - shapes.begin());
        if (shape == static_cast<int>(shapes.size())) shapes.push_back(pl);
        char* meta = ws + off;
        off += meta_bytes(pl);
        if (T.df) {
            T.df_states.push_back(d_states[i]);
            T.df_n16.push_back(uint64_t(1) << pl->n);  // one 16-byte load per complex128 amplitude
            T.df_outs.push_back(reinterpret_cast<int*>(meta + kMaxExpOff));
            T.df_max_n16 = std::max<uint64_t>(T.df_max_n16, uint64_t(1) << pl->n);
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
            prm.status = nullptr;  // set by batch_set_status once the counter block exists
            prm.wait_limit_ns = pl->wait_limit_ns;
            prm.test_skip_first_load = pl->test_skip_first_load;
            int map_idx = -1;
            if (prm.load_mode == 0) {
                if (!fn) return set_cuda_error(cudaErrorNotSupported);
                CUtensorMap m;
                const cuuint32_t estride[5] = {1, 1, 1, 1, 1};
                CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<void*>(prm.in), ph.gdim,
                                ph.gstride, ph.box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) { set_cuda_error_code(static_cast<int>(r)); return QFT_ERR_CUDA; }
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
            T.lay.max_tb = std::max(T.lay.max_tb, static_cast<int32_t>(prm.tb));
            T.lay.max_ntab = std::max(T.lay.max_ntab, static_cast<int32_t>(prm.ntab));
            // twiddle planes: complex entries of the element type
            T.lay.tw_stride = std::max(T.lay.tw_stride, static_cast<int32_t>(prm.ntw * static_cast<int>(pl->esize)));
            prev_ctr = sig;
            prev_tiles = prm.num_tiles;
        }
    }
    T.ncounters = ncounters;
    // two load buffers (the next item's tile loads while this one computes)
    // when they fit, else one
    constexpr size_t kSmemLimit = 227 * 1024 - 4096;
    T.lay.nbuf = 2;
    T.smem = batch_smem_bytes(T.lay, plans[0]->esize);
    if (T.smem > kSmemLimit) {
        T.lay.nbuf = 1;
        T.smem = batch_smem_bytes(T.lay, plans[0]->esize);
    }
    if (T.smem > kSmemLimit) return QFT_ERR_UNSUPPORTED;
    // two CTAs per SM when both fit in shared memory (dynamic + the kernel's
    // 4 KB of static shared memory + 1 KB the SM reserves per CTA; the grid is
    // persistent, so both must be resident) and every block has <= 4 wires
    // (the 128-register kernel), for complex64 passes
    bool small = T.dtype == QFT_C64 && T.lay.max_tb <= 12 && 2 * (T.smem + 5 * 1024) <= 228 * 1024;
    for (const auto& d : descs) {
        for (int s = 0; s < d.nstages; ++s)
            if (d.st[s].r > 4) small = false;
    }
    T.minb = small && !fixed_shape ? 2 : 1;
    // 512-thread CTAs (twice the warps per SM) when every plan asked for them
    // and the batch runs one CTA per SM in complex64 or double-float
    bool t512 = T.minb == 1 && (T.dtype == QFT_C64 || T.df) && !fixed_shape;
    for (int i = 0; i < count; ++i)
        if (plans[i]->threads != 512) t512 = false;
    for (const auto& d : descs) {
        for (int s = 0; s < d.nstages; ++s)
            if (d.st[s].r > (T.df ? 3 : 4)) t512 = false;
    }
    T.lay.threads = t512 ? 512 : 256;
    if (fixed_shape)
        for (int i = 0; i < count; ++i)
            if (plans[i]->threads == 512) return QFT_ERR_UNSUPPORTED;  // the fixed shape is 256 threads

    // Queue order: a wavefront over blocks of about kBlockGrids grids' worth
    // of first-pass items (batch_order.hpp).
    std::vector<BatchItem>& items = T.items;
    {
        constexpr size_t kBlockGrids = 4;
        const size_t block_items = kBlockGrids * static_cast<size_t>(plans[0]->num_sms) * T.minb;
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
    T.nitems = static_cast<int>(items.size());
    T.grid = std::max(1, std::min(plans[0]->num_sms * T.minb, T.nitems));
    return QFT_OK;
}

void batch_set_status(BatchTables& T, int* d_counters) {
    for (auto& d : T.descs) d.status = d_counters + 1;
}

cudaError_t batch_launch(const BatchTables& T, const BatchDevice& D, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(D.counters, 0, sizeof(int) * T.ncounters, st);
    if (e != cudaSuccess) return e;
    // counter indices in the items start at 2: [0] queue head, [1] status word
    if (T.df) {
        e = launch_df_maxexp_list(D.df_states, D.df_n16, D.df_outs, T.count, T.df_max_n16, T.num_sms, st);
        if (e != cudaSuccess) return e;
        return launch_batch_df(T.dir, D.items, T.nitems, D.descs, D.maps, D.counters, D.counters, D.counters + 1,
                               T.wait_ns, T.lay, T.grid, T.smem, st);
    }
    return launch_batch(T.dtype, T.dir, T.minb, D.items, T.nitems, D.descs, D.maps, D.counters, D.counters,
                        D.counters + 1, T.wait_ns, T.lay, T.grid, T.smem, st);
}

// ------------------------------------------------------------ batch slots
// Device tables allocated once for batches of up to the slot's capacity,
// refilled per batch through pinned staging with asynchronous copies (no
// allocation and no synchronous copy per batch).

int slot_create(BatchSlot& S, int max_transforms, size_t max_items) {
    S = BatchSlot{};
    S.cap_transforms = max_transforms;
    S.cap_descs = static_cast<size_t>(max_transforms) * kMaxPasses;
    S.cap_items = max_items;
    S.cap_maps = S.cap_descs;
    S.cap_counters = 2 + S.cap_descs;
    S.bytes = sizeof(PassParams) * S.cap_descs + sizeof(BatchItem) * S.cap_items + sizeof(CUtensorMap) * S.cap_maps +
              sizeof(int) * S.cap_counters + (sizeof(void*) + sizeof(uint64_t) + sizeof(int*)) * max_transforms +
              sizeof(double) * max_transforms + 1024;
    cudaError_t e = cudaMalloc(&S.d_base, S.bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&S.h_base, S.bytes);
    if (e != cudaSuccess) {
        cudaFree(S.d_base);
        S.d_base = nullptr;
        cudaGetLastError();
        return QFT_ERR_NOMEM;
    }
    // carve both areas identically (64-byte aligned parts; tensor maps need 64)
    size_t off = 0;
    auto part = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 63) / 64 * 64;
        return o;
    };
    S.o_maps = part(sizeof(CUtensorMap) * S.cap_maps);
    S.o_descs = part(sizeof(PassParams) * S.cap_descs);
    S.o_items = part(sizeof(BatchItem) * S.cap_items);
    S.o_counters = part(sizeof(int) * S.cap_counters);
    S.o_df_states = part(sizeof(void*) * max_transforms);
    S.o_df_n16 = part(sizeof(uint64_t) * max_transforms);
    S.o_df_outs = part(sizeof(int*) * max_transforms);
    S.o_scale = part(sizeof(double) * max_transforms);
    if (off > S.bytes) return QFT_ERR_NOMEM;
    char* d = static_cast<char*>(S.d_base);
    S.D.maps = reinterpret_cast<CUtensorMap*>(d + S.o_maps);
    S.D.descs = reinterpret_cast<PassParams*>(d + S.o_descs);
    S.D.items = reinterpret_cast<BatchItem*>(d + S.o_items);
    S.D.counters = reinterpret_cast<int*>(d + S.o_counters);
    S.D.df_states = reinterpret_cast<const void**>(d + S.o_df_states);
    S.D.df_n16 = reinterpret_cast<uint64_t*>(d + S.o_df_n16);
    S.D.df_outs = reinterpret_cast<int**>(d + S.o_df_outs);
    S.d_scale = reinterpret_cast<double*>(d + S.o_scale);
    return QFT_OK;
}

void slot_destroy(BatchSlot& S) {
    cudaFree(S.d_base);
    cudaFreeHost(S.h_base);
    S = BatchSlot{};
}

int slot_run(BatchSlot& S, BatchTables& T, cudaStream_t st) {
    if (T.count > S.cap_transforms || T.descs.size() > S.cap_descs || T.items.size() > S.cap_items ||
        T.maps.size() > S.cap_maps || static_cast<size_t>(T.ncounters) > S.cap_counters)
        return QFT_ERR_SIZE;
    batch_set_status(T, S.D.counters);
    char* h = static_cast<char*>(S.h_base);
    std::memcpy(h + S.o_maps, T.maps.data(), sizeof(CUtensorMap) * T.maps.size());
    std::memcpy(h + S.o_descs, T.descs.data(), sizeof(PassParams) * T.descs.size());
    std::memcpy(h + S.o_items, T.items.data(), sizeof(BatchItem) * T.items.size());
    if (T.df) {
        std::memcpy(h + S.o_df_states, T.df_states.data(), sizeof(void*) * T.df_states.size());
        std::memcpy(h + S.o_df_n16, T.df_n16.data(), sizeof(uint64_t) * T.df_n16.size());
        std::memcpy(h + S.o_df_outs, T.df_outs.data(), sizeof(int*) * T.df_outs.size());
    }
    // one copy of the used prefix (maps, descs, items and the rest lie in that order)
    const size_t used = T.df ? S.o_df_outs + sizeof(int*) * T.df_outs.size() : S.o_items + sizeof(BatchItem) * T.items.size();
    cudaError_t e = cudaMemcpyAsync(S.d_base, S.h_base, used, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = batch_launch(T, S.D, st);
    return e == cudaSuccess ? QFT_OK : set_cuda_error(e);
}

}  // namespace qft

extern "C" {

size_t qft_batch_workspace_size(const qft_plan_t* plans, int count) { return batch_workspace_bytes(plans, count); }

int qft_batch_create(qft_batch_t* out, const qft_plan_t* plans, void* const* d_states, int count, void* d_workspace,
                     size_t workspace_bytes, double* d_scale_in, int scale_mode) {
    if (!out) return QFT_ERR_BAD_ARG;
    *out = nullptr;
    qft_batch_s* b = new (std::nothrow) qft_batch_s();
    if (!b) return QFT_ERR_NOMEM;
    int rc = batch_build(plans, d_states, count, d_workspace, workspace_bytes, d_scale_in, scale_mode, false, b->T);
    if (rc != QFT_OK) {
        delete b;
        return rc;
    }
    BatchTables& T = b->T;
    BatchDevice& D = b->D;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&D.counters), sizeof(int) * T.ncounters);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&D.descs), sizeof(PassParams) * T.descs.size());
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&D.items), sizeof(BatchItem) * T.items.size());
    if (e == cudaSuccess && !T.maps.empty())
        e = cudaMalloc(reinterpret_cast<void**>(&D.maps), sizeof(CUtensorMap) * T.maps.size());
    if (e == cudaSuccess && T.df) {
        e = cudaMalloc(reinterpret_cast<void**>(&D.df_states), sizeof(void*) * T.df_states.size());
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&D.df_n16), sizeof(uint64_t) * T.df_n16.size());
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&D.df_outs), sizeof(int*) * T.df_outs.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(D.df_states, T.df_states.data(), sizeof(void*) * T.df_states.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(D.df_n16, T.df_n16.data(), sizeof(uint64_t) * T.df_n16.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(D.df_outs, T.df_outs.data(), sizeof(int*) * T.df_outs.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        free_device(D);
        delete b;
        cudaGetLastError();
        return QFT_ERR_NOMEM;
    }
    batch_set_status(T, D.counters);
    e = cudaMemcpy(D.descs, T.descs.data(), sizeof(PassParams) * T.descs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(D.items, T.items.data(), sizeof(BatchItem) * T.items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !T.maps.empty())
        e = cudaMemcpy(D.maps, T.maps.data(), sizeof(CUtensorMap) * T.maps.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(D.counters, 0, sizeof(int) * T.ncounters);
    if (e != cudaSuccess) {
        free_device(D);
        delete b;
        return set_cuda_error(e);
    }
    *out = b;
    return QFT_OK;
}

int qft_batch_execute(qft_batch_t b, qft_stream_t stream) {
    if (!b) return QFT_ERR_BAD_ARG;
    const cudaError_t e = batch_launch(b->T, b->D, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? QFT_OK : set_cuda_error(e);
}

int qft_batch_status(qft_batch_t b, qft_stream_t stream) {
    if (!b) return QFT_ERR_BAD_ARG;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return set_cuda_error(e);
    int s = 0;
    e = cudaMemcpy(&s, b->D.counters + 1, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(e);
    return s;
}

int qft_batch_destroy(qft_batch_t b) {
    if (b) free_device(b->D);
    delete b;
    return QFT_OK;
}

}  // extern "C"
