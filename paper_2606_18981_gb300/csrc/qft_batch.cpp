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
//
// Wide groups: complex64 natural-order transforms of 14 <= n <= 20 qubits
// (default-shape or wide plans) run instead on the wide pass kernel in group
// mode (qft_wide.cuh), one launch per pass for all transforms of one (n, k,
// direction), on side streams forked from the caller's stream and joined back
// to it, beside the persistent launch over the rest.  Their passes carry
// 2^14-amplitude tiles in one CTA per SM, where the persistent kernel carries
// 2^13 in a CTA that also claims, waits and loads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <tuple>
#include <utility>
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

// One wide group: the transforms of one (n, k, direction) on the wide pass
// kernel in group mode.
struct WideGroup {
    qft_plan_t plan = nullptr;    // its wide plan (owned by the batch)
    std::vector<int> members;     // transform indices
    std::vector<WideParams> wp;   // per pass, device pointers filled in
    std::vector<int> grid;        // per pass
    int side = 0;                 // side stream index
};

struct qft_batch_s {
    BatchTables T;
    BatchDevice D;  // device tables owned by the batch object
    std::vector<WideGroup> wide;
    void* d_wide = nullptr;  // the groups' tensor maps, output pointers, scale pointers and tile sums
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    ~qft_batch_s() {
        for (auto& g : wide) qft_plan_destroy(g.plan);
        cudaFree(d_wide);
        for (auto st : side) cudaStreamDestroy(st);
        for (auto ev : join) cudaEventDestroy(ev);
        if (fork) cudaEventDestroy(fork);
    }
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
                double* d_scale_in, int scale_mode, bool fixed_shape, BatchTables& T, const std::vector<char>* exclude) {
    if (!plans || !d_states || count <= 0 || !d_workspace) return QFT_ERR_BAD_ARG;
    if (scale_mode < QFT_SCALE_STATE || scale_mode > QFT_SCALE_INV_N) return QFT_ERR_BAD_ARG;
    if (reinterpret_cast<uintptr_t>(d_workspace) & (kAlign - 1)) return QFT_ERR_BAD_ARG;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !d_states[i] || (reinterpret_cast<uintptr_t>(d_states[i]) & 255)) return QFT_ERR_BAD_ARG;
        if (plans[i]->dtype != plans[0]->dtype || plans[i]->dir != plans[0]->dir) return QFT_ERR_UNSUPPORTED;
        if (plans[i]->precision) return QFT_ERR_UNSUPPORTED;  // tensor-core tier plans run only through qft_execute
        if (plans[i]->n_addr != plans[i]->n) return QFT_ERR_UNSUPPORTED;  // subset plans run only through qft_execute
        if (plans[i]->df != plans[0]->df) return QFT_ERR_UNSUPPORTED;       // one arithmetic per batch
        if (exclude && (*exclude)[i]) continue;  // run elsewhere (the wide groups of qft_batch_create)
        for (const auto& ph : plans[i]->passes)
            if (ph.wide) return QFT_ERR_UNSUPPORTED;  // wide-tile passes run here only in wide groups
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
    // per-transform workspace (meta, then the ping-pong buffer), in index order
    T.meta_off.assign(count, 0);
    T.work_off.assign(count, 0);
    {
        size_t off = kAlign;
        for (int i = 0; i < count; ++i) {
            T.meta_off[i] = off;
            off += meta_bytes(plans[i]);
            T.work_off[i] = off;
            off += work_bytes(plans[i]);
        }
    }
    int ncounters = 2;  // queue head, status
    for (int oi = 0; oi < count; ++oi) {
        const int i = order[oi];
        if (exclude && (*exclude)[i]) continue;
        qft_plan_s* pl = plans[i];
        int shape = static_cast<int>(std::find(shapes.begin(), shapes.end(), pl) - shapes.begin());
        if (shape == static_cast<int>(shapes.size())) shapes.push_back(pl);
        char* meta = ws + T.meta_off[i];
        if (T.df) {
            T.df_states.push_back(d_states[i]);
            T.df_n16.push_back(uint64_t(1) << pl->n);  // one 16-byte load per complex128 amplitude
            T.df_outs.push_back(reinterpret_cast<int*>(meta + kMaxExpOff));
            T.df_max_n16 = std::max<uint64_t>(T.df_max_n16, uint64_t(1) << pl->n);
        }
        char* work = ws + T.work_off[i];
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
    // when they fit, else one; the kernel's static shared memory takes 4 KB
    // (6.1 KB for double-float, with its per-tile twiddle table)
    const size_t kSmemLimit = 227 * 1024 - (T.df ? 7 : 4) * 1024;
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
        std::vector<std::vector<size_t>> sizes;
        std::vector<int> which;  // the transforms (in sorted order) with items here
        for (int t = 0; t < count; ++t) {
            if (groups[t].empty()) continue;
            which.push_back(t);
            sizes.emplace_back();
            for (const auto& g : groups[t]) sizes.back().push_back(g.size());
        }
        for (const auto& tj : wavefront_order(sizes, block_items)) {
            const auto& g = groups[which[tj.first]][tj.second];
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

cudaError_t batch_launch(const BatchTables& T, const BatchDevice& D, cudaStream_t st, bool zero) {
    cudaError_t e = zero ? cudaMemsetAsync(D.counters, 0, sizeof(int) * T.ncounters, st) : cudaSuccess;
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

// ------------------------------------------------------------ wide groups

namespace {

constexpr int kWideGroupMinN = 14, kWideGroupMaxN = 20;  // the group kernel sums <= 64 tile norms per transform
constexpr int kMaxSide = 4;                              // side streams of a batch

// Complex64 natural-order whole-register plans of 14..20 qubits that leave
// the shape to the planner or ask for 2^14-amplitude tiles (the test hook
// test_skip_first_load stays with the persistent launch unless the plan asked
// for those tiles).
bool wide_group_eligible(const qft_plan_s* pl) {
    return pl->dtype == QFT_C64 && !pl->df && !pl->precision && pl->order == QFT_ORDER_NATURAL &&
           pl->n_addr == pl->n && pl->w0 == 0 && pl->n >= kWideGroupMinN && pl->n <= kWideGroupMaxN &&
           (!pl->shape_given || pl->wide_tiles == 1) && (!pl->test_skip_first_load || pl->wide_tiles == 1);
}

// Form the groups: one wide plan per (n, direction) among the eligible
// transforms (the cutoff k is per transform in group mode; the pass shapes do
// not depend on it); members of a group whose wide plan could not be built
// stay on the persistent launch.  A group holds at most kWideGroupTilesPerCta
// tiles per SM (the group kernel keeps that many decode scales per CTA) and
// kWideGroupMaxK distinct cutoffs; more transforms of one key open another
// group.  exclude[i] = 1 for the grouped transforms.
int wide_groups_form(const qft_plan_t* plans, int count, std::vector<WideGroup>& groups, std::vector<char>& exclude) {
    exclude.assign(count, 0);
    std::vector<std::pair<std::tuple<int, int, int>, int>> keys;  // (n, dir, test hook) -> open group
    for (int i = 0; i < count; ++i) {
        const qft_plan_s* pl = plans[i];
        if (!pl || !wide_group_eligible(pl)) continue;
        const auto key = std::make_tuple(pl->n, pl->dir, pl->test_skip_first_load);
        auto it = std::find_if(keys.begin(), keys.end(), [&](const auto& kv) { return kv.first == key; });
        const size_t cap = (static_cast<size_t>(kWideGroupTilesPerCta) * pl->num_sms) >> (pl->n - 14);
        if (it != keys.end() && it->second >= 0) {
            const WideGroup& og = groups[it->second];
            std::vector<int> ks;
            for (int m : og.members)
                if (std::find(ks.begin(), ks.end(), plans[m]->kk) == ks.end()) ks.push_back(plans[m]->kk);
            const bool new_k = std::find(ks.begin(), ks.end(), pl->kk) == ks.end();
            if (og.members.size() >= cap || (new_k && static_cast<int>(ks.size()) >= kWideGroupMaxK)) {
                keys.erase(it);  // full: this member opens a new group
                it = keys.end();
            }
        }
        int g;
        if (it == keys.end()) {
            qft_opts o{};
            o.order = QFT_ORDER_NATURAL;
            o.tile_bits = 14;
            o.wait_limit_ms = static_cast<int>((pl->wait_limit_ns + 999999ull) / 1000000ull);
            o.test_skip_first_load = pl->test_skip_first_load;
            qft_plan_t wp = nullptr;
            int rc = qft_plan_create(&wp, pl->n, pl->k, pl->dir, QFT_C64, &o);
            if (rc == QFT_ERR_NOMEM) return rc;
            bool ok = rc == QFT_OK && wp->passes.size() >= 2;
            if (ok)
                for (const auto& ph : wp->passes) ok = ok && ph.wide && ph.in_buf == (&ph == &wp->passes[0] ? 0 : 1);
            if (!ok) {
                qft_plan_destroy(wp);
                wp = nullptr;
            }
            g = wp ? static_cast<int>(groups.size()) : -1;
            if (wp) {
                groups.emplace_back();
                groups.back().plan = wp;
            }
            keys.emplace_back(key, g);
        } else {
            g = it->second;
        }
        if (g < 0) continue;
        groups[g].members.push_back(i);
        exclude[i] = 1;
    }
    return QFT_OK;
}

// Device tables of the groups (one allocation): per group and pass a tensor
// map and an output pointer per member, per group a scale pointer and the
// tile sums per member.  Fills each group's WideParams.
int wide_groups_bind(qft_batch_s* b, const qft_plan_t* plans, void* const* d_states, char* ws, double* d_scale_in,
                     int scale_mode) {
    auto& groups = b->wide;
    if (groups.empty()) return QFT_OK;
    auto plans_kk = [&](int i) { return plans[i]->kk; };
    auto fn = get_encode_fn();
    if (!fn) return set_cuda_error(cudaErrorNotSupported);
    size_t n_maps = 0, n_ptrs = 0, n_tp = 0;
    for (const auto& g : groups) {
        const size_t G = g.members.size(), P = g.plan->passes.size();
        n_maps += G * P;
        n_ptrs += G * P + G;
        n_tp += G << (g.plan->n - 14);
    }
    const size_t o_ptrs = n_maps * sizeof(CUtensorMap);
    const size_t o_tp = (o_ptrs + n_ptrs * sizeof(void*) + 255) / 256 * 256;
    const size_t bytes = o_tp + n_tp * sizeof(double);
    cudaError_t e = cudaMalloc(&b->d_wide, bytes);
    if (e != cudaSuccess) {
        b->d_wide = nullptr;
        cudaGetLastError();
        return QFT_ERR_NOMEM;
    }
    std::vector<unsigned char> host(o_tp, 0);
    void** hptrs = reinterpret_cast<void**>(host.data() + o_ptrs);
    char* dbase = static_cast<char*>(b->d_wide);
    size_t im = 0, ip = 0, it = 0;
    const cuuint32_t estride[5] = {1, 1, 1, 1, 1};
    for (auto& g : groups) {
        const qft_plan_s* wp = g.plan;
        const int G = static_cast<int>(g.members.size()), P = static_cast<int>(wp->passes.size());
        // members in runs of equal cutoff (the kernel rebuilds its tables once per run)
        std::stable_sort(g.members.begin(), g.members.end(), [&](int x, int y) { return plans_kk(x) < plans_kk(y); });
        int gk_n = 0;
        int32_t gk_end[kWideGroupMaxK] = {}, gk_val[kWideGroupMaxK] = {};
        for (int m = 0; m < G; ++m) {
            const int kk = plans_kk(g.members[m]);
            if (gk_n == 0 || gk_val[gk_n - 1] != kk) {
                if (gk_n == kWideGroupMaxK) return QFT_ERR_UNSUPPORTED;  // wide_groups_form keeps this from happening
                gk_val[gk_n++] = kk;
            }
            gk_end[gk_n - 1] = m + 1;
        }
        double** d_gscale = reinterpret_cast<double**>(dbase + o_ptrs) + ip;
        for (int m = 0; m < G; ++m) hptrs[ip++] = d_scale_in ? d_scale_in + g.members[m] : nullptr;
        double* d_tp = reinterpret_cast<double*>(dbase + o_tp) + it;
        it += static_cast<size_t>(G) << (wp->n - 14);
        g.wp.clear();
        g.grid.clear();
        for (int j = 0; j < P; ++j) {
            const PassHost& ph = wp->passes[j];
            const CUtensorMap* d_maps = reinterpret_cast<const CUtensorMap*>(dbase) + im;
            void* const* d_outs = reinterpret_cast<void* const*>(dbase + o_ptrs) + ip;
            for (int m = 0; m < G; ++m) {
                const int i = g.members[m];
                void* work = ws + b->T.work_off[i];
                void* in = ph.in_buf == 0 ? d_states[i] : work;
                CUtensorMap tm;  // encoded in place (64-byte aligned), then copied into the upload buffer
                CUresult r = fn(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, in, ph.gdim, ph.gstride, ph.box, estride,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) {
                    set_cuda_error_code(static_cast<int>(r));
                    return QFT_ERR_CUDA;
                }
                std::memcpy(host.data() + sizeof(CUtensorMap) * im++, &tm, sizeof(tm));
                hptrs[ip++] = ph.out_buf == 0 ? d_states[i] : work;
            }
            WideParams W = ph.wp;
            W.scale_mode = scale_mode;
            W.lt_bits = wp->n - 14;
            W.num_tiles = static_cast<int64_t>(G) << W.lt_bits;
            W.maps = d_maps;
            W.outs = d_outs;
            W.tpart = d_tp;
            W.gscale = d_scale_in ? d_gscale : nullptr;
            W.out = nullptr;
            W.partials = nullptr;
            W.npartials = 0;
            W.meta = nullptr;
            W.user_scale = nullptr;
            W.status = b->D.counters + 1;
            W.wait_limit_ns = wp->wait_limit_ns;
            W.test_skip_first_load = wp->test_skip_first_load;
            W.kk = gk_val[0];
            W.gk_n = gk_n;
            for (int r = 0; r < kWideGroupMaxK; ++r) {
                W.gk_end[r] = gk_end[r];
                W.gk_val[r] = gk_val[r];
            }
            g.wp.push_back(W);
            g.grid.push_back(static_cast<int>(std::min<int64_t>(W.num_tiles, wp->num_sms)));
        }
    }
    e = cudaMemcpy(b->d_wide, host.data(), o_tp, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_cuda_error(e);
    // side streams (groups by decreasing size, each to the least-loaded stream) and the fork / join events
    const int nside = std::min<int>(kMaxSide, static_cast<int>(groups.size()));
    std::vector<int> byd(groups.size());
    std::iota(byd.begin(), byd.end(), 0);
    auto tiles = [&](int g) { return groups[g].wp[0].num_tiles; };
    std::stable_sort(byd.begin(), byd.end(), [&](int x, int y) { return tiles(x) > tiles(y); });
    std::vector<int64_t> load(nside, 0);
    for (int g : byd) {
        const int sidx = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
        groups[g].side = sidx;
        load[sidx] += tiles(g);
    }
    std::vector<WideGroup> sorted;
    for (int g : byd) sorted.push_back(std::move(groups[g]));
    groups = std::move(sorted);
    b->side.assign(nside, nullptr);
    b->join.assign(nside, nullptr);
    e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int k = 0; k < nside && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return set_cuda_error(e);
    return QFT_OK;
}

}  // namespace

extern "C" {

size_t qft_batch_workspace_size(const qft_plan_t* plans, int count) { return batch_workspace_bytes(plans, count); }

int qft_batch_create(qft_batch_t* out, const qft_plan_t* plans, void* const* d_states, int count, void* d_workspace,
                     size_t workspace_bytes, double* d_scale_in, int scale_mode) {
    if (!out) return QFT_ERR_BAD_ARG;
    *out = nullptr;
    if (!plans || !d_states || count <= 0 || !d_workspace) return QFT_ERR_BAD_ARG;
    for (int i = 0; i < count; ++i)
        if (!plans[i]) return QFT_ERR_BAD_ARG;
    qft_batch_s* b = new (std::nothrow) qft_batch_s();
    if (!b) return QFT_ERR_NOMEM;
    std::vector<char> exclude;
    int rc = wide_groups_form(plans, count, b->wide, exclude);
    if (rc == QFT_OK)
        rc = batch_build(plans, d_states, count, d_workspace, workspace_bytes, d_scale_in, scale_mode, false, b->T,
                         &exclude);
    if (rc != QFT_OK) {
        delete b;
        return rc;
    }
    BatchTables& T = b->T;
    BatchDevice& D = b->D;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&D.counters), sizeof(int) * T.ncounters);
    if (e == cudaSuccess && !T.descs.empty())
        e = cudaMalloc(reinterpret_cast<void**>(&D.descs), sizeof(PassParams) * T.descs.size());
    if (e == cudaSuccess && !T.items.empty())
        e = cudaMalloc(reinterpret_cast<void**>(&D.items), sizeof(BatchItem) * T.items.size());
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
    if (!T.descs.empty())
        e = cudaMemcpy(D.descs, T.descs.data(), sizeof(PassParams) * T.descs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !T.items.empty())
        e = cudaMemcpy(D.items, T.items.data(), sizeof(BatchItem) * T.items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !T.maps.empty())
        e = cudaMemcpy(D.maps, T.maps.data(), sizeof(CUtensorMap) * T.maps.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(D.counters, 0, sizeof(int) * T.ncounters);
    if (e != cudaSuccess) {
        free_device(D);
        delete b;
        return set_cuda_error(e);
    }
    rc = wide_groups_bind(b, plans, d_states, static_cast<char*>(d_workspace), d_scale_in, scale_mode);
    if (rc != QFT_OK) {
        free_device(D);
        delete b;
        return rc;
    }
    *out = b;
    return QFT_OK;
}

int qft_batch_execute(qft_batch_t b, qft_stream_t stream) {
    if (!b) return QFT_ERR_BAD_ARG;
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (b->wide.empty()) {
        const cudaError_t e = batch_launch(b->T, b->D, st);
        return e == cudaSuccess ? QFT_OK : set_cuda_error(e);
    }
    // zero the counters (and status word), fork the side streams, run the
    // persistent launch and the groups' passes side by side, join
    cudaError_t e = cudaMemsetAsync(b->D.counters, 0, sizeof(int) * b->T.ncounters, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, st);
    for (size_t k = 0; k < b->side.size() && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
    if (e == cudaSuccess && b->T.nitems > 0) e = batch_launch(b->T, b->D, st, false);
    for (const auto& g : b->wide) {
        for (size_t j = 0; j < g.wp.size() && e == cudaSuccess; ++j) {
            const PassHost& ph = g.plan->passes[j];
            e = launch_pass_wide_group(g.plan->dir, ph.wide_r0, ph.wide_r1, ph.wide_top, g.wp[j], g.grid[j],
                                       b->side[g.side]);
        }
    }
    for (size_t k = 0; k < b->side.size() && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->join[k], b->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->join[k], 0);
    }
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

int qft_batch_get_info(qft_batch_t b, qft_batch_info* info) {
    if (!b || !info) return QFT_ERR_BAD_ARG;
    std::memset(info, 0, sizeof(*info));
    info->transforms = b->T.count;
    info->persistent_items = b->T.nitems;
    info->wide_groups = static_cast<int>(b->wide.size());
    int launches = b->T.nitems > 0 ? 1 + (b->T.df ? 1 : 0) : 0;
    for (const auto& g : b->wide) {
        info->wide_transforms += static_cast<int>(g.members.size());
        launches += static_cast<int>(g.wp.size());
    }
    info->kernel_launches = launches;
    info->side_streams = static_cast<int>(b->side.size());
    return QFT_OK;
}

}  // extern "C"
