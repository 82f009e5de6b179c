// batch_host.hpp -- host-side tables of a batched launch (qft_batch.cpp) and
// the reusable batch slots the serving loop runs them in (qft_server.cpp).
// Internal to libqftfft.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "plan_host.hpp"

namespace qft {

// Everything one batched launch needs, built on the host.
struct BatchTables {
    int count = 0, dtype = 0, dir = -1, nitems = 0, grid = 1, minb = 1, ncounters = 2, num_sms = 148;
    BatchLayout lay{1, 1, 1, 8, 256};
    size_t smem = 0;
    uint64_t wait_ns = 2000000000ull;
    bool df = false;  // double-float complex128: a maximum-exponent pre-pass per transform
    uint64_t df_max_n16 = 0;
    std::vector<PassParams> descs;  // per transform and pass
    std::vector<BatchItem> items;   // the ordered work list
    std::vector<CUtensorMap> maps;  // per strided pass
    std::vector<const void*> df_states;
    std::vector<uint64_t> df_n16;
    std::vector<int*> df_outs;
    std::vector<size_t> meta_off, work_off;  // per transform: its meta and ping-pong buffer in the workspace
};

// Device copies of the tables the kernels read.  counters[0] is the work-queue
// head, counters[1] the status word, then the pass-completion counters.
struct BatchDevice {
    PassParams* descs = nullptr;
    BatchItem* items = nullptr;
    CUtensorMap* maps = nullptr;
    int* counters = nullptr;
    const void** df_states = nullptr;
    uint64_t* df_n16 = nullptr;
    int** df_outs = nullptr;
};

// Workspace bytes of a batch of these plans (qft_batch_workspace_size): 256
// plus each transform's share.
size_t batch_workspace_bytes(const qft_plan_t* plans, int count);
size_t batch_transform_workspace_bytes(const qft_plan_s* pl);

// Build the tables of a batch: transform i = plans[i] on d_states[i], its
// per-transform workspace inside d_workspace, scale_in into d_scale_in[i]
// (optional).  fixed_shape: run one 256-thread CTA per SM whatever the plans,
// so that a transform's result does not depend on which others share the
// batch (plans that need 512 threads give QFT_ERR_UNSUPPORTED).  exclude
// (optional, one flag per transform): transforms that get their workspace
// share but no work items (they run in wide groups, below).
int batch_build(const qft_plan_t* plans, void* const* d_states, int count, void* d_workspace, size_t workspace_bytes,
                double* d_scale_in, int scale_mode, bool fixed_shape, BatchTables& T,
                const std::vector<char>* exclude = nullptr);

// Point every descriptor's status word at counters + 1 (before the upload).
void batch_set_status(BatchTables& T, int* d_counters);

// Zero the counters (unless zero = false: the caller did) and launch (with
// the double-float pre-pass first) on st.
cudaError_t batch_launch(const BatchTables& T, const BatchDevice& D, cudaStream_t st, bool zero = true);

// Device tables allocated once for batches up to a capacity, with pinned
// staging of the same layout: slot_run copies a batch's tables into the
// staging, uploads them with one asynchronous copy and launches, all on st.
// The staging is reused by the next slot_run, so a slot runs one batch at a
// time (its caller waits for the previous batch's completion first).
struct BatchSlot {
    void* d_base = nullptr;
    void* h_base = nullptr;
    size_t bytes = 0;
    int cap_transforms = 0;
    size_t cap_descs = 0, cap_items = 0, cap_maps = 0, cap_counters = 0;
    size_t o_maps = 0, o_descs = 0, o_items = 0, o_counters = 0, o_df_states = 0, o_df_n16 = 0, o_df_outs = 0,
           o_scale = 0;
    BatchDevice D;
    double* d_scale = nullptr;  // per-transform scale_in of the slot's batch (device)
};

int slot_create(BatchSlot& S, int max_transforms, size_t max_items);
void slot_destroy(BatchSlot& S);
int slot_run(BatchSlot& S, BatchTables& T, cudaStream_t st);

}  // namespace qft
