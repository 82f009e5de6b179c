// qft_server.cpp -- a continuous-batching request loop for transforms of mixed
// sizes, cutoffs, directions and dtypes.
//
// A worker thread owns CUDA streams, a plan cache keyed by (n, k, direction,
// dtype, order), a pool of device buffers and a few batch slots (device
// tables of a batched launch, allocated once).  Requests are admitted in
// arrival order as soon as the device bytes they need fit in the HBM budget
// together with everything in flight and an in-flight slot is free.
//   * Small requests (n <= the batching limit, 18 by default) join the batch
//     that is forming for their (dtype, direction, scale mode); on every pass
//     of the worker loop each forming batch whose slot is free is launched as
//     one persistent batched launch (qft_batch_kernel) on a high-priority stream:
//     copy-ins, the batch, copy-outs, one read-back of the scale_in values and
//     the status word, an event.  Requests that arrive while batches run are
//     admitted into the next ones as slots and memory free up.
//   * Larger requests run their own passes on the least-loaded of the
//     normal-priority streams (the high-priority batches are scheduled between
//     those passes): out of place from the caller's input into its output when
//     both are device buffers (then the request holds only a workspace), else
//     copy-in, qft_execute, copy-out through a pooled state buffer.
// Completion is detected by polling events; buffers go back to the pool and
// each request's latency (submit to completion) is recorded.  Server batches
// use one fixed kernel shape (one 256-thread CTA per SM), and a transform's
// arithmetic in a batch does not depend on the other transforms in it, so a
// request's result is bit for bit the same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/qftfft.h"
#include "batch_host.hpp"
#include "plan_host.hpp"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    qft_request r{};
    Clock::time_point t_submit;
};

struct InFlight {
    Request req;
    qft_plan_t plan = nullptr;
    void* state = nullptr;
    void* ws = nullptr;
    size_t bytes = 0;
    int stream = 0;
    cudaEvent_t done = nullptr;
    double* h_slot = nullptr;  // pinned 16-byte slot: scale_in (double) then the status word (int)
    int slot = 0;
    size_t reserve = 0;  // batched requests: their share of the batch workspace, held in the budget
    bool direct = false; // single request run from the caller's input into its output (no copies)
};

struct Result {
    int status = 1;  // 1 = pending, 0 = ok, < 0 = error
    double latency_ms = 0.0;
    double scale_in = 0.0;
};

// A batched launch of admitted small requests.
struct Slot {
    qft::BatchSlot S;
    bool busy = false;
    cudaEvent_t done = nullptr;
    std::vector<InFlight> reqs;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    double* h_scale = nullptr;  // pinned: scale_in per transform, then the status word
};

constexpr int kSlotTransforms = 512;      // requests per batched launch, at most
constexpr size_t kSlotItems = size_t(1) << 16;  // tile items per batched launch, at most

}  // namespace

struct qft_server_s {
    size_t budget = 0, in_use = 0;
    int nstreams = 8, max_inflight = 64, device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_load;
    std::map<std::tuple<int, int, int, int, int>, qft_plan_t> plans;
    std::multimap<size_t, void*> pool;  // free device buffers by size
    size_t pooled = 0;
    std::deque<Request> pending;
    std::vector<InFlight> inflight;
    std::unordered_map<uint64_t, Result> results;
    std::vector<double> latencies;
    Clock::time_point t_first{}, t_last{};
    uint64_t next_ticket = 1, completed = 0, failed = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::atomic<bool> stop{false};
    std::thread worker;
    double* slots = nullptr;  // pinned host memory, two doubles per in-flight slot
    std::vector<int> free_slots;
    int fail_allocs = 0;      // test hook: allocations still to fail
    // continuous batching
    int batch_max_n = 18;     // requests with n <= this run in batched launches (0: never)
    cudaStream_t batch_stream = nullptr;
    std::vector<Slot> bslots;
    std::map<std::tuple<int, int, int>, std::vector<InFlight>> forming;  // (dtype, direction, scale mode)
    long long forming_count = 0, batched_count = 0;  // admitted-not-launched, launched-not-finished
    long long batches_launched = 0, batched_requests = 0;
};

namespace {

size_t request_bytes(qft_plan_t p) {
    return ((size_t(1) << p->n) * p->esize + 255) / 256 * 256 + (qft_workspace_size(p) + 255) / 256 * 256;
}

// A single request whose input and output are both device buffers at 256-byte
// alignment runs out of place straight from the input into the output: its
// first pass reads the caller's input, its last pass writes the caller's
// output, and it needs only a workspace (no state buffer and no copies).
bool direct_path(const qft_request& r) {
    return r.input_on_device && r.output_on_device && !(reinterpret_cast<uintptr_t>(r.input) & 255) &&
           !(reinterpret_cast<uintptr_t>(r.output) & 255);
}

// Device buffer of at least `bytes` from the pool (an idle buffer of up to
// twice the size is reused), or a new allocation; idle pooled buffers are
// freed first if a new allocation would exceed the budget.  *got = its size.
void* pool_get(qft_server_s* s, size_t bytes, size_t* got) {
    auto it = s->pool.lower_bound(bytes);
    if (it != s->pool.end() && it->first <= bytes * 2) {
        void* p = it->second;
        *got = it->first;
        s->pooled -= it->first;
        s->pool.erase(it);
        return p;
    }
    while (!s->pool.empty() && s->in_use + s->pooled + bytes > s->budget) {
        auto v = s->pool.begin();
        cudaFree(v->second);
        s->pooled -= v->first;
        s->pool.erase(v);
    }
    void* p = nullptr;
    if (s->fail_allocs > 0) {  // injected failure (test hook)
        --s->fail_allocs;
        return nullptr;
    }
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    *got = bytes;
    return p;
}

void pool_put(qft_server_s* s, void* p, size_t bytes) {
    s->pool.emplace(bytes, p);
    s->pooled += bytes;
}

qft_plan_t get_plan(qft_server_s* s, const qft_request& r) {
    const int kk = (r.k < 0 || r.k > r.n - 1) ? -1 : r.k;
    auto key = std::make_tuple(r.n, kk, r.direction, r.dtype, r.order);
    auto it = s->plans.find(key);
    if (it != s->plans.end()) return it->second;
    qft_opts o{};
    o.order = r.order;
    qft_plan_t p = nullptr;
    if (qft_plan_create(&p, r.n, kk, r.direction, r.dtype, &o) != QFT_OK) return nullptr;
    s->plans[key] = p;
    return p;
}

void finish(qft_server_s* s, const Request& rq, int status, double scale_in) {
    const auto now = Clock::now();
    Result& res = s->results[rq.ticket];
    res.status = status;
    res.scale_in = scale_in;
    res.latency_ms = std::chrono::duration<double, std::milli>(now - rq.t_submit).count();
    if (status == QFT_OK) {
        s->latencies.push_back(res.latency_ms);
        if (s->completed == 0) s->t_first = rq.t_submit;
        s->t_last = now;
        ++s->completed;
    } else {
        ++s->failed;
    }
}

bool batchable(const qft_server_s* s, qft_plan_t p) {
    return s->batch_max_n > 0 && p->n <= s->batch_max_n && !p->precision && p->threads != 512 && p->n_addr == p->n &&
           !s->bslots.empty();
}

size_t state_bytes(qft_plan_t p) { return ((size_t(1) << p->n) * p->esize + 255) / 256 * 256; }

// Launch the oldest requests of one forming batch into a free slot; returns
// QFT_OK (launched), QFT_ERR_NOMEM (no workspace memory now: retry later) or
// an error for the requests taken.
int launch_batch_slot(qft_server_s* s, Slot& slot, std::vector<InFlight>& group, int scale_mode) {
    const size_t take = std::min(group.size(), static_cast<size_t>(kSlotTransforms));
    std::vector<qft_plan_t> plans(take);
    std::vector<void*> states(take);
    size_t items = 0;
    size_t cnt = 0;
    for (; cnt < take; ++cnt) {
        qft_plan_t p = group[cnt].plan;
        size_t it = 0;
        for (const auto& ph : p->passes) it += static_cast<size_t>(ph.prm.num_tiles);
        if (items + it > kSlotItems) break;
        items += it;
        plans[cnt] = p;
        states[cnt] = group[cnt].state;
    }
    plans.resize(cnt);
    states.resize(cnt);
    const int count = static_cast<int>(cnt);
    const size_t wsb = qft::batch_workspace_bytes(plans.data(), count);  // held in the budget since admission
    size_t got = 0;
    void* ws = pool_get(s, wsb, &got);
    if (!ws) return QFT_ERR_NOMEM;
    qft::BatchTables T;
    int rc = qft::batch_build(plans.data(), states.data(), count, ws, got, slot.S.d_scale, scale_mode, true, T);
    cudaStream_t st = s->batch_stream;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < count && rc == QFT_OK && e == cudaSuccess; ++i) {
        const qft_request& r = group[i].req.r;
        e = cudaMemcpyAsync(states[i], r.input, (size_t(1) << r.n) * plans[i]->esize,
                            r.input_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    }
    if (rc == QFT_OK && e == cudaSuccess) rc = qft::slot_run(slot.S, T, st);
    for (int i = 0; i < count && rc == QFT_OK && e == cudaSuccess; ++i) {
        const qft_request& r = group[i].req.r;
        e = cudaMemcpyAsync(r.output, states[i], (size_t(1) << r.n) * plans[i]->esize,
                            r.output_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    }
    if (rc == QFT_OK && e == cudaSuccess)
        e = cudaMemcpyAsync(slot.h_scale, slot.S.d_scale, sizeof(double) * count, cudaMemcpyDeviceToHost, st);
    if (rc == QFT_OK && e == cudaSuccess)
        e = cudaMemcpyAsync(slot.h_scale + kSlotTransforms, slot.S.D.counters + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (rc == QFT_OK && e == cudaSuccess) e = cudaEventRecord(slot.done, st);
    if (rc == QFT_OK && e != cudaSuccess) rc = qft::set_cuda_error(e);
    if (rc != QFT_OK) {
        pool_put(s, ws, got);
        return rc == QFT_ERR_NOMEM ? QFT_ERR_CUDA : rc;
    }
    slot.busy = true;
    slot.ws = ws;
    slot.ws_bytes = got;
    slot.reqs.assign(group.begin(), group.begin() + count);
    group.erase(group.begin(), group.begin() + count);
    s->forming_count -= count;
    s->batched_count += count;
    s->batches_launched += 1;
    s->batched_requests += count;
    return QFT_OK;
}

// Issue one admitted request; returns false if it could not be issued.
int issue(qft_server_s* s, InFlight& f) {
    const qft_request& r = f.req.r;
    const size_t N = size_t(1) << r.n;
    const size_t sbytes = N * f.plan->esize;
    cudaStream_t st = s->streams[f.stream];
    if (f.direct) {
        const int rc = qft_execute_oop(f.plan, r.input, r.output, f.ws, nullptr, r.scale_mode,
                                       reinterpret_cast<qft_stream_t>(st));
        if (rc != QFT_OK) return rc;
        cudaError_t e = cudaMemcpyAsync(f.h_slot, f.ws, 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaEventRecord(f.done, st);
        return e == cudaSuccess ? QFT_OK : qft::set_cuda_error(e);
    }
    cudaError_t e = cudaMemcpyAsync(f.state, r.input, sbytes,
                                    r.input_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return qft::set_cuda_error(e);
    int rc = qft_execute(f.plan, f.state, f.ws, nullptr, r.scale_mode, reinterpret_cast<qft_stream_t>(st));
    if (rc != QFT_OK) return rc;
    e = cudaMemcpyAsync(r.output, f.state, sbytes, r.output_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        st);
    // scale_in (offset 0) and the status word (offset 8) of the workspace in one copy
    if (e == cudaSuccess) e = cudaMemcpyAsync(f.h_slot, f.ws, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(f.done, st);
    return e == cudaSuccess ? QFT_OK : qft::set_cuda_error(e);
}

void fail_request(qft_server_s* s, InFlight& f, int rc) {
    finish(s, f.req, rc, 0.0);
    pool_put(s, f.state, f.bytes);
    s->in_use -= f.bytes + f.reserve;
    s->cv_done.notify_all();
}

void worker_loop(qft_server_s* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (true) {
        // 1. retire finished requests
        for (size_t i = 0; i < s->inflight.size();) {
            InFlight& f = s->inflight[i];
            const cudaError_t q = cudaEventQuery(f.done);
            if (q == cudaErrorNotReady) { ++i; continue; }
            int rc = QFT_OK;
            if (q != cudaSuccess) rc = qft::set_cuda_error(q);
            else {
                int32_t dev_status;
                std::memcpy(&dev_status, f.h_slot + 1, sizeof(dev_status));
                if (dev_status != 0) rc = dev_status;
            }
            const double scale_in = f.h_slot[0];
            finish(s, f.req, rc, scale_in);
            if (rc == QFT_OK && f.req.r.scale_in_out) *f.req.r.scale_in_out = scale_in;
            pool_put(s, f.state, f.bytes);
            s->in_use -= f.bytes;
            s->stream_load[f.stream]--;
            s->free_slots.push_back(f.slot);
            cudaEventDestroy(f.done);
            s->inflight[i] = s->inflight.back();
            s->inflight.pop_back();
            s->cv_done.notify_all();
        }
        // ... and finished batches
        for (Slot& slot : s->bslots) {
            if (!slot.busy) continue;
            const cudaError_t q = cudaEventQuery(slot.done);
            if (q == cudaErrorNotReady) continue;
            int rc = QFT_OK;
            if (q != cudaSuccess) rc = qft::set_cuda_error(q);
            else {
                int32_t dev_status;
                std::memcpy(&dev_status, slot.h_scale + kSlotTransforms, sizeof(dev_status));
                if (dev_status != 0) rc = dev_status;
            }
            for (size_t i = 0; i < slot.reqs.size(); ++i) {
                InFlight& f = slot.reqs[i];
                const double scale_in = slot.h_scale[i];
                finish(s, f.req, rc, scale_in);
                if (rc == QFT_OK && f.req.r.scale_in_out) *f.req.r.scale_in_out = scale_in;
                pool_put(s, f.state, f.bytes);
                s->in_use -= f.bytes + f.reserve;
            }
            s->batched_count -= static_cast<long long>(slot.reqs.size());
            slot.reqs.clear();
            pool_put(s, slot.ws, slot.ws_bytes);
            slot.ws = nullptr;
            slot.busy = false;
            s->cv_done.notify_all();
        }
        // 2. admit in arrival order while budget and slots allow
        auto active = [&]() {
            return static_cast<long long>(s->inflight.size()) + s->forming_count + s->batched_count;
        };
        while (!s->pending.empty() && active() < s->max_inflight) {
            Request& rq = s->pending.front();
            qft_plan_t p = get_plan(s, rq.r);
            if (!p) { finish(s, rq, QFT_ERR_BAD_ARG, 0.0); s->pending.pop_front(); s->cv_done.notify_all(); continue; }
            const bool small = batchable(s, p);
            const bool direct = !small && direct_path(rq.r);
            const size_t bytes = small ? state_bytes(p)
                                       : direct ? (qft_workspace_size(p) + 255) / 256 * 256 : request_bytes(p);
            const size_t reserve = small ? qft::batch_transform_workspace_bytes(p) + 256 : 0;
            if (bytes + reserve > s->budget) { finish(s, rq, QFT_ERR_BUDGET, 0.0); s->pending.pop_front(); s->cv_done.notify_all(); continue; }
            if (s->in_use + bytes + reserve > s->budget) break;  // wait for memory to free up (keeps arrival order)
            InFlight f;
            f.req = rq;
            f.plan = p;
            f.state = pool_get(s, bytes, &f.bytes);
            if (!f.state) {
                // no memory: wait for running requests to free some; with
                // nothing running no progress is possible, so report it
                if (active() > 0) break;
                finish(s, rq, QFT_ERR_NOMEM, 0.0);
                s->pending.pop_front();
                s->cv_done.notify_all();
                continue;
            }
            s->pending.pop_front();
            f.reserve = reserve;
            s->in_use += f.bytes + reserve;
            if (small) {
                s->forming[std::make_tuple(p->dtype, p->dir, f.req.r.scale_mode)].push_back(f);
                s->forming_count += 1;
                continue;
            }
            f.direct = direct;
            f.ws = direct ? static_cast<char*>(f.state) : static_cast<char*>(f.state) + state_bytes(p);
            f.stream = static_cast<int>(std::min_element(s->stream_load.begin(), s->stream_load.end()) - s->stream_load.begin());
            f.slot = s->free_slots.back();
            s->free_slots.pop_back();
            f.h_slot = s->slots + 2 * f.slot;
            cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming);
            const int rc = issue(s, f);
            if (rc != QFT_OK) {
                s->free_slots.push_back(f.slot);
                cudaEventDestroy(f.done);
                fail_request(s, f, rc);
                continue;
            }
            s->stream_load[f.stream]++;
            s->inflight.push_back(f);
        }
        // 3. launch forming batches into free slots, oldest group first
        while (s->forming_count > 0) {
            Slot* slot = nullptr;
            for (Slot& sl : s->bslots)
                if (!sl.busy) { slot = &sl; break; }
            if (!slot) break;
            auto oldest = s->forming.end();
            for (auto it = s->forming.begin(); it != s->forming.end(); ++it)
                if (!it->second.empty() &&
                    (oldest == s->forming.end() || it->second.front().req.t_submit < oldest->second.front().req.t_submit))
                    oldest = it;
            if (oldest == s->forming.end()) break;
            const int rc = launch_batch_slot(s, *slot, oldest->second, std::get<2>(oldest->first));
            if (rc == QFT_ERR_NOMEM) {
                // no workspace memory now: retry on the next pass while others run; with
                // nothing running no progress is possible, so the group fails
                bool running = !s->inflight.empty();
                for (const Slot& sl : s->bslots) running = running || sl.busy;
                if (running) break;
                for (InFlight& f : oldest->second) fail_request(s, f, QFT_ERR_NOMEM);
                s->forming_count -= static_cast<long long>(oldest->second.size());
                oldest->second.clear();
                continue;
            }
            if (rc != QFT_OK) {              // the oldest request of the group fails; the rest retry
                InFlight f = oldest->second.front();
                oldest->second.erase(oldest->second.begin());
                s->forming_count -= 1;
                fail_request(s, f, rc);
            }
        }
        bool busy_slots = false;
        for (const Slot& sl : s->bslots) busy_slots = busy_slots || sl.busy;
        if (s->stop && s->pending.empty() && s->inflight.empty() && s->forming_count == 0 && !busy_slots) break;
        if (s->inflight.empty() && !busy_slots && s->forming_count == 0) {
            s->cv_work.wait_for(lock, std::chrono::milliseconds(2));
        } else {
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lock.lock();
        }
    }
}

}  // namespace

extern "C" {

int qft_server_create(qft_server_t* out, size_t hbm_budget_bytes, int streams, int max_inflight) {
    if (!out) return QFT_ERR_BAD_ARG;
    *out = nullptr;
    if (hbm_budget_bytes == 0 || streams < 0 || streams > 64 || max_inflight < 0 || max_inflight > 4096)
        return QFT_ERR_BAD_ARG;
    qft_server_s* s = new (std::nothrow) qft_server_s();
    if (!s) return QFT_ERR_NOMEM;
    s->budget = hbm_budget_bytes;
    if (streams) s->nstreams = streams;
    if (max_inflight) s->max_inflight = max_inflight;
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return QFT_ERR_CUDA; }
    for (int i = 0; i < s->nstreams; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto x : s->streams) cudaStreamDestroy(x);
            delete s;
            return QFT_ERR_CUDA;
        }
        s->streams.push_back(st);
    }
    s->stream_load.assign(s->nstreams, 0);
    if (cudaMallocHost(&s->slots, 2 * sizeof(double) * s->max_inflight) != cudaSuccess) {
        for (auto x : s->streams) cudaStreamDestroy(x);
        delete s;
        return QFT_ERR_NOMEM;
    }
    for (int i = s->max_inflight - 1; i >= 0; --i) s->free_slots.push_back(i);
    // continuous batching: a high-priority stream and three batch slots
    {
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        bool ok = cudaStreamCreateWithPriority(&s->batch_stream, cudaStreamNonBlocking, greatest) == cudaSuccess;
        for (int i = 0; i < 3 && ok; ++i) {
            Slot sl;
            ok = qft::slot_create(sl.S, kSlotTransforms, kSlotItems) == QFT_OK &&
                 cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
                 cudaMallocHost(&sl.h_scale, sizeof(double) * (kSlotTransforms + 1)) == cudaSuccess;
            if (ok) s->bslots.push_back(sl);
            else {
                qft::slot_destroy(sl.S);
                if (sl.done) cudaEventDestroy(sl.done);
            }
        }
        if (!ok) cudaGetLastError();  // batching unavailable: every request runs on its own
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return QFT_OK;
}

int qft_server_submit(qft_server_t s, const qft_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket || !req->input || !req->output) return QFT_ERR_BAD_ARG;
    if (req->dtype != QFT_C64 && req->dtype != QFT_C128) return QFT_ERR_BAD_ARG;
    if (req->direction != QFT_FORWARD && req->direction != QFT_INVERSE) return QFT_ERR_BAD_ARG;
    if (req->n < 1 || req->n > (req->dtype == QFT_C64 ? 34 : 33)) return QFT_ERR_BAD_ARG;
    if (req->scale_mode < QFT_SCALE_STATE || req->scale_mode > QFT_SCALE_INV_N) return QFT_ERR_BAD_ARG;
    Request r;
    r.r = *req;
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stop) return QFT_ERR_STATE;
        r.ticket = s->next_ticket++;
        s->results[r.ticket] = Result{};
        s->pending.push_back(r);
    }
    s->cv_work.notify_one();
    *ticket = r.ticket;
    return QFT_OK;
}

int qft_server_poll(qft_server_t s, uint64_t ticket, int* done) {
    if (!s || !done) return QFT_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return QFT_ERR_STATE;
    *done = it->second.status != 1;
    return it->second.status == 1 ? QFT_OK : it->second.status;
}

int qft_server_wait(qft_server_t s, uint64_t ticket, int timeout_ms, double* latency_ms) {
    if (!s) return QFT_ERR_BAD_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return QFT_ERR_STATE;
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (s->results[ticket].status == 1) {
        if (timeout_ms >= 0 && s->cv_done.wait_until(lock, deadline) == std::cv_status::timeout &&
            s->results[ticket].status == 1)
            return QFT_ERR_TIMEOUT;
        if (timeout_ms < 0) s->cv_done.wait_for(lock, std::chrono::milliseconds(10));
    }
    const Result res = s->results[ticket];
    if (latency_ms) *latency_ms = res.latency_ms;
    s->results.erase(ticket);
    return res.status;
}

int qft_server_cancel(qft_server_t s, uint64_t ticket) {
    if (!s) return QFT_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
        if (it->ticket != ticket) continue;
        Result& res = s->results[ticket];
        res.status = QFT_ERR_CANCELED;
        res.latency_ms = 0.0;
        s->pending.erase(it);
        s->cv_done.notify_all();
        return QFT_OK;
    }
    return QFT_ERR_STATE;
}

int qft_server_set_batching(qft_server_t s, int max_n) {
    if (!s || max_n < 0 || max_n > 34) return QFT_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    s->batch_max_n = max_n;
    return QFT_OK;
}

int qft_server_inject_alloc_failures(qft_server_t s, int count) {
    if (!s || count < 0) return QFT_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    s->fail_allocs = count;
    return QFT_OK;
}

int qft_server_get_stats(qft_server_t s, qft_server_stats* out) {
    if (!s || !out) return QFT_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = static_cast<long long>(s->completed);
    out->failed = static_cast<long long>(s->failed);
    out->pending = static_cast<long long>(s->pending.size());
    out->in_flight = static_cast<long long>(s->inflight.size());
    out->bytes_in_use = s->in_use;
    out->bytes_pooled = s->pooled;
    out->batches = s->batches_launched;
    out->batched_requests = s->batched_requests;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        auto pct = [&](double p) {
            const size_t i = std::min(v.size() - 1, static_cast<size_t>(p * (v.size() - 1) + 0.5));
            std::nth_element(v.begin(), v.begin() + i, v.end());
            return v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = *std::max_element(s->latencies.begin(), s->latencies.end());
        const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
        out->requests_per_s = span > 0 ? static_cast<double>(s->completed) / span : 0.0;
    }
    return QFT_OK;
}

int qft_server_reset_stats(qft_server_t s) {
    if (!s) return QFT_ERR_BAD_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    s->latencies.clear();
    s->completed = 0;
    s->failed = 0;
    s->batches_launched = 0;
    s->batched_requests = 0;
    return QFT_OK;
}

int qft_server_destroy(qft_server_t s) {
    if (!s) return QFT_ERR_BAD_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& kv : s->pool) cudaFree(kv.second);
    for (auto& kv : s->plans) qft_plan_destroy(kv.second);
    for (auto st : s->streams) cudaStreamDestroy(st);
    for (Slot& sl : s->bslots) {
        qft::slot_destroy(sl.S);
        cudaEventDestroy(sl.done);
        cudaFreeHost(sl.h_scale);
    }
    if (s->batch_stream) cudaStreamDestroy(s->batch_stream);
    cudaFreeHost(s->slots);
    delete s;
    return QFT_OK;
}

}  // extern "C"
