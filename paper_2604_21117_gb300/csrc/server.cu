// Serving loop: continuous batching of point-lookup requests.
//
// The paper times a host that writes a batch, runs the kernel and reads the
// results, and notes that with pipelining the host transfers overlap the
// kernel (Sec. V-B, Fig. 7).  This runtime serves a stream of small requests
// that way: submitted requests wait per tree; a worker thread forms a batch
// of one tree's requests when the oldest has waited `deadline_us` or the
// batch is full, and runs it on a free slot -- its own CUDA stream with
// page-locked staging, device buffers and workspace: host-to-device copy,
// search (plain or learned), device-to-host copy, event.  Several slots are
// in flight at once, so batches overlap on the device while new requests
// keep arriving and are admitted into the next batch as slots free up.
// Work is admitted by memory: a batch is issued only while the staging bytes
// of all batches in flight stay under the cap.  When a slot's event has
// completed, its results are copied into each request's own output buffers
// and the request's latency (completion minus submission) is recorded.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "bt_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_us()
{
    return std::chrono::duration<double, std::micro>(Clock::now().time_since_epoch()).count();
}

struct Request {
    uint32_t tree;
    uint32_t count;
    const void *keys;
    void *vals;
    uint8_t *found;
    uint64_t ticket;
    double t_submit;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    unsigned char *h_q = nullptr, *h_v = nullptr, *h_f = nullptr;  // page-locked staging
    unsigned char *d_q = nullptr, *d_v = nullptr, *d_f = nullptr;
    void *d_ws = nullptr;
    uint64_t ws_bytes = 0;
    bool busy = false;
    uint64_t bytes = 0;
    std::vector<Request> reqs;
};

}  // namespace

struct bt_server {
    std::vector<const bt_tree *> trees;
    std::vector<const bt_model *> models;
    bt_server_opts opts;
    int key_bytes = 8, val_bytes = 8;
    std::vector<Slot> slots;
    std::mutex mu;
    std::vector<std::deque<Request>> pending;
    uint64_t pending_bytes = 0;
    uint64_t inflight_bytes = 0;
    uint64_t next_ticket = 1;
    std::vector<uint64_t> done_tickets;
    std::vector<float> latencies;  // per completed request, us
    uint64_t completed = 0, lookups = 0, batches = 0, submitted = 0;
    uint64_t failed = 0;  // requests of batches that could not be issued
    uint32_t max_inflight_seen = 0;
    std::atomic<bool> stop{false};
    std::thread worker;
    int device = 0;
    bt_status worker_status = BT_OK;
};

namespace {

uint64_t req_bytes(const bt_server *s, uint32_t count)
{
    return static_cast<uint64_t>(count) * (s->key_bytes + s->val_bytes + 1);
}

// Copy finished slots' results to their requests; returns true if any.
bool retire(bt_server *S)
{
    bool any = false;
    for (Slot &sl : S->slots) {
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
            btgb::set_error_detail("server batch", q);
            S->worker_status = BT_ERR_CUDA;
        }
        uint64_t off = 0;
        const double t = now_us();
        std::vector<float> lat;
        lat.reserve(sl.reqs.size());
        for (const Request &r : sl.reqs) {
            memcpy(r.vals, sl.h_v + off * S->val_bytes, static_cast<size_t>(r.count) * S->val_bytes);
            memcpy(r.found, sl.h_f + off, r.count);
            off += r.count;
            lat.push_back(static_cast<float>(t - r.t_submit));
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (size_t i = 0; i < sl.reqs.size(); ++i) {
                S->done_tickets.push_back(sl.reqs[i].ticket);
                S->latencies.push_back(lat[i]);
            }
            S->completed += sl.reqs.size();
            S->lookups += off;
            S->inflight_bytes -= sl.bytes;
        }
        sl.reqs.clear();
        sl.busy = false;
        any = true;
    }
    return any;
}

// Form and issue at most one batch; returns true if it issued one.
bool issue(bt_server *S)
{
    Slot *free_slot = nullptr;
    uint32_t inflight = 0;
    for (Slot &sl : S->slots) {
        if (!sl.busy && !free_slot) free_slot = &sl;
        inflight += sl.busy ? 1u : 0u;
    }
    if (!free_slot) return false;
    Slot &sl = *free_slot;
    const double t = now_us();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        // the tree whose oldest request has waited longest
        int best = -1;
        double oldest = 0;
        for (size_t i = 0; i < S->pending.size(); ++i) {
            if (S->pending[i].empty()) continue;
            if (best < 0 || S->pending[i].front().t_submit < oldest) {
                best = static_cast<int>(i);
                oldest = S->pending[i].front().t_submit;
            }
        }
        if (best < 0) return false;
        std::deque<Request> &pq = S->pending[best];
        uint64_t total = 0;
        for (const Request &r : pq) {
            total += r.count;
            if (total >= S->opts.max_batch) break;
        }
        const bool due = (t - oldest) >= S->opts.deadline_us || total >= S->opts.max_batch;
        if (!due) return false;
        // take requests up to the batch limit, admitted by memory
        uint32_t n = 0;
        uint64_t bytes = 0;
        while (!pq.empty() && n + pq.front().count <= S->opts.max_batch) {
            const uint64_t b = req_bytes(S, pq.front().count);
            if (S->inflight_bytes + bytes + b > S->opts.mem_cap_bytes && n > 0) break;
            if (S->inflight_bytes + bytes + b > S->opts.mem_cap_bytes && inflight > 0) break;
            sl.reqs.push_back(pq.front());
            n += pq.front().count;
            bytes += b;
            S->pending_bytes -= b;
            pq.pop_front();
        }
        if (n == 0) return false;
        S->inflight_bytes += bytes;
        sl.bytes = bytes;
        S->batches += 1;
        S->max_inflight_seen = std::max(S->max_inflight_seen, inflight + 1);
    }
    // stage keys, then copy in, search, copy out, mark done
    uint64_t off = 0;
    for (const Request &r : sl.reqs) {
        memcpy(sl.h_q + off * S->key_bytes, r.keys, static_cast<size_t>(r.count) * S->key_bytes);
        off += r.count;
    }
    const uint32_t tree = sl.reqs.front().tree;
    const bt_stream bs = reinterpret_cast<bt_stream>(sl.stream);
    cudaError_t e = cudaMemcpyAsync(sl.d_q, sl.h_q, off * S->key_bytes, cudaMemcpyHostToDevice, sl.stream);
    bt_status st = BT_OK;
    if (e == cudaSuccess) {
        if (S->models[tree])
            st = bt_learned_search_batch(S->trees[tree], S->models[tree], sl.d_q, off, sl.d_v, sl.d_f, sl.d_ws,
                                         sl.ws_bytes, bs);
        else
            st = bt_search_batch(S->trees[tree], sl.d_q, off, sl.d_v, sl.d_f, sl.d_ws, sl.ws_bytes, bs);
    }
    if (e == cudaSuccess && st == BT_OK)
        e = cudaMemcpyAsync(sl.h_v, sl.d_v, off * S->val_bytes, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess && st == BT_OK) e = cudaMemcpyAsync(sl.h_f, sl.d_f, off, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess && st == BT_OK) e = cudaEventRecord(sl.done, sl.stream);
    if (e != cudaSuccess || st != BT_OK) {
        // the batch never ran: its requests are not reported done (the
        // server's status, returned by every later call, says why), and no
        // results are copied into their buffers
        if (e != cudaSuccess) btgb::set_error_detail("server issue", e);
        std::lock_guard<std::mutex> lk(S->mu);
        S->worker_status = st != BT_OK ? st : BT_ERR_CUDA;
        S->failed += sl.reqs.size();
        S->inflight_bytes -= sl.bytes;
        sl.reqs.clear();
        return true;
    }
    sl.busy = true;
    return true;
}

void worker_main(bt_server *S)
{
    cudaSetDevice(S->device);
    while (!S->stop.load(std::memory_order_acquire)) {
        const bool r = retire(S);
        const bool i = issue(S);
        if (!r && !i) std::this_thread::yield();
    }
    // drain: finish everything already admitted or pending
    for (;;) {
        retire(S);
        bool idle;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            idle = true;
            for (auto &p : S->pending) idle &= p.empty();
        }
        bool busy = false;
        for (Slot &sl : S->slots) busy |= sl.busy;
        if (idle && !busy) break;
        if (!issue(S)) std::this_thread::yield();
    }
}

void free_slots(bt_server *S)
{
    for (Slot &sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.h_q) cudaFreeHost(sl.h_q);
        if (sl.h_v) cudaFreeHost(sl.h_v);
        if (sl.h_f) cudaFreeHost(sl.h_f);
        if (sl.d_q) cudaFree(sl.d_q);
        if (sl.d_v) cudaFree(sl.d_v);
        if (sl.d_f) cudaFree(sl.d_f);
        if (sl.d_ws) cudaFree(sl.d_ws);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
}

}  // namespace

extern "C" bt_status bt_server_create(const bt_tree *const *trees, const bt_model *const *models, uint32_t ntrees,
                                      const bt_server_opts *opts, bt_server **out)
{
    if (!trees || !opts || !out || ntrees == 0) return BT_ERR_ARG;
    if (opts->slots == 0 || opts->slots > 64 || opts->max_batch == 0 || opts->max_batch > (1u << 24))
        return BT_ERR_ARG;
    for (uint32_t i = 0; i < ntrees; ++i) {
        if (!trees[i] || trees[i]->dev.key_bytes != trees[0]->dev.key_bytes ||
            trees[i]->dev.val_bytes != trees[0]->dev.val_bytes)
            return BT_ERR_ARG;
        if (models && models[i] &&
            (trees[i]->dev.height == 0 || models[i]->dev.leaves != trees[i]->dev.nodes[trees[i]->dev.height - 1]))
            return BT_ERR_ARG;
    }
    bt_server *S = new (std::nothrow) bt_server;
    if (!S) return BT_ERR_NOMEM;
    S->trees.assign(trees, trees + ntrees);
    S->models.assign(ntrees, nullptr);
    if (models) S->models.assign(models, models + ntrees);
    S->opts = *opts;
    if (S->opts.mem_cap_bytes == 0) S->opts.mem_cap_bytes = ~0ull;
    S->key_bytes = trees[0]->dev.key_bytes;
    S->val_bytes = trees[0]->dev.val_bytes;
    S->pending.resize(ntrees);
    cudaGetDevice(&S->device);
    S->slots.resize(opts->slots);
    const uint64_t B = opts->max_batch;
    uint64_t ws = 0;
    for (uint32_t i = 0; i < ntrees; ++i) ws = std::max<uint64_t>(ws, bt_search_workspace_bytes(trees[i], B));
    cudaError_t e = cudaSuccess;
    for (Slot &sl : S->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_q, B * S->key_bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_v, B * S->val_bytes);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_f, B);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_q, B * S->key_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_v, B * S->val_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_f, B);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_ws, ws > 0 ? ws : 256);
        sl.ws_bytes = ws;
    }
    if (e != cudaSuccess) {
        btgb::set_error_detail("server buffers", e);
        free_slots(S);
        delete S;
        return e == cudaErrorMemoryAllocation ? BT_ERR_NOMEM : BT_ERR_CUDA;
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return BT_OK;
}

extern "C" bt_status bt_server_submit(bt_server *S, uint32_t tree, const void *h_keys, uint32_t count,
                                      void *h_out_vals, uint8_t *h_out_found, uint64_t *ticket)
{
    if (!S || tree >= S->trees.size() || count == 0 || !h_keys || !h_out_vals || !h_out_found) return BT_ERR_ARG;
    if (count > S->opts.max_batch) return BT_ERR_ARG;
    const uint64_t b = req_bytes(S, count);
    // a request larger than the pending cap could never be admitted
    if (S->opts.pending_cap_bytes && b > S->opts.pending_cap_bytes) return BT_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->worker_status != BT_OK) return S->worker_status;
    if (S->opts.pending_cap_bytes && S->pending_bytes + b > S->opts.pending_cap_bytes) return BT_ERR_NOMEM;
    Request r{tree, count, h_keys, h_out_vals, h_out_found, S->next_ticket++, now_us()};
    S->pending[tree].push_back(r);
    S->pending_bytes += b;
    S->submitted += 1;
    if (ticket) *ticket = r.ticket;
    return BT_OK;
}

extern "C" bt_status bt_server_poll(bt_server *S, uint64_t *tickets, uint32_t max, uint32_t *n)
{
    if (!S || !n || (max && !tickets)) return BT_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    const uint32_t k = static_cast<uint32_t>(std::min<size_t>(max, S->done_tickets.size()));
    for (uint32_t i = 0; i < k; ++i) tickets[i] = S->done_tickets[i];
    S->done_tickets.erase(S->done_tickets.begin(), S->done_tickets.begin() + k);
    *n = k;
    return S->worker_status;
}

extern "C" bt_status bt_server_drain(bt_server *S, double timeout_s)
{
    if (!S) return BT_ERR_ARG;
    const double t_end = now_us() + timeout_s * 1e6;
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->worker_status != BT_OK) return S->worker_status;
            if (S->completed + S->failed == S->submitted) return BT_OK;
        }
        if (now_us() > t_end) return BT_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" bt_status bt_server_get_stats(bt_server *S, bt_server_stats *out, int reset)
{
    if (!S || !out) return BT_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->lookups = S->lookups;
    out->batches = S->batches;
    out->max_inflight = S->max_inflight_seen;
    if (!S->latencies.empty()) {
        std::vector<float> l = S->latencies;
        std::sort(l.begin(), l.end());
        out->p50_us = l[l.size() / 2];
        out->p99_us = l[std::min(l.size() - 1, static_cast<size_t>(0.99 * l.size()))];
        out->max_us = l.back();
    }
    if (reset) {
        S->latencies.clear();
        S->submitted -= S->completed;
        S->completed = 0;
        S->lookups = 0;
        S->batches = 0;
        S->max_inflight_seen = 0;
    }
    return S->worker_status;
}

extern "C" void bt_server_destroy(bt_server *S)
{
    if (!S) return;
    S->stop.store(true, std::memory_order_release);
    if (S->worker.joinable()) S->worker.join();
    free_slots(S);
    delete S;
}

extern "C" bt_status bt_server_run_trace(bt_server *S, uint64_t n, const double *t_arrival_s, const uint32_t *tree,
                                         const uint32_t *count, const uint64_t *key_offset, const void *h_keys,
                                         void *h_out_vals, uint8_t *h_out_found, double *wall_s)
{
    if (!S || (n && (!t_arrival_s || !tree || !count || !key_offset || !h_keys || !h_out_vals || !h_out_found)))
        return BT_ERR_ARG;
    const unsigned char *k = static_cast<const unsigned char *>(h_keys);
    unsigned char *v = static_cast<unsigned char *>(h_out_vals);
    const double t0 = now_us();
    for (uint64_t i = 0; i < n; ++i) {
        const double due = t0 + t_arrival_s[i] * 1e6;
        while (now_us() < due) {
        }
        bt_status st;
        for (;;) {  // back-pressure: retry while the pending cap is full
            st = bt_server_submit(S, tree[i], k + key_offset[i] * S->key_bytes, count[i],
                                  v + key_offset[i] * S->val_bytes, h_out_found + key_offset[i], nullptr);
            if (st != BT_ERR_NOMEM) break;
            std::this_thread::yield();
        }
        if (st != BT_OK) return st;
    }
    const bt_status st = bt_server_drain(S, 60.0);
    if (wall_s) *wall_s = (now_us() - t0) / 1e6;
    return st;
}
