// Serving loop: continuous batching of point-lookup requests.
//
// The paper times a host that writes a batch, runs the kernel and reads the
// results, and notes that with pipelining the host transfers overlap the
// kernel (Sec. V-B, Fig. 7).  This runtime serves a stream of small requests
// that way, with the host transfers replaced by device reads and writes of
// host memory:
//
// - Submission (any thread) copies a request's keys into its tree's ring of
//   lookups: page-locked, device-mapped host memory, one region per tree.
// - A worker thread forms a batch when the oldest waiting request has waited
//   `deadline_us` or a full batch is waiting: it takes waiting requests of
//   every tree (up to max_batch lookups, admitted while the bytes of all
//   batches in flight stay under the memory cap), describes each tree's
//   contiguous ring stretch as one work-list entry, and issues one launch of
//   the multi-tree batching kernel on a free slot (its own stream).  The
//   kernel reads the keys from the rings and writes values and found flags
//   back into them, then its last block raises the slot's flag in host
//   memory -- one API call per batch, no copies, no events.
// - Several slots are in flight at once, so batches overlap on the device
//   while new requests keep arriving and are admitted into the next batch.
//   Batches retire in issue order: the worker sees the flag, copies each
//   request's results into the request's own buffers, records its latency
//   (completion minus submission) and frees its ring space.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "bt_internal.h"
#include "forest.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_us()
{
    return std::chrono::duration<double, std::micro>(Clock::now().time_since_epoch()).count();
}

struct alignas(64) Request {  // one cache line each: the worker reads only finished ones
    uint32_t count;
    uint64_t pos;  // first lookup, as a running position of the tree's ring (ring index = pos % cap)
    void *vals;
    uint8_t *found;
    uint64_t ticket;
    double t_submit;
};

// One tree's ring of lookups (its stretch of the shared host arrays) and of
// requests.  Positions only grow; index = position % capacity.  Submitters
// (serialised by the server's submit lock) own `tail` and publish requests
// by `rtail`; the worker owns `rissued` and frees space through `head` and
// `rhead`.  The two sides' fields sit on separate cache lines, so a
// submission touches no line the worker writes except when a batch retires.
struct Ring {
    uint64_t base = 0;  // first lookup of this tree's stretch in the shared arrays
    uint64_t cap = 0;   // lookups
    std::vector<Request> req;
    alignas(128) uint64_t tail = 0;      // submitters
    std::atomic<uint64_t> rtail{0};      // submitters publish, the worker reads
    alignas(128) std::atomic<uint64_t> head{0};  // the worker frees, submitters read
    std::atomic<uint64_t> rhead{0};
    alignas(128) uint64_t rissued = 0;   // the worker only
    uint64_t rknown = 0;                 // requests whose counts the worker has added up
};

struct Slot {
    cudaStream_t stream = nullptr;
    bt_batch_desc *h_desc = nullptr;     // work list (host-mapped)
    uint32_t *h_cs = nullptr;            // its chunk offsets (host-mapped)
    unsigned long long *h_flag = nullptr;  // completion flag, written by the kernel (host-mapped)
    bt_batch_desc *d_desc = nullptr;     // device views of the same
    uint32_t *d_cs = nullptr;
    unsigned long long *d_flag = nullptr;
    unsigned int *d_counter = nullptr;   // arrivals of the launch's blocks (device)
    unsigned long long seq = 0;
    bool busy = false;
    double t_issue = 0;
    uint64_t bytes = 0, lookups = 0;
    std::vector<uint64_t> r0, r1;        // per tree: requests [r0, r1) of this batch
};

}  // namespace

struct bt_server {
    std::vector<const bt_tree *> trees;
    std::vector<const bt_model *> models;
    bt_forest *forest = nullptr;
    bt_server_opts opts;
    int key_bytes = 8, val_bytes = 8;
    uint32_t warps = 8;
    std::vector<Ring> rings;
    unsigned char *h_keys = nullptr, *h_vals = nullptr;  // shared lookup arrays (host-mapped)
    uint8_t *h_found = nullptr;
    void *d_keys = nullptr, *d_vals = nullptr;
    uint8_t *d_found = nullptr;
    uint64_t total_cap = 0;
    std::vector<Slot> slots;
    int device = 0;
    std::thread worker;
    // submitters (under sub_mu)
    alignas(128) std::mutex sub_mu;
    uint64_t next_ticket = 1;
    uint64_t sub_lookups = 0;    // lookups submitted
    uint64_t sub_bytes = 0;      // their bytes
    // the worker: written once per batch, read by submitters
    alignas(128) std::atomic<uint64_t> issued_bytes{0};
    // the worker only
    alignas(128) uint64_t inflight_bytes = 0;
    uint64_t known_lookups = 0;  // lookups published and not yet issued, as the worker has counted them
    std::deque<uint32_t> fifo;   // busy slots in issue order
    std::vector<uint64_t> rt_tmp;
    std::vector<size_t> order_tmp;
    std::vector<bt_batch_desc> desc_tmp;
    // completion records (under done_mu)
    alignas(128) std::mutex done_mu;
    std::vector<uint64_t> done_tickets;
    std::vector<float> latencies;  // per completed request, us
    uint64_t completed = 0, lookups = 0, batches = 0, failed = 0;
    uint64_t reset_base = 0;  // requests counted before the last statistics reset
    uint32_t max_inflight_seen = 0;
    // rarely written
    alignas(128) std::atomic<bool> stop{false};
    std::atomic<int> worker_status{BT_OK};
};

namespace {

uint64_t req_bytes(const bt_server *s, uint32_t count)
{
    return static_cast<uint64_t>(count) * (s->key_bytes + s->val_bytes + 1);
}

void fail(bt_server *S, bt_status st) { S->worker_status.store(st, std::memory_order_release); }

// Retire finished batches in issue order; returns true if any.
bool retire(bt_server *S)
{
    bool any = false;
    while (!S->fifo.empty()) {
        Slot &sl = S->slots[S->fifo.front()];
        const unsigned long long f = __atomic_load_n(sl.h_flag, __ATOMIC_ACQUIRE);
        if (f != sl.seq) {
            // a launch that failed never raises its flag: look at the stream
            // now and then
            if (now_us() - sl.t_issue > 100000.0) {
                const cudaError_t q = cudaStreamQuery(sl.stream);
                if (q != cudaErrorNotReady && q != cudaSuccess) {
                    btgb::set_error_detail("server batch", q);
                    fail(S, BT_ERR_CUDA);
                }
                sl.t_issue = now_us();
            }
            break;
        }
        const double t = now_us();
        std::vector<uint64_t> tickets;
        std::vector<float> lat;
        for (size_t i = 0; i < S->rings.size(); ++i) {
            Ring &R = S->rings[i];
            const uint64_t rc = R.req.size();
            uint64_t end = 0;
            for (uint64_t j = sl.r0[i]; j < sl.r1[i]; ++j) {
                const Request &r = R.req[j % rc];
                const uint64_t at = R.base + r.pos % R.cap;
                memcpy(r.vals, S->h_vals + at * S->val_bytes, static_cast<size_t>(r.count) * S->val_bytes);
                memcpy(r.found, S->h_found + at, r.count);
                tickets.push_back(r.ticket);
                lat.push_back(static_cast<float>(t - r.t_submit));
                end = r.pos + r.count;
            }
            if (sl.r1[i] > sl.r0[i]) {
                R.head.store(end, std::memory_order_release);
                R.rhead.store(sl.r1[i], std::memory_order_release);
            }
        }
        {
            std::lock_guard<std::mutex> lk(S->done_mu);
            S->done_tickets.insert(S->done_tickets.end(), tickets.begin(), tickets.end());
            S->latencies.insert(S->latencies.end(), lat.begin(), lat.end());
            S->completed += tickets.size();
            S->lookups += sl.lookups;
        }
        S->inflight_bytes -= sl.bytes;
        sl.busy = false;
        S->fifo.pop_front();
        any = true;
    }
    return any;
}

// Form and issue at most one batch; returns true if it issued one.
bool issue(bt_server *S, bool force)
{
    if (S->worker_status.load(std::memory_order_acquire) != BT_OK) return false;
    Slot *free_slot = nullptr;
    for (Slot &sl : S->slots)
        if (!sl.busy) {
            free_slot = &sl;
            break;
        }
    if (!free_slot) return false;
    const size_t nt = S->rings.size();
    // newly published requests, and the oldest waiting one; a batch is due
    // when that has waited the deadline or a full batch is waiting
    double oldest = 0;
    bool have = false;
    std::vector<uint64_t> &rt = S->rt_tmp;
    for (size_t i = 0; i < nt; ++i) {
        Ring &R = S->rings[i];
        rt[i] = R.rtail.load(std::memory_order_acquire);
        const uint64_t rc = R.req.size();
        for (; R.rknown < rt[i]; ++R.rknown) S->known_lookups += R.req[R.rknown % rc].count;
        if (R.rissued < rt[i]) {
            const double ts = R.req[R.rissued % rc].t_submit;
            if (!have || ts < oldest) oldest = ts;
            have = true;
        }
    }
    if (!have) return false;
    const double t = now_us();
    const bool due = force || (t - oldest) >= S->opts.deadline_us || S->known_lookups >= S->opts.max_batch;
    if (!due) return false;
    Slot &sl = *free_slot;
    // take waiting requests tree by tree (oldest tree first), up to the
    // batch limit, admitted by memory; each tree's run of ring positions
    // becomes work-list entries (a new entry where the run wraps)
    std::vector<size_t> &order = S->order_tmp;
    for (size_t i = 0; i < nt; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const Ring &A = S->rings[a], &B = S->rings[b];
        const bool ha = A.rissued < rt[a], hb = B.rissued < rt[b];
        if (ha != hb) return ha;
        if (!ha) return a < b;
        return A.req[A.rissued % A.req.size()].t_submit < B.req[B.rissued % B.req.size()].t_submit;
    });
    std::vector<bt_batch_desc> &desc = S->desc_tmp;
    desc.clear();
    uint64_t n = 0, bytes = 0;
    const bool idle = S->fifo.empty();
    for (size_t i = 0; i < nt; ++i) sl.r0[i] = sl.r1[i] = S->rings[i].rissued;
    bool full = false;
    for (size_t oi = 0; oi < nt && !full; ++oi) {
        const size_t i = order[oi];
        Ring &R = S->rings[i];
        const uint64_t rc = R.req.size();
        while (R.rissued < rt[i]) {
            const Request &r = R.req[R.rissued % rc];
            const uint64_t b = req_bytes(S, r.count);
            if (n + r.count > S->opts.max_batch ||
                (S->inflight_bytes + bytes + b > S->opts.mem_cap_bytes && (n > 0 || !idle))) {
                full = true;
                break;
            }
            const uint64_t at = R.base + r.pos % R.cap;
            if (!desc.empty() && desc.back().tree == i && desc.back().offset + desc.back().count == at)
                desc.back().count += r.count;
            else
                desc.push_back(bt_batch_desc{static_cast<uint32_t>(i), r.count, at});
            n += r.count;
            bytes += b;
            ++R.rissued;
        }
        sl.r1[i] = R.rissued;
    }
    if (n == 0) return false;
    S->known_lookups -= n;
    S->issued_bytes.fetch_add(bytes, std::memory_order_acq_rel);
    const uint32_t nd = static_cast<uint32_t>(desc.size());
    memcpy(sl.h_desc, desc.data(), sizeof(bt_batch_desc) * nd);
    btgb::forest_chunks(S->forest, sl.h_desc, nd, sl.h_cs);
    sl.seq += 1;
    const cudaError_t e = btgb::forest_run(S->forest, sl.d_desc, nd, sl.d_cs, sl.h_cs[nd], nullptr, S->d_keys,
                                           S->total_cap, S->d_vals, S->d_found, S->warps, sl.stream,
                                           btgb::ForestDone{sl.d_counter, sl.d_flag, sl.seq});
    if (e != cudaSuccess) {
        // the batch never ran: its requests are not reported done (the
        // server's status, returned by every later call, says why), and no
        // results are copied into their buffers
        btgb::set_error_detail("server issue", e);
        fail(S, BT_ERR_CUDA);
        uint64_t lost = 0;
        for (size_t i = 0; i < nt; ++i) lost += sl.r1[i] - sl.r0[i];
        std::lock_guard<std::mutex> lk(S->done_mu);
        S->failed += lost;
        return true;
    }
    sl.busy = true;
    sl.t_issue = t;
    sl.bytes = bytes;
    sl.lookups = n;
    S->inflight_bytes += bytes;
    S->fifo.push_back(static_cast<uint32_t>(&sl - S->slots.data()));
    {
        std::lock_guard<std::mutex> lk(S->done_mu);
        S->batches += 1;
        S->max_inflight_seen = std::max<uint32_t>(S->max_inflight_seen, static_cast<uint32_t>(S->fifo.size()));
    }
    return true;
}

bool all_submitted_issued(bt_server *S)
{
    for (Ring &R : S->rings)
        if (R.rissued < R.rtail.load(std::memory_order_acquire)) return false;
    return true;
}

uint64_t submitted(bt_server *S)
{
    uint64_t n = 0;
    for (Ring &R : S->rings) n += R.rtail.load(std::memory_order_acquire);
    return n;
}

// About a microsecond on the worker's own core: the worker then looks at
// the shared ring counters about once per microsecond, not continuously.
void pause_us(double us)
{
    const double end = now_us() + us;
    while (now_us() < end) {
    }
}

void worker_main(bt_server *S)
{
    cudaSetDevice(S->device);
    while (!S->stop.load(std::memory_order_acquire)) {
        const bool r = retire(S);
        const bool i = issue(S, false);
        if (!r && !i) pause_us(1.0);
    }
    // finish everything already admitted or waiting
    while (S->worker_status.load(std::memory_order_acquire) == BT_OK) {
        retire(S);
        if (all_submitted_issued(S) && S->fifo.empty()) break;
        if (!issue(S, true)) pause_us(1.0);
    }
}

void free_all(bt_server *S)
{
    for (Slot &sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.h_desc) cudaFreeHost(sl.h_desc);
        if (sl.h_cs) cudaFreeHost(sl.h_cs);
        if (sl.h_flag) cudaFreeHost(sl.h_flag);
        if (sl.d_counter) cudaFree(sl.d_counter);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (S->h_keys) cudaFreeHost(S->h_keys);
    if (S->h_vals) cudaFreeHost(S->h_vals);
    if (S->h_found) cudaFreeHost(S->h_found);
    bt_forest_free(S->forest);
}

template <typename T>
cudaError_t host_mapped(T **h, T **d, uint64_t bytes)
{
    void *p = nullptr;
    cudaError_t e = cudaHostAlloc(&p, bytes > 0 ? bytes : 16, cudaHostAllocMapped);
    if (e != cudaSuccess) return e;
    memset(p, 0, bytes > 0 ? bytes : 16);
    *h = static_cast<T *>(p);
    void *dp = nullptr;
    e = cudaHostGetDevicePointer(&dp, p, 0);
    if (e == cudaSuccess) *d = static_cast<T *>(dp);
    return e;
}

}  // namespace

extern "C" bt_status bt_server_create(const bt_tree *const *trees, const bt_model *const *models, uint32_t ntrees,
                                      const bt_server_opts *opts, bt_server **out)
{
    if (!trees || !opts || !out || ntrees == 0) return BT_ERR_ARG;
    if (opts->slots == 0 || opts->slots > 64 || opts->max_batch == 0 || opts->max_batch > (1u << 24))
        return BT_ERR_ARG;
    for (uint32_t i = 0; i < ntrees; ++i) {
        if (!trees[i] || trees[i]->dev.key_bytes == 32 || trees[i]->dev.key_bytes != trees[0]->dev.key_bytes ||
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
    cudaGetDevice(&S->device);
    bt_status st = models ? bt_forest_create_learned(trees, models, ntrees, &S->forest)
                          : bt_forest_create(trees, ntrees, &S->forest);
    if (st != BT_OK) {
        delete S;
        return st;
    }
    S->warps = btgb::forest_default_warps(S->forest);
    // every tree's ring holds the slots' batches plus two more
    const uint64_t B = opts->max_batch;
    const uint64_t cap = std::max<uint64_t>(2 * B, std::min<uint64_t>(B * (opts->slots + 2ull), 1ull << 22));
    const uint64_t rcap = std::min<uint64_t>(cap, 1ull << 20);
    S->rings = std::vector<Ring>(ntrees);
    for (uint32_t i = 0; i < ntrees; ++i) {
        S->rings[i].base = i * cap;
        S->rings[i].cap = cap;
        S->rings[i].req.resize(rcap);
    }
    S->total_cap = ntrees * cap;
    cudaError_t e = host_mapped(&S->h_keys, reinterpret_cast<unsigned char **>(&S->d_keys), S->total_cap * S->key_bytes);
    if (e == cudaSuccess)
        e = host_mapped(&S->h_vals, reinterpret_cast<unsigned char **>(&S->d_vals), S->total_cap * S->val_bytes);
    if (e == cudaSuccess) e = host_mapped(&S->h_found, &S->d_found, S->total_cap);
    const uint32_t maxd = 2 * ntrees + 2;  // a tree's run wraps at most once per batch
    S->slots.resize(opts->slots);
    S->desc_tmp.reserve(maxd);
    S->rt_tmp.assign(ntrees, 0);
    S->order_tmp.assign(ntrees, 0);
    for (Slot &sl : S->slots) {
        sl.r0.assign(ntrees, 0);
        sl.r1.assign(ntrees, 0);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = host_mapped(&sl.h_desc, &sl.d_desc, sizeof(bt_batch_desc) * maxd);
        if (e == cudaSuccess) e = host_mapped(&sl.h_cs, &sl.d_cs, sizeof(uint32_t) * (maxd + 1));
        if (e == cudaSuccess) e = host_mapped(&sl.h_flag, &sl.d_flag, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_counter, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(sl.d_counter, 0, sizeof(unsigned int));
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        btgb::set_error_detail("server buffers", e);
        free_all(S);
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
    if (!S || tree >= S->rings.size() || count == 0 || !h_keys || !h_out_vals || !h_out_found) return BT_ERR_ARG;
    if (count > S->opts.max_batch) return BT_ERR_ARG;
    const uint64_t b = req_bytes(S, count);
    // a request larger than the pending cap could never be admitted
    if (S->opts.pending_cap_bytes && b > S->opts.pending_cap_bytes) return BT_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->sub_mu);
    const int ws = S->worker_status.load(std::memory_order_acquire);
    if (ws != BT_OK) return static_cast<bt_status>(ws);
    if (S->opts.pending_cap_bytes &&
        S->sub_bytes - S->issued_bytes.load(std::memory_order_acquire) + b > S->opts.pending_cap_bytes)
        return BT_ERR_NOMEM;
    Ring &R = S->rings[tree];
    uint64_t p = R.tail;
    if (p % R.cap + count > R.cap) p += R.cap - p % R.cap;  // a request never wraps
    if (p + count - R.head.load(std::memory_order_acquire) > R.cap) return BT_ERR_NOMEM;
    const uint64_t rt = R.rtail.load(std::memory_order_relaxed);
    if (rt - R.rhead.load(std::memory_order_acquire) >= R.req.size()) return BT_ERR_NOMEM;
    memcpy(S->h_keys + (R.base + p % R.cap) * S->key_bytes, h_keys, static_cast<size_t>(count) * S->key_bytes);
    Request &r = R.req[rt % R.req.size()];
    r.count = count;
    r.pos = p;
    r.vals = h_out_vals;
    r.found = h_out_found;
    r.ticket = S->next_ticket++;
    r.t_submit = now_us();
    R.tail = p + count;
    S->sub_bytes += b;
    S->sub_lookups += count;
    if (ticket) *ticket = r.ticket;
    R.rtail.store(rt + 1, std::memory_order_release);
    return BT_OK;
}

extern "C" bt_status bt_server_poll(bt_server *S, uint64_t *tickets, uint32_t max, uint32_t *n)
{
    if (!S || !n || (max && !tickets)) return BT_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->done_mu);
    const uint32_t k = static_cast<uint32_t>(std::min<size_t>(max, S->done_tickets.size()));
    for (uint32_t i = 0; i < k; ++i) tickets[i] = S->done_tickets[i];
    S->done_tickets.erase(S->done_tickets.begin(), S->done_tickets.begin() + k);
    *n = k;
    return static_cast<bt_status>(S->worker_status.load(std::memory_order_acquire));
}

extern "C" bt_status bt_server_drain(bt_server *S, double timeout_s)
{
    if (!S) return BT_ERR_ARG;
    const double t_end = now_us() + timeout_s * 1e6;
    for (;;) {
        const int ws = S->worker_status.load(std::memory_order_acquire);
        if (ws != BT_OK) return static_cast<bt_status>(ws);
        {
            std::lock_guard<std::mutex> lk(S->done_mu);
            if (S->completed + S->failed == submitted(S) - S->reset_base) return BT_OK;
        }
        if (now_us() > t_end) return BT_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" bt_status bt_server_get_stats(bt_server *S, bt_server_stats *out, int reset)
{
    if (!S || !out) return BT_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->done_mu);
    memset(out, 0, sizeof(*out));
    out->submitted = submitted(S) - S->reset_base;
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
        S->reset_base += S->completed + S->failed;
        S->completed = 0;
        S->failed = 0;
        S->lookups = 0;
        S->batches = 0;
        S->max_inflight_seen = 0;
    }
    return static_cast<bt_status>(S->worker_status.load(std::memory_order_acquire));
}

extern "C" void bt_server_destroy(bt_server *S)
{
    if (!S) return;
    S->stop.store(true, std::memory_order_release);
    if (S->worker.joinable()) S->worker.join();
    free_all(S);
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
    double now = t0;
    for (uint64_t i = 0; i < n; ++i) {
        const double due = t0 + t_arrival_s[i] * 1e6;
        while (now < due) now = now_us();
        bt_status st;
        for (;;) {  // back-pressure: retry while the pending cap or the ring is full
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
