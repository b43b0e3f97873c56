// Autotuner: fanout and descent launch parameters chosen by measurement.
//
// For a key set and a sample batch, every fanout in {8, 16, 32, 64} is
// built and the sample searched with every combination of warps per block
// {4, 8, 16}, shared-memory pin budget {0, 16 KB, 48 KB} and descent design
// (pipelined with inner levels through L1 or staged; synchronous with
// cp.async or bulk-copy staging; two queries per lane); the fastest
// combination (median of timed repetitions, CUDA events on the caller's
// stream) wins and its tree is returned with those settings applied.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "bt_internal.h"

namespace {

struct Scratch {
    void *ws = nullptr, *vals = nullptr, *found = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Scratch()
    {
        if (ws) cudaFree(ws);
        if (vals) cudaFree(vals);
        if (found) cudaFree(found);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Keeps the stream busy for a fixed number of clock cycles, so that the
// calls queued behind it run back to back on the device however slowly the
// host submits them.
__global__ void k_spin(long long cycles)
{
    const long long t0 = clock64();
    while (clock64() - t0 < cycles) {
    }
}

// Device time per call of the sample: kCalls calls issued behind a spin of
// about 100 us and timed together, median of kReps such runs.  (Single calls
// would time the host's submission too, and the event timer moves in steps
// of about 2 us.)
bt_status time_search(const bt_tree *t, const void *d_sample, uint64_t nq, Scratch &sc, uint64_t ws_bytes,
                      cudaStream_t s, float *us)
{
    constexpr int kCalls = 10, kReps = 5;
    constexpr long long kSpinCycles = 200000;
    const bt_stream bs = reinterpret_cast<bt_stream>(s);
    for (int i = 0; i < 2; ++i) {
        const bt_status st = bt_search_batch(t, d_sample, nq, sc.vals, static_cast<uint8_t *>(sc.found), sc.ws,
                                             ws_bytes, bs);
        if (st != BT_OK) return st;
    }
    std::vector<float> ms;
    for (int rep = 0; rep < kReps; ++rep) {
        k_spin<<<1, 32, 0, s>>>(kSpinCycles);
        if (cudaGetLastError() != cudaSuccess) return BT_ERR_CUDA;
        cudaEventRecord(sc.e0, s);
        for (int i = 0; i < kCalls; ++i) {
            const bt_status st = bt_search_batch(t, d_sample, nq, sc.vals, static_cast<uint8_t *>(sc.found), sc.ws,
                                                 ws_bytes, bs);
            if (st != BT_OK) return st;
        }
        cudaEventRecord(sc.e1, s);
        if (cudaEventSynchronize(sc.e1) != cudaSuccess) return BT_ERR_CUDA;
        float x = 0;
        cudaEventElapsedTime(&x, sc.e0, sc.e1);
        ms.push_back(x / kCalls);
    }
    std::sort(ms.begin(), ms.end());
    *us = 1000.0f * ms[ms.size() / 2];
    return BT_OK;
}

}  // namespace

extern "C" bt_status bt_autotune(const void *h_keys, const void *h_vals, uint64_t n, bt_width key_w, bt_width val_w,
                                 const void *d_sample, uint64_t nsample, bt_stream stream, bt_tree **out,
                                 bt_tune *best)
{
    if (!out || !best || !d_sample || nsample == 0 || nsample >= (1ull << 31)) return BT_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scratch sc;
    // a search's workspace for any key width: at most 44 bytes per query
    // (32-byte keys: keys, positions and pairs) plus alignment and counters
    const uint64_t ws_bytes = 64 * nsample + 1024 * 1024;
    cudaError_t e = cudaMalloc(&sc.ws, ws_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&sc.vals, nsample * 8);
    if (e == cudaSuccess) e = cudaMalloc(&sc.found, nsample);
    if (e == cudaSuccess) e = cudaEventCreate(&sc.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&sc.e1);
    if (e != cudaSuccess) {
        btgb::set_error_detail("autotune scratch", e);
        return e == cudaErrorMemoryAllocation ? BT_ERR_NOMEM : BT_ERR_CUDA;
    }
    const uint32_t fanouts[] = {8, 16, 32, 64};
    const uint32_t warps[] = {4, 8, 16};
    const uint32_t pins[] = {0, 16384, 49152};
    // The pipelined descent runs a batch with fewer 32-query chunks per SM
    // than the warps per block in blocks of that many warps (at least two):
    // a sample that small cannot choose those warps, which then keep the
    // default (8).
    int sms = 0;
    e = btgb::dev_sm_count(&sms);
    if (e != cudaSuccess) {
        btgb::set_error_detail("autotune device query", e);
        return BT_ERR_CUDA;
    }
    const uint64_t sample_per_sm = ((nsample + 31) / 32 + static_cast<uint64_t>(sms > 0 ? sms : 1) - 1) /
                                   static_cast<uint64_t>(sms > 0 ? sms : 1);
    constexpr uint32_t kDefaultWarps = 8;
    bt_tree *keep = nullptr;
    bt_tune b{0, 0, 0, 0, 1, 0, 0.0f};
    for (uint32_t m : fanouts) {
        bt_tree *t = nullptr;
        bt_status st = bt_build(h_keys, h_vals, n, key_w, val_w, m, stream, &t);
        if (st != BT_OK) {
            bt_free(keep);
            return st;
        }
        if (bt_search_workspace_bytes(t, nsample) > ws_bytes) {
            bt_free(t);
            bt_free(keep);
            return BT_ERR_ARG;
        }
        bool won = false;
        for (uint32_t w : warps)
            for (uint32_t p : pins)
                for (uint32_t cfg = 0; cfg < 5; ++cfg) {
                // (staging, queries per lane, inner levels staged): (pipelined, 1, L1),
                // (pipelined, 1, staged), (cp.async, 1), (bulk, 1), (cp.async, 2)
                static const uint32_t kStage[5] = {BT_STAGE_PIPELINED, BT_STAGE_PIPELINED, BT_STAGE_CP_ASYNC,
                                                   BT_STAGE_BULK, BT_STAGE_CP_ASYNC};
                const uint32_t sm = kStage[cfg], lq = cfg == 4 ? 2u : 1u, inner = cfg == 1 ? 1u : 0u;
                if (sm == BT_STAGE_PIPELINED && sample_per_sm < w && w != kDefaultWarps) continue;
                bt_tree_set_launch(t, w, p);
                bt_tree_set_staging(t, sm);
                bt_tree_set_lane_queries(t, lq);
                bt_tree_set_descent(t, inner, 0);
                float us = 0;
                st = time_search(t, d_sample, nsample, sc, ws_bytes, s, &us);
                if (st != BT_OK) {
                    bt_free(t);
                    bt_free(keep);
                    return st;
                }
                if (b.fanout == 0 || us < b.us_per_batch) {
                    b = bt_tune{m, w, p, sm, lq, inner, us};
                    won = true;
                }
            }
        if (won) {
            bt_free(keep);
            keep = t;
        } else {
            bt_free(t);
        }
    }
    bt_tree_set_launch(keep, b.warps_per_block, b.pin_bytes);
    bt_tree_set_staging(keep, b.staging);
    bt_tree_set_lane_queries(keep, b.lane_queries);
    bt_tree_set_descent(keep, b.inner_staged, 0);
    *out = keep;
    *best = b;
    return BT_OK;
}
