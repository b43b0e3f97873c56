// bt_search_batch_noalloc: the batch search for callers that cannot
// allocate device memory.  Its scratch space is one file-scope device
// array, loaded with the library and held by every GPU that loads it until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "bt_internal.h"

namespace {

// Scratch for one search of up to BT_NOALLOC_MAX_QUERIES integer queries
// (the partitioned batch, scattered and sorted, and the partition's bucket
// counters): 4 MiB.
constexpr uint64_t kNoallocScratchBytes = 4ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device.  In host code the array's name is only a host-side stand-in,
// so it must never be passed to a kernel directly.
bt_status noalloc_scratch(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        btgb::set_error_detail("cudaGetDevice", e);
        return BT_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return BT_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            btgb::set_error_detail("cudaGetSymbolAddress(no-alloc scratch)", e);
            return BT_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return BT_OK;
}

}  // namespace

extern "C" bt_status bt_search_batch_noalloc(const bt_tree *tree, const void *d_queries, uint64_t nq,
                                             void *d_out_vals, uint8_t *d_out_found, bt_stream stream)
{
    if (!tree) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    if (nq > BT_NOALLOC_MAX_QUERIES) {
        btgb::set_error_detail("bt_search_batch_noalloc: nq exceeds BT_NOALLOC_MAX_QUERIES (65536)",
                               cudaErrorInvalidValue);
        return BT_ERR_ARG;
    }
    if (bt_search_workspace_bytes(tree, nq) > kNoallocScratchBytes) {
        btgb::set_error_detail("bt_search_batch_noalloc: scratch array too small for this batch",
                               cudaErrorInvalidValue);
        return BT_ERR_WORKSPACE;
    }
    void *ws = nullptr;
    const bt_status st = noalloc_scratch(&ws);
    if (st != BT_OK) return st;
    return bt_search_batch_ex(tree, d_queries, nq, d_out_vals, d_out_found, ws, kNoallocScratchBytes,
                              nullptr, stream);
}
