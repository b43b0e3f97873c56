// Range-partitioned search: one key set split into P subtrees over
// contiguous key ranges (the paper's kernel instances share one batch,
// Sec. IV-G; split by key range, each instance needs only its part of the
// tree -- across GPUs, one part per GPU, with queries routed to the part
// whose range holds them and results routed back).  On one device:
//
//   k_route_count    per block, the part counts of a slice of the batch
//                    (part = the number of splitters below the query, the
//                    splitters being every part's largest key but the
//                    last's), added to the totals with one atomic per part
//                    whose return value is the block's offset in that part;
//   (host)           the P totals are read back (the one synchronisation of
//                    a call: every part's search needs its size);
//   k_route_scatter  the same slices: each query goes to its part's next
//                    position with its input position;
//   per part         bt_search_batch on the part's contiguous sub-batch;
//   k_unroute        every result back to its input position.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "bt_internal.h"

namespace {

constexpr uint32_t kMaxParts = 64;
constexpr int kRouteThreads = 256;
constexpr uint64_t kRoutePerBlock = 4096;
constexpr uint64_t kRouteMaxBlocks = 1024;

static inline uint64_t a256(uint64_t x) { return (x + 255) & ~255ull; }

template <typename K>
__device__ __forceinline__ uint32_t route_part(const K *sp, uint32_t ns, K q)
{
    uint32_t lo = 0, hi = ns;  // first splitter >= q
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (sp[mid] < q)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

template <typename K>
__global__ void __launch_bounds__(kRouteThreads) k_route_count(const K *__restrict__ q, uint64_t nq,
                                                               const K *__restrict__ split, uint32_t parts,
                                                               unsigned int *__restrict__ total,
                                                               uint32_t *__restrict__ blkoff)
{
    __shared__ K sp[kMaxParts];
    __shared__ unsigned int cnt[kMaxParts];
    for (uint32_t j = threadIdx.x; j < parts; j += blockDim.x) {
        if (j + 1 < parts) sp[j] = split[j];
        cnt[j] = 0;
    }
    __syncthreads();
    const uint64_t per = (nq + gridDim.x - 1) / gridDim.x;
    const uint64_t s0 = blockIdx.x * per < nq ? blockIdx.x * per : nq;
    const uint64_t s1 = s0 + per < nq ? s0 + per : nq;
    for (uint64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) atomicAdd(cnt + route_part(sp, parts - 1, q[i]), 1u);
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < parts; j += blockDim.x)
        blkoff[static_cast<uint64_t>(blockIdx.x) * parts + j] = cnt[j] ? atomicAdd(total + j, cnt[j]) : 0u;
}

template <typename K>
__global__ void __launch_bounds__(kRouteThreads) k_route_scatter(const K *__restrict__ q, uint64_t nq,
                                                                 const K *__restrict__ split, uint32_t parts,
                                                                 const unsigned int *__restrict__ total,
                                                                 const uint32_t *__restrict__ blkoff,
                                                                 K *__restrict__ rq, uint32_t *__restrict__ ridx)
{
    __shared__ K sp[kMaxParts];
    __shared__ unsigned int base[kMaxParts];
    if (threadIdx.x == 0) {
        unsigned int run = 0;
        for (uint32_t j = 0; j < parts; ++j) {
            base[j] = run + blkoff[static_cast<uint64_t>(blockIdx.x) * parts + j];
            run += total[j];
        }
    }
    for (uint32_t j = threadIdx.x; j + 1 < parts; j += blockDim.x) sp[j] = split[j];
    __syncthreads();
    const uint64_t per = (nq + gridDim.x - 1) / gridDim.x;
    const uint64_t s0 = blockIdx.x * per < nq ? blockIdx.x * per : nq;
    const uint64_t s1 = s0 + per < nq ? s0 + per : nq;
    for (uint64_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
        const K key = q[i];
        const unsigned int pos = atomicAdd(base + route_part(sp, parts - 1, key), 1u);
        if (pos < nq) {  // always true when the counts agree; keeps a stray write in bounds
            rq[pos] = key;
            ridx[pos] = static_cast<uint32_t>(i);
        }
    }
}

template <typename V>
__global__ void k_unroute(const V *__restrict__ rv, const uint8_t *__restrict__ rf, const uint32_t *__restrict__ ridx,
                          uint64_t nq, V *__restrict__ out_v, uint8_t *__restrict__ out_f)
{
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < nq;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t d = ridx[i];
        if (d < nq) {
            out_v[d] = rv[i];
            out_f[d] = rf[i];
        }
    }
}

struct RangeWs {
    uint64_t rq, ridx, rv, rf, total, blkoff, search, bytes;
};

}  // namespace

struct bt_range {
    uint32_t parts;
    int key_bytes, val_bytes;
    uint64_t n;
    bt_tree *tree[kMaxParts];
    uint64_t h_split[kMaxParts];  // splitter j: the largest key of part j (j < parts - 1)
    void *d_split;                // the same, key width
    unsigned int *h_counts;       // page-locked, parts words
};

namespace {

RangeWs range_ws(const bt_range *r, uint64_t nq)
{
    RangeWs w;
    uint64_t o = 0;
    w.rq = o;
    o = a256(o + nq * r->key_bytes);
    w.ridx = o;
    o = a256(o + nq * 4);
    w.rv = o;
    o = a256(o + nq * r->val_bytes);
    w.rf = o;
    o = a256(o + nq);
    w.total = o;
    o = a256(o + kMaxParts * 4);
    w.blkoff = o;
    const uint64_t g = (nq + kRoutePerBlock - 1) / kRoutePerBlock;
    o = a256(o + (g < kRouteMaxBlocks ? g : kRouteMaxBlocks) * kMaxParts * 4);
    w.search = o;
    o += bt_search_workspace_bytes(r->tree[0], nq);
    w.bytes = nq ? o : 0;
    return w;
}

template <typename K>
cudaError_t route(const bt_range *r, const void *q, uint64_t nq, unsigned char *ws, const RangeWs &w,
                  cudaStream_t s)
{
    uint64_t g = (nq + kRoutePerBlock - 1) / kRoutePerBlock;
    if (g > kRouteMaxBlocks) g = kRouteMaxBlocks;
    unsigned int *total = reinterpret_cast<unsigned int *>(ws + w.total);
    uint32_t *blkoff = reinterpret_cast<uint32_t *>(ws + w.blkoff);
    cudaError_t e = cudaMemsetAsync(total, 0, kMaxParts * 4, s);
    if (e != cudaSuccess) return e;
    k_route_count<K><<<static_cast<unsigned>(g), kRouteThreads, 0, s>>>(
        static_cast<const K *>(q), nq, static_cast<const K *>(r->d_split), r->parts, total, blkoff);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->h_counts, total, r->parts * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    k_route_scatter<K><<<static_cast<unsigned>(g), kRouteThreads, 0, s>>>(
        static_cast<const K *>(q), nq, static_cast<const K *>(r->d_split), r->parts, total, blkoff,
        reinterpret_cast<K *>(ws + w.rq), reinterpret_cast<uint32_t *>(ws + w.ridx));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the part sizes, for the searches
    return e;
}

}  // namespace

using namespace btgb;

extern "C" bt_status bt_range_build(const void *h_keys, const void *h_vals, uint64_t n, bt_width key_w,
                                    bt_width val_w, uint32_t fanout, uint32_t parts, bt_stream stream,
                                    bt_range **out)
{
    if (!out || parts == 0 || parts > kMaxParts || n < parts || !h_keys || !h_vals) return BT_ERR_ARG;
    if (key_w != BT_U32 && key_w != BT_U64) return BT_ERR_ARG;
    if (val_w != BT_U32 && val_w != BT_U64) return BT_ERR_ARG;
    bt_range *r = new (std::nothrow) bt_range;
    if (!r) return BT_ERR_NOMEM;
    memset(r, 0, sizeof(*r));
    r->parts = parts;
    r->key_bytes = static_cast<int>(key_w);
    r->val_bytes = static_cast<int>(val_w);
    r->n = n;
    const unsigned char *kb = static_cast<const unsigned char *>(h_keys);
    const unsigned char *vb = static_cast<const unsigned char *>(h_vals);
    bt_status st = BT_OK;
    for (uint32_t p = 0; p < parts && st == BT_OK; ++p) {
        const uint64_t lo = p * n / parts, hi = (p + 1) * n / parts;  // ranks [lo, hi)
        st = bt_build(kb + lo * key_w, vb + lo * val_w, hi - lo, key_w, val_w, fanout, stream, &r->tree[p]);
        if (st == BT_OK && p + 1 < parts) {
            uint64_t k = 0;
            memcpy(&k, kb + (hi - 1) * key_w, key_w);
            r->h_split[p] = k;
        }
    }
    // the parts' ranges must be ordered: bt_build checked each part's keys,
    // the splitters check the boundaries between parts
    for (uint32_t p = 0; p + 1 < parts && st == BT_OK; ++p) {
        uint64_t first = 0;
        memcpy(&first, kb + ((p + 1) * n / parts) * key_w, key_w);
        if (first < r->h_split[p]) st = BT_ERR_UNSORTED;
        else if (first == r->h_split[p]) st = BT_ERR_DUPLICATE;
    }
    if (st == BT_OK) {
        cudaError_t e = cudaMalloc(&r->d_split, kMaxParts * 8);
        if (e == cudaSuccess) {
            if (key_w == BT_U64) {
                e = cudaMemcpy(r->d_split, r->h_split, (parts - 1) * 8ull, cudaMemcpyHostToDevice);
            } else {
                uint32_t s32[kMaxParts];
                for (uint32_t p = 0; p + 1 < parts; ++p) s32[p] = static_cast<uint32_t>(r->h_split[p]);
                e = cudaMemcpy(r->d_split, s32, (parts - 1) * 4ull, cudaMemcpyHostToDevice);
            }
        }
        if (e == cudaSuccess) e = cudaMallocHost(&r->h_counts, kMaxParts * 4);
        if (e != cudaSuccess) {
            set_error_detail("range splitters", e);
            st = e == cudaErrorMemoryAllocation ? BT_ERR_NOMEM : BT_ERR_CUDA;
        }
    }
    if (st != BT_OK) {
        bt_range_free(r);
        return st;
    }
    *out = r;
    return BT_OK;
}

extern "C" void bt_range_free(bt_range *r)
{
    if (!r) return;
    for (uint32_t p = 0; p < r->parts; ++p) bt_free(r->tree[p]);
    if (r->d_split) cudaFree(r->d_split);
    if (r->h_counts) cudaFreeHost(r->h_counts);
    delete r;
}

extern "C" bt_status bt_range_info(const bt_range *r, uint32_t *parts, uint64_t *h_splitters, uint64_t *h_part_keys)
{
    if (!r || !parts) return BT_ERR_ARG;
    *parts = r->parts;
    for (uint32_t p = 0; p < r->parts; ++p) {
        if (h_splitters && p + 1 < r->parts) h_splitters[p] = r->h_split[p];
        if (h_part_keys) h_part_keys[p] = (p + 1) * r->n / r->parts - p * r->n / r->parts;
    }
    return BT_OK;
}

extern "C" const bt_tree *bt_range_part(const bt_range *r, uint32_t p)
{
    return (r && p < r->parts) ? r->tree[p] : nullptr;
}

extern "C" uint64_t bt_range_workspace_bytes(const bt_range *r, uint64_t nq)
{
    if (!r) return 0;
    return range_ws(r, nq).bytes;
}

extern "C" bt_status bt_range_search(const bt_range *r, const void *d_queries, uint64_t nq, void *d_out_vals,
                                     uint8_t *d_out_found, void *d_workspace, uint64_t ws_bytes, bt_stream stream)
{
    if (!r) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    if (nq >= (1ull << 31) || !d_queries || !d_out_vals || !d_out_found) return BT_ERR_ARG;
    // queries and values aligned to their element sizes
    if ((reinterpret_cast<uintptr_t>(d_queries) & static_cast<uintptr_t>(r->key_bytes - 1)) ||
        (reinterpret_cast<uintptr_t>(d_out_vals) & static_cast<uintptr_t>(r->val_bytes - 1)))
        return BT_ERR_ARG;
    const RangeWs w = range_ws(r, nq);
    if (!d_workspace || ws_bytes < w.bytes || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return BT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(d_workspace);
    cudaError_t e = r->key_bytes == 8 ? route<uint64_t>(r, d_queries, nq, ws, w, s)
                                      : route<uint32_t>(r, d_queries, nq, ws, w, s);
    if (e != cudaSuccess) {
        set_error_detail("range routing", e);
        return BT_ERR_CUDA;
    }
    // every part's sub-batch through the single-tree search, in turn
    uint64_t start = 0;
    const uint64_t sws = ws_bytes - w.search;
    for (uint32_t p = 0; p < r->parts; ++p) {
        const uint64_t c = r->h_counts[p];
        if (c) {
            const bt_status st = bt_search_batch(
                r->tree[p], ws + w.rq + start * r->key_bytes, c, ws + w.rv + start * r->val_bytes, ws + w.rf + start,
                ws + w.search, sws, stream);
            if (st != BT_OK) return st;
        }
        start += c;
    }
    const unsigned grid = static_cast<unsigned>((nq + 255) / 256 < 4096 ? (nq + 255) / 256 : 4096);
    if (r->val_bytes == 8)
        k_unroute<uint64_t><<<grid, 256, 0, s>>>(reinterpret_cast<const uint64_t *>(ws + w.rv), ws + w.rf,
                                                 reinterpret_cast<const uint32_t *>(ws + w.ridx), nq,
                                                 static_cast<uint64_t *>(d_out_vals), d_out_found);
    else
        k_unroute<uint32_t><<<grid, 256, 0, s>>>(reinterpret_cast<const uint32_t *>(ws + w.rv), ws + w.rf,
                                                 reinterpret_cast<const uint32_t *>(ws + w.ridx), nq,
                                                 static_cast<uint32_t *>(d_out_vals), d_out_found);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error_detail("range unroute", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}
