// Batched level-wise B+ tree point search on GB300 (sm_103a).
//
// One search is (Sec. IV-A, IV-F):
//   1. an on-device LSD radix sort of (query, input position) pairs on the
//      leading bits of the normalised query key, so that queries routed to the
//      same node end up adjacent (the paper's sorted batch);
//   2. the level-wise descent: each warp takes 32 consecutive queries of the
//      sorted batch and walks them down the tree together; at every level it
//      finds the distinct nodes its queries need (warp match/ballot/popc, the
//      paper's (address, count) FIFO entries), stages each distinct node's
//      key block into shared memory once with 16-byte asynchronous copies,
//      and every query then finds its child rank -- the number of separators
//      smaller than the query, i.e. the first separator it is <= to
//      (Sec. IV-E's priority encoder) -- by a branchless binary search in
//      shared memory;
//   3. the leaf probe (Sec. IV-D): the same rank in the leaf block is the
//      only slot that can hold an equal key; a hit reads the value, a miss
//      returns all-ones (the paper's -1) with found = 0;
//   4. the scatter of each result back to the query's input position.
// Everything is integer compares; nothing here is a dense contraction, so
// no tensor-core path is used.
#include <cuda_runtime.h>

#include <cstdint>

#include "bt_internal.h"

namespace btgb {

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ void cp_async16_ca(void *smem_dst, const void *gsrc)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async16_cg(void *smem_dst, const void *gsrc)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Normalised sort field of a query: its offset above the smallest key,
// clamped to the key range, shifted right so `bits` leading bits remain.
// Monotone in the query, so sorting by it is a partial sort by key.
struct SortNorm {
    uint64_t kmin;
    uint64_t range;
    int shift;
    int passes;
};

template <typename K>
__device__ __forceinline__ uint32_t sort_digit(K q, const SortNorm &s, int pass)
{
    const uint64_t x = static_cast<uint64_t>(q);
    uint64_t nk = (x <= s.kmin) ? 0 : x - s.kmin;
    if (nk > s.range) nk = s.range;
    return static_cast<uint32_t>((nk >> (s.shift + 8 * pass)) & 0xFFu);
}

// ------------------------------------------------------- radix sort (a2)
//
// Classic stable LSD radix sort with 8-bit digits in three kernels: per-tile
// histograms of every pass's digit (one read of the queries), a scan of each
// pass's (digit, tile) count matrix in digit-major order, and one stable
// scatter per pass.

constexpr int kSortTile = 4096;
constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortPerWarp = kSortTile / kSortWarps;  // 256 = 8 rounds of 32
constexpr int kMaxPasses = 8;

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const K *__restrict__ q, uint64_t nq,
                                                             SortNorm sn, uint32_t *__restrict__ counts,
                                                             uint32_t ntiles)
{
    __shared__ uint32_t h[kMaxPasses * 256];
    for (int i = threadIdx.x; i < sn.passes * 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kSortTile;
    for (int e = threadIdx.x; e < kSortTile; e += blockDim.x) {
        const uint64_t pos = base + e;
        const bool valid = pos < nq;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (valid) {
            const K key = q[pos];
            for (int p = 0; p < sn.passes; ++p) {
                const uint32_t d = sort_digit(key, sn, p);
                const unsigned same = __match_any_sync(vm, d);
                if ((same & lanemask_lt()) == 0) atomicAdd(&h[p * 256 + d], __popc(same));
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < sn.passes * 256; i += blockDim.x)
        counts[static_cast<uint64_t>(i) * ntiles + blockIdx.x] = h[i];
}

// Exclusive scan of one pass's [256][ntiles] count matrix (one CTA per pass).
__global__ void __launch_bounds__(1024) k_radix_scan(uint32_t *__restrict__ counts, uint32_t ntiles)
{
    __shared__ uint32_t warp_tot[32];
    uint32_t *c = counts + static_cast<uint64_t>(blockIdx.x) * 256u * ntiles;
    const uint64_t total = 256ull * ntiles;
    const uint64_t per = (total + blockDim.x - 1) / blockDim.x;
    const uint64_t lo = threadIdx.x * per;
    const uint64_t hi = lo + per < total ? lo + per : total;
    uint32_t sum = 0;
    for (uint64_t i = lo; i < hi; ++i) sum += c[i];
    // block-wide exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < (blockDim.x >> 5)) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;  // inclusive
    }
    __syncthreads();
    uint32_t run = x - sum + (warp > 0 ? warp_tot[warp - 1] : 0);
    for (uint64_t i = lo; i < hi; ++i) {
        const uint32_t v = c[i];
        c[i] = run;
        run += v;
    }
}

// Stable scatter of one pass.  Warp w of tile t owns tile elements
// [w*256, (w+1)*256) and ranks them in order, 32 at a time, against
// warp-private digit counters; a per-digit scan over the warps and the
// tile's global digit offsets then give every element its output slot.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const K *__restrict__ qin, const uint32_t *__restrict__ iin, K *__restrict__ qout,
    uint32_t *__restrict__ iout, uint64_t nq, SortNorm sn, int pass,
    const uint32_t *__restrict__ offs, uint32_t ntiles)
{
    __shared__ uint32_t wh[kSortWarps][256];
    __shared__ uint32_t toff[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * 256; i += blockDim.x) (&wh[0][0])[i] = 0;
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        toff[i] = offs[static_cast<uint64_t>(i) * ntiles + blockIdx.x];
    __syncthreads();

    constexpr int R = kSortPerWarp / 32;
    K key[R];
    uint32_t idx[R], dig[R], rank[R];
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kSortTile + warp * kSortPerWarp;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t pos = base + r * 32 + lane;
        const bool valid = pos < nq;
        if (valid) {
            key[r] = qin[pos];
            idx[r] = iin ? iin[pos] : static_cast<uint32_t>(pos);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t pos = base + r * 32 + lane;
        const bool valid = pos < nq;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        unsigned same = 0;
        if (valid) {
            dig[r] = sort_digit(key[r], sn, pass);
            same = __match_any_sync(vm, dig[r]);
            rank[r] = wh[warp][dig[r]] + __popc(same & lanemask_lt());
        }
        __syncwarp();
        if (valid && (same & lanemask_lt()) == 0) wh[warp][dig[r]] += __popc(same);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t v = wh[w][d];
            wh[w][d] = run;
            run += v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t pos = base + r * 32 + lane;
        if (pos < nq) {
            const uint32_t o = toff[dig[r]] + wh[warp][dig[r]] + rank[r];
            qout[o] = key[r];
            iout[o] = idx[r];
        }
    }
}

// -------------------------------------------- level-wise descent (a3-a5)

constexpr int kDescWarps = 4;

template <typename K, int M>
constexpr int desc_smem_bytes()
{
    return kDescWarps * (32 * M * static_cast<int>(sizeof(K)) + 32 * 4);
}

template <typename K, typename V, int M, bool COUNT>
__global__ void __launch_bounds__(kDescWarps * 32) k_descend(
    const DevTree t, const K *__restrict__ q, const uint32_t *__restrict__ qidx, uint64_t nq,
    V *__restrict__ out_v, uint8_t *__restrict__ out_f, unsigned long long *__restrict__ fetch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int CH = M * static_cast<int>(sizeof(K)) / 16;  // 16-byte chunks per node block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    K *stage = reinterpret_cast<K *>(smem) + warp * 32 * M;
    uint32_t *list = reinterpret_cast<uint32_t *>(smem + kDescWarps * 32 * M * sizeof(K)) + warp * 32;
    const uint64_t nchunks = (nq + 31) / 32;
    const int H = t.height;

    for (uint64_t c = static_cast<uint64_t>(blockIdx.x) * kDescWarps + warp; c < nchunks;
         c += static_cast<uint64_t>(gridDim.x) * kDescWarps) {
        const uint64_t pos = c * 32 + lane;
        const bool valid = pos < nq;
        // Tail lanes follow lane 0's query so they never add a node fetch.
        const K key = q[valid ? pos : c * 32];
        const uint32_t dst = valid ? (qidx ? qidx[pos] : static_cast<uint32_t>(pos)) : 0u;
        uint32_t node = 0;

        for (int l = 0; l < H; ++l) {
            const K *lk = static_cast<const K *>(t.keys[l]);
            // Distinct nodes among the warp's queries: one leader per node.
            const unsigned same = __match_any_sync(0xffffffffu, node);
            const int leader = __ffs(same) - 1;
            const unsigned leaders = __ballot_sync(0xffffffffu, lane == leader);
            const int U = __popc(leaders);
            const int slot = __popc(leaders & ((1u << leader) - 1u));
            if (lane == leader) list[slot] = node;
            if (COUNT && lane == 0) atomicAdd(fetch + l, static_cast<unsigned long long>(U));
            __syncwarp();
            // Stage each distinct node's key block once.
            const bool last = (l + 1 == H);
            for (int i = lane; i < U * CH; i += 32) {
                const int u = i / CH, part = i - u * CH;
                const unsigned char *src = reinterpret_cast<const unsigned char *>(
                                               lk + static_cast<uint64_t>(list[u]) * M) + part * 16;
                unsigned char *dstp = reinterpret_cast<unsigned char *>(stage + u * M) + part * 16;
                if (last)
                    cp_async16_cg(dstp, src);
                else
                    cp_async16_ca(dstp, src);
            }
            cp_async_wait_all();
            __syncwarp();
            // Child rank = number of slots holding a key < query.  Slot M-1
            // is always padding (all-ones), so log2(M) probes suffice.
            const K *blk = stage + slot * M;
            int r = 0;
#pragma unroll
            for (int hlf = M / 2; hlf >= 1; hlf >>= 1)
                if (blk[r + hlf - 1] < key) r += hlf;
            if (!last) {
                const uint64_t base = t.cbase[l], rem = t.crem[l];
                node = static_cast<uint32_t>(node * base + (node < rem ? node : rem) + r);
            } else {
                const uint64_t cnt = t.cbase[l] + (node < t.crem[l] ? 1u : 0u);
                const bool hit = (static_cast<uint64_t>(r) < cnt) && (blk[r] == key);
                V val = static_cast<V>(~static_cast<V>(0));
                if (hit) val = static_cast<const V *>(t.vals)[static_cast<uint64_t>(node) * M + r];
                if (valid) {
                    out_v[dst] = val;
                    out_f[dst] = hit ? 1 : 0;
                }
            }
            __syncwarp();
        }
    }
}

template <typename V>
__global__ void k_fill_miss(V *__restrict__ out_v, uint8_t *__restrict__ out_f, uint64_t nq)
{
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < nq;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        out_v[i] = static_cast<V>(~static_cast<V>(0));
        out_f[i] = 0;
    }
}

// ------------------------------------------------------------ host side

static inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

static inline uint32_t sort_tiles(uint64_t nq) { return static_cast<uint32_t>((nq + kSortTile - 1) / kSortTile); }

struct WsLayout {
    uint64_t qa, ia, qb, ib, counts, total;
};

static WsLayout ws_layout(int kb, uint64_t nq)
{
    WsLayout w;
    uint64_t o = 0;
    w.qa = o;
    o = align256(o + nq * kb);
    w.ia = o;
    o = align256(o + nq * 4);
    w.qb = o;
    o = align256(o + nq * kb);
    w.ib = o;
    o = align256(o + nq * 4);
    w.counts = o;
    o = align256(o + static_cast<uint64_t>(kMaxPasses) * 256u * sort_tiles(nq) * 4u);
    w.total = nq ? o : 0;
    return w;
}

static int bitlen(uint64_t x) { return x ? 64 - __builtin_clzll(x) : 0; }

// Queries per batch from which the sort pays for itself by node reuse.
constexpr uint64_t kAutoSortMinBatch = 16384;
constexpr int kAutoSortBits = 16;

template <typename K, typename V, int M, bool COUNT>
static cudaError_t launch_descend(const DevTree &t, const void *q, const uint32_t *qidx, uint64_t nq,
                                  void *out_v, uint8_t *out_f, unsigned long long *fetch,
                                  cudaStream_t s)
{
    constexpr int smem = desc_smem_bytes<K, M>();
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_descend<K, V, M, COUNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    const uint64_t chunks = (nq + 31) / 32;
    uint64_t grid = (chunks + kDescWarps - 1) / kDescWarps;
    if (grid > (1u << 30)) grid = 1u << 30;
    k_descend<K, V, M, COUNT><<<static_cast<unsigned>(grid), kDescWarps * 32, smem, s>>>(
        t, static_cast<const K *>(q), qidx, nq, static_cast<V *>(out_v), out_f, fetch);
    return cudaGetLastError();
}

template <typename K, typename V, int M>
static cudaError_t dispatch_count(const DevTree &t, const void *q, const uint32_t *qidx, uint64_t nq,
                                  void *out_v, uint8_t *out_f, unsigned long long *fetch,
                                  cudaStream_t s)
{
    if (fetch) return launch_descend<K, V, M, true>(t, q, qidx, nq, out_v, out_f, fetch, s);
    return launch_descend<K, V, M, false>(t, q, qidx, nq, out_v, out_f, nullptr, s);
}

template <typename K, typename V>
static cudaError_t dispatch_m(const DevTree &t, const void *q, const uint32_t *qidx, uint64_t nq,
                              void *out_v, uint8_t *out_f, unsigned long long *fetch, cudaStream_t s)
{
    switch (t.m) {
    case 8: return dispatch_count<K, V, 8>(t, q, qidx, nq, out_v, out_f, fetch, s);
    case 16: return dispatch_count<K, V, 16>(t, q, qidx, nq, out_v, out_f, fetch, s);
    case 32: return dispatch_count<K, V, 32>(t, q, qidx, nq, out_v, out_f, fetch, s);
    default: return dispatch_count<K, V, 64>(t, q, qidx, nq, out_v, out_f, fetch, s);
    }
}

static cudaError_t descend(const DevTree &t, const void *q, const uint32_t *qidx, uint64_t nq,
                           void *out_v, uint8_t *out_f, unsigned long long *fetch, cudaStream_t s)
{
    if (t.key_bytes == 8) {
        if (t.val_bytes == 8) return dispatch_m<uint64_t, uint64_t>(t, q, qidx, nq, out_v, out_f, fetch, s);
        return dispatch_m<uint64_t, uint32_t>(t, q, qidx, nq, out_v, out_f, fetch, s);
    }
    if (t.val_bytes == 8) return dispatch_m<uint32_t, uint64_t>(t, q, qidx, nq, out_v, out_f, fetch, s);
    return dispatch_m<uint32_t, uint32_t>(t, q, qidx, nq, out_v, out_f, fetch, s);
}

template <typename K>
__global__ void k_copy_identity(const K *__restrict__ q, K *__restrict__ qo, uint32_t *__restrict__ io,
                                uint64_t nq)
{
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < nq;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        qo[i] = q[i];
        io[i] = static_cast<uint32_t>(i);
    }
}

// Sort (query, position) pairs: passes before the last ping-pong between the
// workspace buffers A and B (A first), the last pass writes (dst_q, dst_i).
template <typename K>
static cudaError_t radix_sort(const K *q, uint64_t nq, const SortNorm &sn, unsigned char *ws,
                              const WsLayout &w, K *dst_q, uint32_t *dst_i, cudaStream_t s)
{
    const uint32_t ntiles = sort_tiles(nq);
    uint32_t *counts = reinterpret_cast<uint32_t *>(ws + w.counts);
    k_radix_hist<K><<<ntiles, kSortThreads, 0, s>>>(q, nq, sn, counts, ntiles);
    k_radix_scan<<<sn.passes, 1024, 0, s>>>(counts, ntiles);
    K *qa = reinterpret_cast<K *>(ws + w.qa), *qb = reinterpret_cast<K *>(ws + w.qb);
    uint32_t *ia = reinterpret_cast<uint32_t *>(ws + w.ia), *ib = reinterpret_cast<uint32_t *>(ws + w.ib);
    const K *src_q = q;
    const uint32_t *src_i = nullptr;
    for (int p = 0; p < sn.passes; ++p) {
        const bool final_pass = (p + 1 == sn.passes);
        K *dq = final_pass ? dst_q : ((p & 1) ? qb : qa);
        uint32_t *di = final_pass ? dst_i : ((p & 1) ? ib : ia);
        k_radix_scatter<K><<<ntiles, kSortThreads, 0, s>>>(
            src_q, src_i, dq, di, nq, sn, p, counts + static_cast<uint64_t>(p) * 256u * ntiles, ntiles);
        src_q = dq;
        src_i = di;
    }
    return cudaGetLastError();
}

// Where bt_search_batch puts the sorted batch: whichever of A/B the last
// intermediate pass did not write.
static void internal_sort_dst(const SortNorm &sn, unsigned char *ws, const WsLayout &w, void **dq,
                              uint32_t **di)
{
    const bool use_b = sn.passes >= 2 && ((sn.passes - 2) % 2 == 0);
    *dq = ws + (use_b ? w.qb : w.qa);
    *di = reinterpret_cast<uint32_t *>(ws + (use_b ? w.ib : w.ia));
}

static cudaError_t sort_any(const DevTree &t, const void *q, uint64_t nq, const SortNorm &sn,
                            unsigned char *ws, const WsLayout &w, void *dq, uint32_t *di,
                            cudaStream_t s)
{
    if (t.key_bytes == 8)
        return radix_sort<uint64_t>(static_cast<const uint64_t *>(q), nq, sn, ws, w,
                                    static_cast<uint64_t *>(dq), di, s);
    return radix_sort<uint32_t>(static_cast<const uint32_t *>(q), nq, sn, ws, w,
                                static_cast<uint32_t *>(dq), di, s);
}

static SortNorm make_norm(const DevTree &t, int32_t sort_bits, uint64_t nq)
{
    SortNorm sn{t.kmin, t.kmax - t.kmin, 0, 0};
    int bits = sort_bits;
    if (bits < 0) bits = (nq >= kAutoSortMinBatch) ? kAutoSortBits : 0;
    const int rl = bitlen(sn.range);
    if (bits > rl) bits = rl;
    if (bits > 8 * t.key_bytes) bits = 8 * t.key_bytes;
    if (bits <= 0) return sn;
    sn.passes = (bits + 7) / 8;
    const int used = 8 * sn.passes;
    sn.shift = rl > used ? rl - used : 0;
    return sn;
}

}  // namespace btgb

using namespace btgb;

extern "C" int32_t bt_sort_passes(const bt_tree *tree, uint64_t nq, int32_t sort_bits)
{
    if (!tree) return -1;
    if (tree->dev.height == 0 || nq == 0) return 0;
    return make_norm(tree->dev, sort_bits, nq).passes;
}

extern "C" uint64_t bt_search_workspace_bytes(const bt_tree *tree, uint64_t nq)
{
    if (!tree) return 0;
    return ws_layout(tree->dev.key_bytes, nq).total;
}

extern "C" uint64_t bt_search_host_workspace_bytes(const bt_tree *tree, uint64_t nq)
{
    if (!tree) return 0;
    const uint64_t io = align256(nq * tree->dev.key_bytes) + align256(nq * tree->dev.val_bytes) + align256(nq);
    return io + bt_search_workspace_bytes(tree, nq);
}

extern "C" bt_status bt_search_batch_ex(const bt_tree *tree, const void *d_queries, uint64_t nq,
                                        void *d_out_vals, uint8_t *d_out_found, void *d_workspace,
                                        uint64_t ws_bytes, const bt_search_opts *opts,
                                        bt_stream stream)
{
    if (!tree) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    if (nq >= (1ull << 31)) return BT_ERR_ARG;
    if (!d_queries || !d_out_vals || !d_out_found) return BT_ERR_ARG;
    const DevTree &t = tree->dev;
    const WsLayout w = ws_layout(t.key_bytes, nq);
    if (!d_workspace || ws_bytes < w.total || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return BT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;

    if (t.height == 0) {
        const unsigned grid = static_cast<unsigned>((nq + 255) / 256 < 4096 ? (nq + 255) / 256 : 4096);
        if (t.val_bytes == 8)
            k_fill_miss<uint64_t><<<grid, 256, 0, s>>>(static_cast<uint64_t *>(d_out_vals), d_out_found, nq);
        else
            k_fill_miss<uint32_t><<<grid, 256, 0, s>>>(static_cast<uint32_t *>(d_out_vals), d_out_found, nq);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error_detail("fill-miss launch", e);
            return BT_ERR_CUDA;
        }
        return BT_OK;
    }

    const SortNorm sn = make_norm(t, opts ? opts->sort_bits : -1, nq);
    const void *q = d_queries;
    const uint32_t *qidx = nullptr;
    unsigned char *ws = static_cast<unsigned char *>(d_workspace);
    if (sn.passes > 0) {
        void *dq;
        uint32_t *di;
        internal_sort_dst(sn, ws, w, &dq, &di);
        e = sort_any(t, d_queries, nq, sn, ws, w, dq, di, s);
        if (e != cudaSuccess) {
            set_error_detail("radix sort launch", e);
            return BT_ERR_CUDA;
        }
        q = dq;
        qidx = di;
    }
    e = descend(t, q, qidx, nq, d_out_vals, d_out_found, opts ? opts->d_fetch_counts : nullptr, s);
    if (e != cudaSuccess) {
        set_error_detail("descent launch", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}

extern "C" bt_status bt_search_batch(const bt_tree *tree, const void *d_queries, uint64_t nq,
                                     void *d_out_vals, uint8_t *d_out_found, void *d_workspace,
                                     uint64_t ws_bytes, bt_stream stream)
{
    return bt_search_batch_ex(tree, d_queries, nq, d_out_vals, d_out_found, d_workspace, ws_bytes,
                              nullptr, stream);
}

extern "C" bt_status bt_search_batch_host(const bt_tree *tree, const void *h_queries, uint64_t nq,
                                          void *h_out_vals, uint8_t *h_out_found, void *d_workspace,
                                          uint64_t ws_bytes, bt_stream stream)
{
    if (!tree) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    if (nq >= (1ull << 31)) return BT_ERR_ARG;
    if (!h_queries || !h_out_vals || !h_out_found) return BT_ERR_ARG;
    const uint64_t need = bt_search_host_workspace_bytes(tree, nq);
    if (!d_workspace || ws_bytes < need || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return BT_ERR_WORKSPACE;
    const int kb = tree->dev.key_bytes, vb = tree->dev.val_bytes;
    unsigned char *base = static_cast<unsigned char *>(d_workspace);
    unsigned char *dq = base;
    unsigned char *dv = dq + align256(nq * kb);
    unsigned char *df = dv + align256(nq * vb);
    unsigned char *ws = df + align256(nq);
    const uint64_t ws_rest = need - static_cast<uint64_t>(ws - base);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(dq, h_queries, nq * kb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        set_error_detail("query copy to device", e);
        return BT_ERR_CUDA;
    }
    bt_status st = bt_search_batch_ex(tree, dq, nq, dv, df, ws, ws_rest, nullptr, stream);
    if (st != BT_OK) return st;
    e = cudaMemcpyAsync(h_out_vals, dv, nq * vb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_out_found, df, nq, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) {
        set_error_detail("result copy to host", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}

extern "C" bt_status bt_sort_batch(const bt_tree *tree, const void *d_queries, uint64_t nq,
                                   int32_t sort_bits, void *d_sorted_queries, uint32_t *d_sorted_index,
                                   void *d_workspace, uint64_t ws_bytes, bt_stream stream)
{
    if (!tree) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    if (nq >= (1ull << 31)) return BT_ERR_ARG;
    if (!d_queries || !d_sorted_queries || !d_sorted_index) return BT_ERR_ARG;
    const DevTree &t = tree->dev;
    const WsLayout w = ws_layout(t.key_bytes, nq);
    if (!d_workspace || ws_bytes < w.total || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return BT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const SortNorm sn = make_norm(t, sort_bits, nq);
    cudaError_t e;
    if (sn.passes == 0) {
        const unsigned grid = static_cast<unsigned>((nq + 255) / 256 < 4096 ? (nq + 255) / 256 : 4096);
        if (t.key_bytes == 8)
            k_copy_identity<uint64_t><<<grid, 256, 0, s>>>(static_cast<const uint64_t *>(d_queries),
                                                           static_cast<uint64_t *>(d_sorted_queries),
                                                           d_sorted_index, nq);
        else
            k_copy_identity<uint32_t><<<grid, 256, 0, s>>>(static_cast<const uint32_t *>(d_queries),
                                                           static_cast<uint32_t *>(d_sorted_queries),
                                                           d_sorted_index, nq);
        e = cudaGetLastError();
    } else {
        e = sort_any(t, d_queries, nq, sn, static_cast<unsigned char *>(d_workspace), w, d_sorted_queries,
                     d_sorted_index, s);
    }
    if (e != cudaSuccess) {
        set_error_detail("radix sort launch", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}

extern "C" bt_status bt_descend_sorted(const bt_tree *tree, const void *d_queries, const uint32_t *d_index,
                                       uint64_t nq, void *d_out_vals, uint8_t *d_out_found,
                                       unsigned long long *d_fetch_counts, bt_stream stream)
{
    if (!tree) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    if (nq >= (1ull << 31)) return BT_ERR_ARG;
    if (!d_queries || !d_out_vals || !d_out_found) return BT_ERR_ARG;
    const DevTree &t = tree->dev;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (t.height == 0) {
        const unsigned grid = static_cast<unsigned>((nq + 255) / 256 < 4096 ? (nq + 255) / 256 : 4096);
        if (t.val_bytes == 8)
            k_fill_miss<uint64_t><<<grid, 256, 0, s>>>(static_cast<uint64_t *>(d_out_vals), d_out_found, nq);
        else
            k_fill_miss<uint32_t><<<grid, 256, 0, s>>>(static_cast<uint32_t *>(d_out_vals), d_out_found, nq);
        e = cudaGetLastError();
    } else {
        e = descend(t, d_queries, d_index, nq, d_out_vals, d_out_found, d_fetch_counts, s);
    }
    if (e != cudaSuccess) {
        set_error_detail("descent launch", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}
