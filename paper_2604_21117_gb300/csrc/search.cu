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
#include "radix_sort.cuh"

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

// -------------------------------------------- level-wise descent (a3-a5)
//
// Persistent blocks of kDescWarps warps.  Each block first copies the top
// levels of the tree (as many whole levels as fit kPinBudget bytes, never
// the leaves) into shared memory once; a warp then loops over chunks of 32
// consecutive queries of the (sorted) batch, prefetching the next chunk's
// queries and output positions while it works on the current one.  Per
// level below the pinned ones, the warp's distinct nodes are staged into
// its shared-memory slots (rounds of `stage_slots` nodes) before the binary
// searches.

constexpr int kDescWarps = 8;
constexpr int kPinBudget = 16384;

template <typename K, int M>
constexpr int stage_slots()
{
    return (M * static_cast<int>(sizeof(K)) >= 512) ? 8 : 16;
}

template <typename K, int M>
constexpr int desc_smem_fixed()
{
    return kDescWarps * (stage_slots<K, M>() * M * static_cast<int>(sizeof(K)) + 32 * 4);
}

// Number of slots of a node block holding a key smaller than `key`: the
// child rank at an inner node (the first separator the key is <= to), the
// only possible match position at a leaf.  Slot M-1 is always padding
// (all-ones), so log2(M) probes of a branchless binary search suffice.
template <typename K, int M>
__device__ __forceinline__ int block_rank(const K *blk, K key)
{
    int r = 0;
#pragma unroll
    for (int hlf = M / 2; hlf >= 1; hlf >>= 1)
        if (blk[r + hlf - 1] < key) r += hlf;
    return r;
}

// The distinct node ids among the warp's 32 lanes -- the paper's FIFO
// entries (node address, number of queries) for this warp.  Writes them to
// list[0..U) and gives each lane the position `slot` of its own node there.
// A sorted batch keeps a warp's nodes within a narrow range, handled with
// warp reductions and a 32-bit presence mask; a wider range falls back to
// warp match.  Every lane of the warp must call it.
__device__ __forceinline__ void warp_distinct(uint32_t node, int lane, uint32_t *list, int &U, int &slot)
{
    const uint32_t nmin = __reduce_min_sync(0xffffffffu, node);
    const uint32_t nmax = __reduce_max_sync(0xffffffffu, node);
    if (nmax - nmin < 32u) {
        const unsigned bit = 1u << (node - nmin);
        const unsigned mask = __reduce_or_sync(0xffffffffu, bit);
        U = __popc(mask);
        slot = __popc(mask & (bit - 1u));
        if ((mask >> lane) & 1u) list[__popc(mask & ((1u << lane) - 1u))] = nmin + lane;
    } else {
        const unsigned same = __match_any_sync(0xffffffffu, node);
        const int leader = __ffs(same) - 1;
        const unsigned leaders = __ballot_sync(0xffffffffu, lane == leader);
        U = __popc(leaders);
        slot = __popc(leaders & ((1u << leader) - 1u));
        if (lane == leader) list[slot] = node;
    }
}

__device__ __forceinline__ uint32_t child_of(const DevTree &t, int l, uint32_t node, int r)
{
    const uint64_t base = t.cbase[l], rem = t.crem[l];
    return static_cast<uint32_t>(node * base + (node < rem ? node : rem) + r);
}

template <typename K, typename V, int M, bool COUNT>
__global__ void __launch_bounds__(kDescWarps * 32) k_descend(
    const DevTree t, const K *__restrict__ q, const uint32_t *__restrict__ qidx, uint64_t nq,
    V *__restrict__ out_v, uint8_t *__restrict__ out_f, unsigned long long *__restrict__ fetch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int CH = M * static_cast<int>(sizeof(K)) / 16;  // 16-byte chunks per node block
    constexpr int SLOTS = stage_slots<K, M>();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t pin_bytes = t.pin_bytes;
    unsigned char *pin = smem;
    K *stage = reinterpret_cast<K *>(smem + pin_bytes) + warp * SLOTS * M;
    uint32_t *list = reinterpret_cast<uint32_t *>(smem + pin_bytes + kDescWarps * SLOTS * M * sizeof(K)) + warp * 32;

    // Top levels, pinned once per block.
    const unsigned char *top = static_cast<const unsigned char *>(t.keys[0]);
    for (uint32_t i = threadIdx.x * 16u; i < pin_bytes; i += blockDim.x * 16u) cp_async16_ca(pin + i, top + i);
    cp_async_wait_all();
    __syncthreads();

    const uint64_t nchunks = (nq + 31) / 32;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kDescWarps;
    const int H = t.height, P = t.pin_levels;
    uint64_t c = static_cast<uint64_t>(blockIdx.x) * kDescWarps + warp;
    if (c >= nchunks) return;

    // Tail lanes follow lane 0's query so they never add a node fetch.
    K key_n;
    uint32_t dst_n;
    {
        const uint64_t pos = c * 32 + lane;
        const bool v = pos < nq;
        key_n = q[v ? pos : c * 32];
        dst_n = v ? (qidx ? qidx[pos] : static_cast<uint32_t>(pos)) : 0u;
    }
    for (;;) {
        const uint64_t pos = c * 32 + lane;
        const bool valid = pos < nq;
        const K key = key_n;
        const uint32_t dst = dst_n;
        const uint64_t cn = c + stride;
        if (cn < nchunks) {  // prefetch the next chunk
            const uint64_t pn = cn * 32 + lane;
            const bool vn = pn < nq;
            key_n = q[vn ? pn : cn * 32];
            dst_n = vn ? (qidx ? qidx[pn] : static_cast<uint32_t>(pn)) : 0u;
        }

        uint32_t node = 0;
        int l = 0;
        for (; l < P; ++l) {  // pinned levels: search the block's shared copy
            if (COUNT) {
                int U, slot;
                warp_distinct(node, lane, list, U, slot);
                __syncwarp();
                if (lane == 0) atomicAdd(fetch + l, static_cast<unsigned long long>(U));
            }
            const K *blk = reinterpret_cast<const K *>(
                               pin + (static_cast<const unsigned char *>(t.keys[l]) - top)) +
                           static_cast<uint64_t>(node) * M;
            node = child_of(t, l, node, block_rank<K, M>(blk, key));
        }
        for (; l < H; ++l) {
            const K *lk = static_cast<const K *>(t.keys[l]);
            const bool last = (l + 1 == H);
            int U, slot;
            warp_distinct(node, lane, list, U, slot);
            if (COUNT && lane == 0) atomicAdd(fetch + l, static_cast<unsigned long long>(U));
            __syncwarp();
            int r = 0;
            bool eq = false;
            for (int rb = 0; rb < U; rb += SLOTS) {
                const int nu = (U - rb < SLOTS) ? U - rb : SLOTS;
                // Stage each distinct node's key block once.
                for (int i = lane; i < nu * CH; i += 32) {
                    const int u = i / CH, part = i - u * CH;
                    const unsigned char *src = reinterpret_cast<const unsigned char *>(
                                                   lk + static_cast<uint64_t>(list[rb + u]) * M) + part * 16;
                    unsigned char *dp = reinterpret_cast<unsigned char *>(stage + u * M) + part * 16;
                    if (last)
                        cp_async16_cg(dp, src);
                    else
                        cp_async16_ca(dp, src);
                }
                cp_async_wait_all();
                __syncwarp();
                if (slot >= rb && slot < rb + nu) {
                    const K *blk = stage + (slot - rb) * M;
                    r = block_rank<K, M>(blk, key);
                    eq = (blk[r] == key);
                }
                __syncwarp();
            }
            if (!last) {
                node = child_of(t, l, node, r);
            } else {
                const uint64_t cnt = t.cbase[l] + (node < t.crem[l] ? 1u : 0u);
                const bool hit = (static_cast<uint64_t>(r) < cnt) && eq;
                V val = static_cast<V>(~static_cast<V>(0));
                if (hit) val = static_cast<const V *>(t.vals)[static_cast<uint64_t>(node) * M + r];
                if (valid) {
                    out_v[dst] = val;
                    out_f[dst] = hit ? 1 : 0;
                }
            }
        }
        if (cn >= nchunks) break;
        c = cn;
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
    uint64_t qa, ia, qb, ib, meta, status, total;
};

// Workspace: two ping-pong (query, position) buffers, then the sort's
// metadata block (global digit histograms, tile counters, error word) and
// the per-tile look-back status words.
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
    w.meta = o;
    o = align256(o + (kMaxPasses * 256 + kMaxPasses + 1) * 4);
    w.status = o;
    o = align256(o + static_cast<uint64_t>(kMaxPasses) * sort_tiles(nq) * 256u * 8u);
    w.total = nq ? o : 0;
    return w;
}

static SortMeta sort_meta(unsigned char *ws, const WsLayout &w)
{
    SortMeta m;
    m.ghist = reinterpret_cast<uint32_t *>(ws + w.meta);
    m.tile_ctr = m.ghist + kMaxPasses * 256;
    m.err = m.tile_ctr + kMaxPasses;
    m.status = reinterpret_cast<unsigned long long *>(ws + w.status);
    return m;
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
    constexpr int fixed = desc_smem_fixed<K, M>();
    constexpr int threads = kDescWarps * 32;
    auto kern = k_descend<K, V, M, COUNT>;
    static const cudaError_t attr =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, fixed + kPinBudget);
    if (attr != cudaSuccess) return attr;
    const int smem = fixed + static_cast<int>(t.pin_bytes);
    // resident blocks per SM for this shared-memory size (cached per size)
    static int occ_cache[kPinBudget / 256 + 2] = {0};
    const int key = static_cast<int>((t.pin_bytes + 255) / 256);
    if (occ_cache[key] == 0) {
        int b = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, fixed + key * 256);
        if (e != cudaSuccess) return e;
        occ_cache[key] = b > 0 ? b : 1;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const uint64_t chunks = (nq + 31) / 32;
    uint64_t grid = (chunks + kDescWarps - 1) / kDescWarps;
    const uint64_t cap = static_cast<uint64_t>(sms) * occ_cache[key];
    if (grid > cap) grid = cap;
    kern<<<static_cast<unsigned>(grid), threads, smem, s>>>(t, static_cast<const K *>(q), qidx, nq,
                                                           static_cast<V *>(out_v), out_f, fetch);
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
    const SortMeta meta = sort_meta(ws, w);
    // histograms, tile counters, error word and the used status words start at zero
    cudaError_t e = cudaMemsetAsync(ws + w.meta, 0,
                                    (w.status - w.meta) + static_cast<uint64_t>(sn.passes) * ntiles * 256u * 8u, s);
    if (e != cudaSuccess) return e;
    constexpr int smem = sort_pass_smem_bytes<K>();
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_sort_pass<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    k_sort_hist<K><<<ntiles, kSortThreads, 0, s>>>(q, nq, sn, meta.ghist);
    K *qa = reinterpret_cast<K *>(ws + w.qa), *qb = reinterpret_cast<K *>(ws + w.qb);
    uint32_t *ia = reinterpret_cast<uint32_t *>(ws + w.ia), *ib = reinterpret_cast<uint32_t *>(ws + w.ib);
    const K *src_q = q;
    const uint32_t *src_i = nullptr;
    for (int p = 0; p < sn.passes; ++p) {
        const bool final_pass = (p + 1 == sn.passes);
        K *dq = final_pass ? dst_q : ((p & 1) ? qb : qa);
        uint32_t *di = final_pass ? dst_i : ((p & 1) ? ib : ia);
        k_sort_pass<K><<<ntiles, kSortThreads, smem, s>>>(src_q, src_i, dq, di, nq, sn, p, meta, ntiles);
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

extern "C" bt_status bt_workspace_status(const bt_tree *tree, const void *d_workspace, uint64_t nq)
{
    if (!tree || !d_workspace) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    const WsLayout w = ws_layout(tree->dev.key_bytes, nq);
    uint32_t err = 0;
    const unsigned char *ws = static_cast<const unsigned char *>(d_workspace);
    cudaError_t e = cudaMemcpy(&err, ws + w.meta + (kMaxPasses * 256 + kMaxPasses) * 4, 4,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_error_detail("workspace status read", e);
        return BT_ERR_CUDA;
    }
    return err ? BT_ERR_TIMEOUT : BT_OK;
}

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
