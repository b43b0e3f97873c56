// Batched level-wise B+ tree point search on GB300 (sm_103a): the search
// entry points.
//
// One search is (Sec. IV-A, IV-F):
//   1. an on-device partition of (query, input position) pairs by a bucket
//      number monotone in the key (part_sort.cuh), so that queries routed
//      to the same node end up adjacent (the paper's sorted batch);
//   2. the level-wise descent (desc_pipe.cu; desc_sync.cu holds the
//      synchronous alternatives): each warp takes 32 consecutive queries of
//      the sorted batch and walks them down the tree together, every node a
//      query needs fetched once per warp, and every query finding its child
//      rank -- the number of separators smaller than the query, i.e. the
//      first separator it is <= to (Sec. IV-E's priority encoder);
//   3. the leaf probe (Sec. IV-D): the same rank in the leaf block is the
//      only slot that can hold an equal key; a hit reads the value, a miss
//      returns all-ones (the paper's -1) with found = 0;
//   4. the scatter of each result back to the query's input position.
// Everything is integer compares; nothing here is a dense contraction, so
// no tensor-core path is used.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <type_traits>

#include "descent.cuh"
#include "part_sort.cuh"

namespace btgb {

cudaError_t persistent_grid(const void *kern, int threads, int smem, uint64_t units_per_block, uint64_t units,
                            unsigned *grid, int max_per_sm)
{
    int per_sm = 0, sms = 0;
    cudaError_t e = blocks_per_sm(kern, threads, smem, &per_sm);
    if (e == cudaSuccess) e = dev_sm_count(&sms);
    if (e != cudaSuccess) return e;
    if (max_per_sm > 0 && max_per_sm < per_sm) per_sm = max_per_sm;
    uint64_t g = (units + units_per_block - 1) / units_per_block;
    const uint64_t cap = static_cast<uint64_t>(sms) * static_cast<uint64_t>(per_sm);
    if (g > cap) g = cap;
    *grid = static_cast<unsigned>(g > 0 ? g : 1);
    return cudaSuccess;
}

static cudaError_t descend_any(const DescendArgs &a, cudaStream_t s)
{
    if (a.md || (a.t->staging == BT_STAGE_PIPELINED && a.t->lane_queries == 1)) return descend_pipelined(a, s);
    return descend_synchronous(a, s);
}

// view: the tree as the descent sees it (null: the tree itself).
static cudaError_t descend(const bt_tree *tree, const void *q, const uint32_t *qidx, const void *recs, uint64_t nq,
                           void *out_v, uint8_t *out_f, unsigned long long *fetch, cudaStream_t s,
                           const DevTree *view = nullptr)
{
    const DescendArgs a{view ? view : &tree->dev, tree, q, qidx, recs, nq, out_v, out_f, fetch, nullptr, nullptr};
    return descend_any(a, s);
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

struct WsLayout {
    uint64_t rec, ridx, pairs, counts, total;
};

// Coarse-bucket totals of the partition and its two grid-barrier counters:
// at most 2^kMaxCoarseBits buckets.
constexpr uint64_t kPartCountWords = (1ull << kMaxCoarseBits) + 4;

// Queries per partition block (at least).
constexpr uint64_t kPartPerBlock = 2048;

// Workspace: the partitioned batch -- for integer keys one record per
// query (key, input position, local digit), for 32-byte keys an array of
// the keys (rec) and one of their input positions (ridx), made from the
// scattered (position, digit) pairs -- and the partition's bucket totals
// and barrier counters.
static WsLayout ws_layout(int kb, uint64_t nq)
{
    WsLayout w;
    uint64_t o = 0;
    w.rec = o;
    if (kb > 8) {
        o = align256(o + nq * sizeof(Raw32));
        w.ridx = o;
        o = align256(o + nq * 4);
    } else {
        o = align256(o + nq * sizeof(PartRec<uint64_t>));
        w.ridx = w.rec;
    }
    w.pairs = o;
    if (kb > 8) o = align256(o + nq * 8);
    w.counts = o;
    o = align256(o + kPartCountWords * 4);
    w.total = nq ? o : 0;
    return w;
}

static int bitlen(uint64_t x) { return x ? 64 - __builtin_clzll(x) : 0; }

// Device arrays a search reads or writes are aligned to their element size
// (32-byte keys: to 16 bytes, the width of the loads and stores that move
// them); qidx and vals may be null (not checked).
static bool arrays_aligned(const DevTree &t, const void *keys, const void *qidx, const void *vals)
{
    const uintptr_t ka = static_cast<uintptr_t>(t.key_bytes > 16 ? 16 : t.key_bytes);
    const uintptr_t va = static_cast<uintptr_t>(t.val_bytes);
    return (reinterpret_cast<uintptr_t>(keys) & (ka - 1)) == 0 && (reinterpret_cast<uintptr_t>(qidx) & 3u) == 0 &&
           (reinterpret_cast<uintptr_t>(vals) & (va - 1)) == 0;
}

// Queries per batch from which the automatic choice partitions the batch,
// for trees larger than a quarter of the L2 (DevTree::sort_pays).  Measured
// on uint64 trees at fanout 32: on 2^24 keys the unsorted descent is faster
// up to 2^19 queries (53 against 61 us), the sorted search from 2^20 (86
// against 90 us); on 4 * 10^6 keys (67 MB) likewise (49 against 52 us at 2^19,
// 79 against 82 at 2^20); on 10^6 keys (17 MB) the unsorted descent is faster
// at every size to 2^20 (61 against 72 us there).
constexpr uint64_t kAutoSortMinBatch = 786432;
// The same for 32-byte keys, whose comparisons and 512-byte node blocks make
// the unsorted descent dearer: on 2^20 keys at fanout 16 (47 MB) the sorted
// search is faster from 2^19 queries (70 against 73 us with the L2 warm, 75
// against 82 flushed), the unsorted one at 2^18 (43 against 47 us).
constexpr uint64_t kAutoSortMinBatch32 = 393216;
// Automatic bits: coarse buckets of 512 to 1023 queries on average, each
// ordered by kLocalBits more bits -- finer than one leaf per query at every
// configured batch size; at least 2 buckets and at most 2^kMaxCoarseBits,
// so from 2^22 queries the average bucket reaches the local sort's tile and
// larger buckets keep the scatter's order.
static int auto_part_bits(int key_bytes, uint64_t nq)
{
    (void)key_bytes;
    int cb = bitlen(nq) - 10;
    cb = cb < 1 ? 1 : (cb > kMaxCoarseBits ? kMaxCoarseBits : cb);
    return cb + kLocalBits;
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

// Partition parameters for a tree and batch: how c (the splitter count
// below the query) and the interpolation bits r make f on `bits` bits, and
// how f splits into the coarse bucket and the local digit.
struct PartPlan {
    int bits;       // 0: no partition
    int r;          // interpolation bits inside a splitter segment
    int cshift;     // right shift of c when bits < the splitter bits
    int lb;         // digit bits (0: no local sort)
    uint32_t nb;    // coarse buckets, rounded up to a multiple of 4
};

// sort_bits < 0: auto_part_bits for batches of at least kAutoSortMinBatch
// queries (kAutoSortMinBatch32 for 32-byte keys) over trees larger than a
// quarter of the L2, else none; sort_bits > 0: that many
// bits, at most kMaxPartBits.
static PartPlan plan_partition(const DevTree &t, int32_t sort_bits, uint64_t nq)
{
    PartPlan p{0, 0, 0, 0, 0};
    int bits = sort_bits;
    if (bits < 0) {
        const uint64_t min_nq = t.key_bytes == 32 ? kAutoSortMinBatch32 : kAutoSortMinBatch;
        bits = (t.sort_pays && nq >= min_nq) ? auto_part_bits(t.key_bytes, nq) : 0;
    }
    if (bits > kMaxPartBits) bits = kMaxPartBits;
    if (bits <= 0 || t.height == 0) return p;
    const int cbits = bitlen(t.nsplit);  // c is in [0, nsplit]
    p.bits = bits;
    p.r = bits > cbits ? bits - cbits : 0;
    p.cshift = cbits > bits ? cbits - bits : 0;
    p.lb = bits - 1 < kLocalBits ? bits - 1 : kLocalBits;
    const uint64_t fmax = p.r ? ((static_cast<uint64_t>(t.nsplit) << p.r) | ((1ull << p.r) - 1))
                              : (static_cast<uint64_t>(t.nsplit) >> p.cshift);
    const uint64_t nb = (fmax >> p.lb) + 1;
    p.nb = static_cast<uint32_t>((nb + 3) / 4 * 4);
    return p;
}

template <typename K>
static void tree_bounds(const DevTree &t, K *lo, K *hi)
{
    *lo = static_cast<K>(t.kmin);
    *hi = static_cast<K>(t.kmax);
}

template <>
void tree_bounds<Key32>(const DevTree &t, Key32 *lo, Key32 *hi)
{
    for (int j = 0; j < 4; ++j) {
        lo->w[j] = t.kmin32[j];
        hi->w[j] = t.kmax32[j];
    }
}

// Kernels the partition launches for a plan (plus one memset).
static int part_kernels(const PartPlan &pp) { return pp.bits ? 1 : 0; }

// out_q / out_i: where 32-byte keys' partitioned keys and positions go
// (unused for integer keys, whose records stay in the workspace).
template <typename K>
static cudaError_t part_sort(const DevTree &t, const RawOf<K> *q, uint64_t nq, const PartPlan &pp,
                             unsigned char *ws, const WsLayout &w, RawOf<K> *out_q, uint32_t *out_i,
                             cudaStream_t s)
{
    PartNorm<K> pn;
    pn.split = static_cast<const K *>(t.split);
    pn.split_inv = t.split_inv;
    pn.split_off = t.split_off;
    tree_bounds<K>(t, &pn.kmin, &pn.kmax);
    pn.nsplit = t.nsplit;
    pn.r = pp.r;
    pn.cshift = pp.cshift;
    pn.lb = pp.lb;
    pn.scale = static_cast<float>(1u << pp.r);
    pn.split_R = t.split_R;
    pn.rshift = t.split_rshift;
    pn.p0 = t.split_p0;
    pn.wmin = t.split_wmin;
    unsigned int *total = reinterpret_cast<unsigned int *>(ws + w.counts);
    PartRec<K> *rec = part_narrow<K>() ? nullptr : reinterpret_cast<PartRec<K> *>(ws + w.rec);
    uint2 *pairs = part_narrow<K>() ? reinterpret_cast<uint2 *>(ws + w.pairs) : nullptr;
    if (!part_narrow<K>()) {
        out_q = nullptr;
        out_i = nullptr;
    }
    cudaError_t e = cudaMemsetAsync(total, 0, (static_cast<uint64_t>(pp.nb) + 4) * 4, s);
    if (e != cudaSuccess) return e;
    const void *kern = reinterpret_cast<const void *>(k_partition<K>);
    e = ensure_dyn_smem(kern, part_dyn<K>(1u << kMaxCoarseBits));
    if (e != cudaSuccess) return e;
    const int dyn = part_dyn<K>(pp.nb);
    int sms = 0, occ = 0;
    e = dev_sm_count(&sms);
    if (e == cudaSuccess) e = blocks_per_sm(kern, kPartThreads, dyn, &occ);
    if (e != cudaSuccess) return e;
    // one slice per block, at least kPartPerBlock queries each, every block
    // resident (the kernel's grid barriers need all of them)
    uint64_t g = (nq + kPartPerBlock - 1) / kPartPerBlock;
    if (t.corun_partition_bps > 0 && t.corun_partition_bps < occ) occ = t.corun_partition_bps;
    const uint64_t cap = static_cast<uint64_t>(occ) * static_cast<uint64_t>(sms);
    if (g > cap) g = cap;
    if (g > kMaxPartBlocks) g = kMaxPartBlocks;
    uint32_t nb = pp.nb, polls = first_wait_polls();
    void *args[] = {const_cast<RawOf<K> **>(&q), &nq, &pn, &total, &nb, &rec, &pairs, &out_q, &out_i, &polls};
    return cudaLaunchCooperativeKernel(kern, dim3(static_cast<unsigned>(g)), dim3(kPartThreads), args,
                                       static_cast<size_t>(dyn), s);
}

// Where the descent finds a partitioned batch: the workspace's records
// (integer keys), or its key and position arrays (32-byte keys).
struct PartOut {
    const void *q;
    const uint32_t *qidx;
    const void *recs;
};

static PartOut part_output(const DevTree &t, const unsigned char *ws, const WsLayout &w)
{
    if (t.key_bytes == 32) return {ws + w.rec, reinterpret_cast<const uint32_t *>(ws + w.ridx), nullptr};
    return {nullptr, nullptr, ws + w.rec};
}

// The descent's view of a tree for a partitioned batch: inner-level staging
// left to the library ("auto") is on, as for a batch given as records.
static DevTree partitioned_view(const DevTree &t)
{
    DevTree v = t;
    if (v.inner_stage == 2) v.inner_stage = 1;
    return v;
}

// The partition of a batch into the workspace (32-byte keys: into out_q /
// out_i when given, else the workspace's key and position arrays).
static cudaError_t sort_any(const DevTree &t, const void *q, uint64_t nq, const PartPlan &pp,
                            unsigned char *ws, const WsLayout &w, cudaStream_t s, void *out_q = nullptr,
                            uint32_t *out_i = nullptr)
{
    if (t.key_bytes == 32) {
        Raw32 *oq = out_q ? static_cast<Raw32 *>(out_q) : reinterpret_cast<Raw32 *>(ws + w.rec);
        uint32_t *oi = out_i ? out_i : reinterpret_cast<uint32_t *>(ws + w.ridx);
        return part_sort<Key32>(t, static_cast<const Raw32 *>(q), nq, pp, ws, w, oq, oi, s);
    }
    if (t.key_bytes == 8)
        return part_sort<uint64_t>(t, static_cast<const uint64_t *>(q), nq, pp, ws, w, nullptr, nullptr, s);
    return part_sort<uint32_t>(t, static_cast<const uint32_t *>(q), nq, pp, ws, w, nullptr, nullptr, s);
}

// The records of integer keys split into the caller's key and position
// arrays.
static cudaError_t unpack_any(const DevTree &t, const unsigned char *recs, uint64_t nq, void *dq, uint32_t *di,
                              cudaStream_t s)
{
    const unsigned grid = static_cast<unsigned>((nq + 255) / 256 < 4096 ? (nq + 255) / 256 : 4096);
    if (t.key_bytes == 8)
        k_part_unpack<uint64_t><<<grid, 256, 0, s>>>(reinterpret_cast<const PartRec<uint64_t> *>(recs), nq,
                                                     static_cast<uint64_t *>(dq), di);
    else
        k_part_unpack<uint32_t><<<grid, 256, 0, s>>>(reinterpret_cast<const PartRec<uint32_t> *>(recs), nq,
                                                     static_cast<uint32_t *>(dq), di);
    return cudaGetLastError();
}

}  // namespace btgb

using namespace btgb;

extern "C" int32_t bt_sort_launches(const bt_tree *tree, uint64_t nq, int32_t sort_bits)
{
    if (!tree) return -1;
    if (tree->dev.height == 0 || nq == 0) return 0;
    return part_kernels(plan_partition(tree->dev, sort_bits, nq));
}

extern "C" int32_t bt_sort_bits(const bt_tree *tree, uint64_t nq, int32_t sort_bits)
{
    if (!tree) return -1;
    if (tree->dev.height == 0 || nq == 0) return 0;
    return plan_partition(tree->dev, sort_bits, nq).bits;
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
    if (!arrays_aligned(tree->dev, d_queries, nullptr, d_out_vals)) return BT_ERR_ARG;
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

    const PartPlan pp = plan_partition(t, opts ? opts->sort_bits : -1, nq);
    const void *q = d_queries;
    const uint32_t *qidx = nullptr;
    const void *recs = nullptr;
    unsigned char *ws = static_cast<unsigned char *>(d_workspace);
    DevTree pv;
    const DevTree *view = nullptr;
    if (pp.bits > 0) {
        e = sort_any(t, d_queries, nq, pp, ws, w, s);
        if (e != cudaSuccess) {
            set_error_detail("batch partition launch", e);
            return BT_ERR_CUDA;
        }
        const PartOut po = part_output(t, ws, w);
        q = po.q;
        qidx = po.qidx;
        recs = po.recs;
        if (!recs) {
            pv = partitioned_view(t);
            view = &pv;
        }
    }
    if (opts && opts->phase_event) {
        e = cudaEventRecord(static_cast<cudaEvent_t>(opts->phase_event), s);
        if (e != cudaSuccess) {
            set_error_detail("phase event", e);
            return BT_ERR_CUDA;
        }
    }
    e = descend(tree, q, qidx, recs, nq, d_out_vals, d_out_found, opts ? opts->d_fetch_counts : nullptr, s, view);
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
    if (!arrays_aligned(tree->dev, d_queries, d_sorted_index, nullptr) ||
        !arrays_aligned(tree->dev, d_sorted_queries, nullptr, nullptr))
        return BT_ERR_ARG;
    const DevTree &t = tree->dev;
    const WsLayout w = ws_layout(t.key_bytes, nq);
    if (!d_workspace || ws_bytes < w.total || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return BT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const PartPlan pp = plan_partition(t, sort_bits, nq);
    cudaError_t e;
    if (pp.bits == 0) {
        const unsigned grid = static_cast<unsigned>((nq + 255) / 256 < 4096 ? (nq + 255) / 256 : 4096);
        if (t.key_bytes == 32)
            k_copy_identity<Raw32><<<grid, 256, 0, s>>>(static_cast<const Raw32 *>(d_queries),
                                                        static_cast<Raw32 *>(d_sorted_queries), d_sorted_index, nq);
        else if (t.key_bytes == 8)
            k_copy_identity<uint64_t><<<grid, 256, 0, s>>>(static_cast<const uint64_t *>(d_queries),
                                                           static_cast<uint64_t *>(d_sorted_queries),
                                                           d_sorted_index, nq);
        else
            k_copy_identity<uint32_t><<<grid, 256, 0, s>>>(static_cast<const uint32_t *>(d_queries),
                                                           static_cast<uint32_t *>(d_sorted_queries),
                                                           d_sorted_index, nq);
        e = cudaGetLastError();
    } else {
        unsigned char *ws = static_cast<unsigned char *>(d_workspace);
        if (t.key_bytes == 32) {  // written straight into the caller's arrays
            e = sort_any(t, d_queries, nq, pp, ws, w, s, d_sorted_queries, d_sorted_index);
        } else {
            e = sort_any(t, d_queries, nq, pp, ws, w, s);
            if (e == cudaSuccess) e = unpack_any(t, ws + w.rec, nq, d_sorted_queries, d_sorted_index, s);
        }
    }
    if (e != cudaSuccess) {
        set_error_detail("batch partition launch", e);
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
    if (!arrays_aligned(tree->dev, d_queries, d_index, d_out_vals)) return BT_ERR_ARG;
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
        e = descend(tree, d_queries, d_index, nullptr, nq, d_out_vals, d_out_found, d_fetch_counts, s);
    }
    if (e != cudaSuccess) {
        set_error_detail("descent launch", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}

extern "C" bt_status bt_learned_descend_sorted(const bt_tree *tree, const bt_model *model, const void *d_queries,
                                               const uint32_t *d_index, uint64_t nq, void *d_out_vals,
                                               uint8_t *d_out_found, unsigned long long *d_stats, bt_stream stream)
{
    if (!tree || !model) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    if (nq >= (1ull << 31)) return BT_ERR_ARG;
    if (!d_queries || !d_out_vals || !d_out_found) return BT_ERR_ARG;
    if (!arrays_aligned(tree->dev, d_queries, d_index, d_out_vals)) return BT_ERR_ARG;
    const DevTree &t = tree->dev;
    if (t.height == 0 || model->dev.leaves != t.nodes[t.height - 1]) return BT_ERR_ARG;
    const DescendArgs a{&t, tree, d_queries, d_index, nullptr, nq, d_out_vals, d_out_found, nullptr, &model->dev,
                        d_stats};
    const cudaError_t e = descend_any(a, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        set_error_detail("learned descent launch", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}

extern "C" bt_status bt_learned_search_batch(const bt_tree *tree, const bt_model *model, const void *d_queries,
                                             uint64_t nq, void *d_out_vals, uint8_t *d_out_found, void *d_workspace,
                                             uint64_t ws_bytes, bt_stream stream)
{
    if (!tree || !model) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    if (nq >= (1ull << 31)) return BT_ERR_ARG;
    if (!d_queries || !d_out_vals || !d_out_found) return BT_ERR_ARG;
    if (!arrays_aligned(tree->dev, d_queries, nullptr, d_out_vals)) return BT_ERR_ARG;
    const DevTree &t = tree->dev;
    if (t.height == 0 || model->dev.leaves != t.nodes[t.height - 1]) return BT_ERR_ARG;
    const WsLayout w = ws_layout(t.key_bytes, nq);
    if (!d_workspace || ws_bytes < w.total || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return BT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const PartPlan pp = plan_partition(t, -1, nq);
    const void *q = d_queries;
    const uint32_t *qidx = nullptr;
    const void *recs = nullptr;
    unsigned char *ws = static_cast<unsigned char *>(d_workspace);
    cudaError_t e;
    if (pp.bits > 0) {
        e = sort_any(t, d_queries, nq, pp, ws, w, s);
        if (e != cudaSuccess) {
            set_error_detail("batch partition launch", e);
            return BT_ERR_CUDA;
        }
        const PartOut po = part_output(t, ws, w);
        q = po.q;
        qidx = po.qidx;
        recs = po.recs;
    }
    const DescendArgs a{&t, tree, q, qidx, recs, nq, d_out_vals, d_out_found, nullptr, &model->dev, nullptr};
    e = descend_any(a, s);
    if (e != cudaSuccess) {
        set_error_detail("learned descent launch", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}

extern "C" bt_status bt_check_timeouts(void)
{
    unsigned timeouts = 0, pending = 0;
    cudaError_t e = take_wait_counters_pipelined(&timeouts, &pending);
    if (e == cudaSuccess) {
        unsigned v = 0;
        e = cudaMemcpyFromSymbol(&v, g_part_timeouts, sizeof(v));
        const unsigned zero = 0;
        if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_part_timeouts, &zero, sizeof(zero));
        timeouts += v;
    }
    if (e == cudaSuccess) e = take_wait_counters_synchronous(&timeouts, &pending);
    if (e != cudaSuccess) {
        set_error_detail("timeout counters", e);
        return BT_ERR_CUDA;
    }
    return (timeouts || pending) ? BT_ERR_TIMEOUT : BT_OK;
}

extern "C" bt_status bt_paper_descend_sorted(const bt_tree *tree, const void *d_queries, const uint32_t *d_index,
                                             uint64_t nq, void *d_out_vals, uint8_t *d_out_found, bt_stream stream)
{
    if (!tree) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    if (nq >= (1ull << 31)) return BT_ERR_ARG;
    if (!d_queries || !d_out_vals || !d_out_found) return BT_ERR_ARG;
    if (!arrays_aligned(tree->dev, d_queries, d_index, d_out_vals)) return BT_ERR_ARG;
    if (tree->dev.height > 0 && !tree->d_paper) return BT_ERR_ARG;
    if (tree->dev.height == 0) return bt_descend_sorted(tree, d_queries, d_index, nq, d_out_vals, d_out_found,
                                                        nullptr, stream);
    const cudaError_t e = descend_paper_layout(tree->dev, tree->paper, d_queries, d_index, nullptr, nq, d_out_vals,
                                               d_out_found, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        set_error_detail("paper-layout descent launch", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}

extern "C" bt_status bt_paper_search_batch(const bt_tree *tree, const void *d_queries, uint64_t nq, void *d_out_vals,
                                           uint8_t *d_out_found, void *d_workspace, uint64_t ws_bytes,
                                           bt_stream stream)
{
    if (!tree) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    if (nq >= (1ull << 31)) return BT_ERR_ARG;
    if (!d_queries || !d_out_vals || !d_out_found) return BT_ERR_ARG;
    if (!arrays_aligned(tree->dev, d_queries, nullptr, d_out_vals)) return BT_ERR_ARG;
    const DevTree &t = tree->dev;
    if (t.height > 0 && !tree->d_paper) return BT_ERR_ARG;
    if (t.height == 0)
        return bt_search_batch(tree, d_queries, nq, d_out_vals, d_out_found, d_workspace, ws_bytes, stream);
    const WsLayout w = ws_layout(t.key_bytes, nq);
    if (!d_workspace || ws_bytes < w.total || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return BT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const PartPlan pp = plan_partition(t, -1, nq);
    const void *q = d_queries;
    const uint32_t *qidx = nullptr;
    const void *recs = nullptr;
    unsigned char *ws = static_cast<unsigned char *>(d_workspace);
    cudaError_t e;
    if (pp.bits > 0) {
        e = sort_any(t, d_queries, nq, pp, ws, w, s);
        if (e != cudaSuccess) {
            set_error_detail("batch partition launch", e);
            return BT_ERR_CUDA;
        }
        const PartOut po = part_output(t, ws, w);
        q = po.q;
        qidx = po.qidx;
        recs = po.recs;
    }
    e = descend_paper_layout(t, tree->paper, q, qidx, recs, nq, d_out_vals, d_out_found, s);
    if (e != cudaSuccess) {
        set_error_detail("paper-layout descent launch", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}
