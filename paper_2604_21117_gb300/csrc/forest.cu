// Many batches over several resident trees in one persistent launch.
//
// A "forest" is a table of built trees sharing key and value widths
// (fanouts may differ), each with its own launch settings: the top levels
// pinned in shared memory, queries per lane, and whether the levels below
// the pinned ones are read lane by lane through L1 or staged per warp (each
// distinct node of the warp's chunk loaded once into shared memory), plus an
// optional learned leaf predictor.  The settings come from the trees' own
// tuning (bt_autotune) and can be overridden for the whole forest
// (bt_forest_set_launch), or chosen by timing the forest itself on a work
// list (bt_forest_autotune).
//
// A search takes a work list of batches, each naming a tree, a count and an
// offset into flat query/result arrays, and runs all of them in one launch:
// a plan (a one-block kernel, or the host) turns the batch counts into chunk
// offsets (32 or 64 queries per chunk, by tree), then persistent warps take
// chunks in turn and walk each chunk's queries down that chunk's tree level
// by level, writing value and found flag at the queries' positions.  Nothing
// is allocated and nothing is synchronised, so the whole call can be
// captured in a CUDA graph and replayed for every new work list.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "bt_internal.h"
#include "descent.cuh"
#include "forest.h"

struct bt_forest {
    btgb::ForestTree *d_tab;
    std::vector<btgb::ForestTree> h_tab;  // as applied (what d_tab holds)
    std::vector<const bt_tree *> trees;
    std::vector<const bt_model *> models;
    uint32_t count;
    int key_bytes, val_bytes;
    uint32_t warps;        // default warps per block
    uint32_t pin_budget;   // shared-memory bytes for all trees' pinned levels
    uint32_t lane_mode;    // 0: each tree's tuned queries per lane, else that number for all
    uint32_t stage_mode;   // 0: each tree's tuned design, 1: all through L1, 2: all staged
    uint32_t pin_total;    // bytes of the pinned levels actually applied
    uint32_t stage_bytes;  // per warp, 0 when no tree is staged
    int model_set;         // kModelNone (no model), kModelPL (PL models only), kModelMLP (any model)
};

namespace btgb {

// Work-list entries rejected by k_forest (tree out of range, or queries
// beyond the arrays); read and cleared by bt_forest_bad_batches.
__device__ unsigned long long g_bt_bad_batches;

constexpr int kForestStageBytes = 4096;  // per warp, staged trees: 8..64 node blocks per round
constexpr uint32_t kForestSmemList = 64;  // work lists up to this long are read from shared memory
constexpr uint32_t kForestPinMax = 98304;
constexpr int kForestSmemMax = 200 * 1024;

__host__ __device__ inline bool forest_desc_ok(const bt_batch_desc &bd, uint32_t ntrees, uint64_t nq)
{
    return bd.tree < ntrees && bd.offset <= nq && bd.count <= nq - bd.offset;
}

__host__ __device__ inline uint32_t forest_desc_chunks(const bt_batch_desc &bd, uint32_t ntrees, uint64_t nq,
                                                       int lq)
{
    // a rejected entry keeps one chunk so that the kernel sees it and counts it
    if (!forest_desc_ok(bd, ntrees, nq)) return 1u;
    const uint32_t w = 32u * static_cast<uint32_t>(lq);
    return (bd.count + w - 1u) / w;
}

// chunk_start[b] = number of chunks in batches before b (one block).
__global__ void __launch_bounds__(1024) k_forest_plan(const ForestTree *__restrict__ ft, uint32_t ntrees,
                                                      const bt_batch_desc *__restrict__ batches, uint32_t nb,
                                                      uint64_t nq, uint32_t *__restrict__ chunk_start)
{
    __shared__ uint32_t tmp[32];
    uint32_t run = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t base = 0; base < nb; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        uint32_t c = 0;
        if (i < nb) {
            const bt_batch_desc bd = batches[i];
            c = forest_desc_chunks(bd, ntrees, nq, bd.tree < ntrees ? ft[bd.tree].lq : 1);
        }
        // block exclusive scan of c
        uint32_t x = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) tmp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < static_cast<int>(blockDim.x >> 5) ? tmp[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            tmp[lane] = w;
        }
        __syncthreads();
        const uint32_t ex = x - c + (warp > 0 ? tmp[warp - 1] : 0u);
        if (i < nb) chunk_start[i] = run + ex;
        const uint32_t total = tmp[(blockDim.x >> 5) - 1];
        __syncthreads();
        run += total;
    }
    if (threadIdx.x == 0) chunk_start[nb] = run;
}

// Per-lane state of one query of a chunk.
template <typename K>
struct FQuery {
    K key;
    uint64_t pos;
    uint32_t node;
    int start;  // first level this query walks (the leaf level when its learned window proved the leaf)
    bool valid;
};

// The model's leaf for q when its error window proves it (the leaf before
// the window ends below q and the first window leaf whose largest key is
// >= q is the leaf, or q lies above every key); the window's largest keys
// are read through L1 after a prefetch of their lines.
template <typename K, int MODELS>
__device__ __noinline__ bool forest_window(const ModelDev *__restrict__ mdp, K key, uint32_t *leaf)
{
    const ModelDev &md = *mdp;
    const uint32_t L = md.leaves;
    uint32_t hat;
    if constexpr (MODELS == kModelPL)  // every model of the forest piecewise linear
        hat = leaf_from_pred(pl_predict(md.b, md.inv_w, md.slope, md.icpt, md.segments, static_cast<uint64_t>(key)), L);
    else
        hat = model_leaf(md, md.b, md.inv_w, md.slope, md.icpt, md.mlp, static_cast<uint64_t>(key));
    const uint32_t er = __ldg(md.errs + err_range(hat, L));
    const uint32_t lo = hat > er ? hat - er : 0u;
    const uint32_t hi = (static_cast<uint64_t>(hat) + er < L) ? hat + er : L - 1;
    const K *lm = static_cast<const K *>(md.leaf_max);
    const uint32_t first = lo > 0 ? lo - 1 : 0;
    const uintptr_t w0 = reinterpret_cast<uintptr_t>(lm + first) & ~uintptr_t(127);
    const uintptr_t w1 = reinterpret_cast<uintptr_t>(lm + hi + 1);
    if (w1 - w0 <= 4 * 128)
        for (uintptr_t a = w0; a < w1; a += 128) prefetch_l1(reinterpret_cast<const void *>(a));
    const bool low_ok = (lo == 0) || (ld_key(lm + lo - 1) < key);
    uint32_t a = lo, e = hi + 1;  // first j in [lo, hi] with key <= leaf_max[j]
    while (a < e) {
        const uint32_t mid = (a + e) >> 1;
        if (ld_key(lm + mid) < key)
            a = mid + 1;
        else
            e = mid;
    }
    if (a <= hi) {
        *leaf = a;
        return low_ok;
    }
    if (hi == L - 1) {
        *leaf = L - 1;
        return low_ok;
    }
    return false;
}

// One level of the chunk, staged per warp: the distinct nodes of the warp's
// lanes (query u of every lane) are copied into the warp's stage area in
// rounds of as many blocks as fit, and each lane searches its own block.
template <typename K, int M>
__device__ __forceinline__ int forest_staged_rank(const K *lk, uint32_t node, K key, unsigned char *stage,
                                                  uint32_t *list, int lane, bool &eq)
{
    constexpr int kBlk = M * static_cast<int>(sizeof(K));
    constexpr int kSlots = kForestStageBytes / kBlk;
    constexpr int kCh = kBlk / 16;
    int U, slot;
    warp_distinct(node, lane, list, U, slot);
    __syncwarp();
    int r = 0;
    eq = false;
    for (int rb = 0; rb < U; rb += kSlots) {
        const int nu = (U - rb < kSlots) ? U - rb : kSlots;
        for (int i = lane; i < nu * kCh; i += 32) {
            const int u = i / kCh, part = i - u * kCh;
            cp_async16_cg(stage + u * kBlk + part * 16,
                          reinterpret_cast<const unsigned char *>(lk + static_cast<uint64_t>(list[rb + u]) * M) +
                              part * 16);
        }
        cp_async_wait_all();
        __syncwarp();
        if (slot >= rb && slot < rb + nu) {
            const K *blk = reinterpret_cast<const K *>(stage + (slot - rb) * kBlk);
            r = block_rank<K, M>(blk, key);
            eq = (blk[r] == key);
        }
        __syncwarp();
    }
    return r;
}

template <typename V>
__device__ __forceinline__ V ld_value(const V *p)
{
    if constexpr (sizeof(V) == 8)
        return static_cast<V>(__ldcs(reinterpret_cast<const unsigned long long *>(p)));
    else
        return static_cast<V>(__ldcs(reinterpret_cast<const unsigned int *>(p)));
}

// One chunk of a batch: 32 * LQ queries (lane + 32 u for u < LQ) starting at
// query `first` of the batch at q[off ..], walked down tree F level by level.
// Lanes past the batch's end carry the chunk's first query (same nodes, no
// extra traffic) and write nothing.
template <typename K, typename V, int M, int LQ, int MODELS>
__device__ __forceinline__ void forest_chunk(const ForestTree &F, const unsigned char *pin, unsigned char *stage,
                                             uint32_t *list, const K *__restrict__ q, V *__restrict__ out_v,
                                             uint8_t *__restrict__ out_f, uint64_t off, uint32_t first,
                                             uint32_t count, int lane)
{
    const DevTree &t = F.t;
    const int H = t.height;
    FQuery<K> Q[LQ];
    const K k0 = q[off + first];
#pragma unroll
    for (int u = 0; u < LQ; ++u) {
        const uint32_t j = first + static_cast<uint32_t>(u * 32 + lane);
        Q[u].valid = j < count;
        Q[u].pos = off + (Q[u].valid ? j : first);
        Q[u].key = Q[u].valid ? q[Q[u].pos] : k0;
        Q[u].node = 0;
        Q[u].start = 0;
    }
    if (H == 0) {  // empty tree: every query misses
#pragma unroll
        for (int u = 0; u < LQ; ++u)
            if (Q[u].valid) {
                out_v[Q[u].pos] = static_cast<V>(~static_cast<V>(0));
                out_f[Q[u].pos] = 0;
            }
        return;
    }
    if (MODELS != kModelNone && F.md.kind != kModelNone) {
#pragma unroll
        for (int u = 0; u < LQ; ++u) {
            uint32_t leaf = 0;
            if (forest_window<K, MODELS>(&F.md, Q[u].key, &leaf)) {
                Q[u].node = leaf;
                Q[u].start = H - 1;
            }
        }
    }
    const unsigned char *top = static_cast<const unsigned char *>(t.keys[0]);
    const int P = t.pin_levels;
    const bool staged = F.staged != 0;
    constexpr int kLines = (M * static_cast<int>(sizeof(K)) + 127) / 128;
    for (int l = 0; l < H; ++l) {
        const bool leaf = (l == H - 1);
        int r[LQ];
        bool eq[LQ];
        if (l < P) {  // pinned level: the block's shared copy (never the leaf level)
            const K *lk = reinterpret_cast<const K *>(pin + (static_cast<const unsigned char *>(t.keys[l]) - top));
#pragma unroll
            for (int u = 0; u < LQ; ++u) {
                r[u] = 0;
                eq[u] = false;
                if (l >= Q[u].start) r[u] = block_rank<K, M>(lk + static_cast<uint64_t>(Q[u].node) * M, Q[u].key);
            }
        } else if (staged) {  // every lane takes part (staged trees carry no model)
            const K *lk = static_cast<const K *>(t.keys[l]);
#pragma unroll
            for (int u = 0; u < LQ; ++u)
                r[u] = forest_staged_rank<K, M>(lk, Q[u].node, Q[u].key, stage, list, lane, eq[u]);
        } else {  // lane by lane through L1: every line of each block prefetched, then the probes
            const K *lk = static_cast<const K *>(t.keys[l]);
            const K *blk[LQ];
            bool act[LQ];
#pragma unroll
            for (int u = 0; u < LQ; ++u) {
                blk[u] = lk + static_cast<uint64_t>(Q[u].node) * M;
                act[u] = l >= Q[u].start;
                r[u] = 0;
                eq[u] = false;
                if (kLines > 1 && act[u]) {
#pragma unroll
                    for (int i = 0; i < kLines; ++i) prefetch_l1(reinterpret_cast<const unsigned char *>(blk[u]) + 128 * i);
                }
            }
#pragma unroll
            for (int h = M / 2; h >= 1; h >>= 1) {
#pragma unroll
                for (int u = 0; u < LQ; ++u)
                    if (act[u] && ld_key(blk[u] + r[u] + h - 1) < Q[u].key) r[u] += h;
            }
            if (leaf) {
#pragma unroll
                for (int u = 0; u < LQ; ++u) eq[u] = ld_key(blk[u] + r[u]) == Q[u].key;
            }
        }
        if (!leaf) {
#pragma unroll
            for (int u = 0; u < LQ; ++u)
                if (l >= Q[u].start) Q[u].node = child_of(t, l, Q[u].node, r[u]);
        } else {
            const uint64_t cb = t.cbase[l], cr = t.crem[l];
            const V *vals = static_cast<const V *>(t.vals);
#pragma unroll
            for (int u = 0; u < LQ; ++u) {
                const uint64_t cnt = cb + (Q[u].node < cr ? 1u : 0u);
                const bool hit = (static_cast<uint64_t>(r[u]) < cnt) && eq[u];
                V val = static_cast<V>(~static_cast<V>(0));
                if (hit && Q[u].valid) val = ld_value(vals + static_cast<uint64_t>(Q[u].node) * M + r[u]);
                if (Q[u].valid) {
                    out_v[Q[u].pos] = val;
                    out_f[Q[u].pos] = hit ? 1 : 0;
                }
            }
        }
    }
}

template <typename K, typename V, int LQ, int MODELS>
__device__ __forceinline__ void forest_chunk_m(const ForestTree &F, int m, const unsigned char *pin,
                                               unsigned char *stage, uint32_t *list, const K *q, V *out_v,
                                               uint8_t *out_f, uint64_t off, uint32_t first, uint32_t count,
                                               int lane)
{
    switch (m) {
    case 8:
        forest_chunk<K, V, 8, LQ, MODELS>(F, pin, stage, list, q, out_v, out_f, off, first, count, lane);
        break;
    case 16:
        forest_chunk<K, V, 16, LQ, MODELS>(F, pin, stage, list, q, out_v, out_f, off, first, count, lane);
        break;
    case 32:
        forest_chunk<K, V, 32, LQ, MODELS>(F, pin, stage, list, q, out_v, out_f, off, first, count, lane);
        break;
    default:
        forest_chunk<K, V, 64, LQ, MODELS>(F, pin, stage, list, q, out_v, out_f, off, first, count, lane);
        break;
    }
}

// Persistent warps over the chunks of all batches.  Shared memory: the
// pinned levels of trees 0..npin-1 (at their pin_off), then a short work
// list and its chunk offsets (nb <= kForestSmemList), then per warp a stage
// area of stage_bytes and a 32-entry node list.
template <typename K, typename V, int MODELS>
__global__ void __launch_bounds__(512, 2) k_forest(const ForestTree *__restrict__ ft, uint32_t ntrees, uint32_t npin,
                                                uint32_t pin_total, const bt_batch_desc *__restrict__ batches,
                                                uint32_t nb, const uint32_t *__restrict__ chunk_start,
                                                const K *__restrict__ q, uint64_t nq, V *__restrict__ out_v,
                                                uint8_t *__restrict__ out_f, uint32_t stage_bytes, ForestDone done)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool small = nb <= kForestSmemList;
    bt_batch_desc *sb = reinterpret_cast<bt_batch_desc *>(smem + pin_total);
    uint32_t *scs = reinterpret_cast<uint32_t *>(sb + (small ? nb : 0u));
    const uint32_t list_bytes = small ? (nb * 16u + (nb + 1u) * 4u + 15u) & ~15u : 0u;
    unsigned char *stage = smem + pin_total + list_bytes + warp * (stage_bytes + 128u);
    uint32_t *list = reinterpret_cast<uint32_t *>(stage + stage_bytes);
    for (uint32_t i = 0; i < npin; ++i) {
        const uint32_t pb = ft[i].t.pin_bytes;
        if (ft[i].t.pin_levels == 0 || pb == 0) continue;
        const unsigned char *src = static_cast<const unsigned char *>(ft[i].t.keys[0]);
        unsigned char *dst = smem + ft[i].pin_off;
        for (uint32_t o = threadIdx.x * 16u; o < pb; o += blockDim.x * 16u) cp_async16_ca(dst + o, src + o);
    }
    if (small) {
        for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) sb[i] = batches[i];
        for (uint32_t i = threadIdx.x; i <= nb; i += blockDim.x) scs[i] = chunk_start[i];
    }
    cp_async_wait_all();
    __syncthreads();
    const bt_batch_desc *B = small ? sb : batches;
    const uint32_t *CS = small ? scs : chunk_start;
    const uint32_t nchunks = nb ? CS[nb] : 0u;
    for (uint32_t c = blockIdx.x * nw + warp; c < nchunks; c += gridDim.x * nw) {
        // the batch holding chunk c: last b with CS[b] <= c
        uint32_t lo = 0, hi = nb - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (CS[mid] <= c)
                lo = mid;
            else
                hi = mid - 1;
        }
        const bt_batch_desc bd = B[lo];
        // a descriptor naming a tree outside the forest, or queries beyond
        // the arrays, is skipped (nothing written) and counted
        if (!forest_desc_ok(bd, ntrees, nq)) {
            if (lane == 0 && c == CS[lo]) atomicAdd(&g_bt_bad_batches, 1ull);
            continue;
        }
        const ForestTree &F = ft[bd.tree];
        const int lq = F.lq, m = F.t.m;
        const uint32_t first = (c - CS[lo]) * 32u * static_cast<uint32_t>(lq);
        const unsigned char *pin = smem + F.pin_off;
        if (lq == 2)
            forest_chunk_m<K, V, 2, MODELS>(F, m, pin, stage, list, q, out_v, out_f, bd.offset, first, bd.count, lane);
        else
            forest_chunk_m<K, V, 1, MODELS>(F, m, pin, stage, list, q, out_v, out_f, bd.offset, first, bd.count, lane);
    }
    if (done.counter) {
        // every thread's results visible system-wide, then one arrival per block;
        // the last block to arrive resets the counter and raises the flag
        __threadfence_system();
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned prev = atomicAdd(done.counter, 1u);
            if (prev == gridDim.x - 1) {
                *done.counter = 0u;
                __threadfence_system();
                asm volatile("st.release.sys.u64 [%0], %1;" ::"l"(done.flag), "l"(done.seq) : "memory");
            }
        }
    }
}

template <typename K, typename V>
static cudaError_t forest_launch_t(const bt_forest *f, const bt_batch_desc *b, uint32_t nb, const uint32_t *cs,
                                   uint32_t host_chunks, uint32_t *plan_ws, const void *q, uint64_t nq, void *ov, uint8_t *of,
                                   uint32_t warps, cudaStream_t s, ForestDone done)
{
    const int threads = static_cast<int>(warps) * 32;
    const uint32_t list_bytes = nb <= kForestSmemList ? (nb * 16u + (nb + 1u) * 4u + 15u) & ~15u : 0u;
    const int smem = static_cast<int>(f->pin_total + list_bytes + warps * (f->stage_bytes + 128u));
    void (*kern)(const ForestTree *, uint32_t, uint32_t, uint32_t, const bt_batch_desc *, uint32_t, const uint32_t *,
                 const K *, uint64_t, V *, uint8_t *, uint32_t, ForestDone) =
        f->model_set == kModelNone ? k_forest<K, V, kModelNone>
                                   : (f->model_set == kModelPL ? k_forest<K, V, kModelPL> : k_forest<K, V, kModelMLP>);
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(kern), kForestSmemMax);
    int per_sm = 0, sms = 0;
    if (e == cudaSuccess) e = blocks_per_sm(reinterpret_cast<const void *>(kern), threads, smem, &per_sm);
    if (e == cudaSuccess) e = dev_sm_count(&sms);
    if (e != cudaSuccess) return e;
    uint32_t grid = static_cast<uint32_t>(sms * (per_sm > 0 ? per_sm : 1));
    if (cs) {
        // the host planned the list: no more blocks than chunks need
        const uint32_t need = (host_chunks + warps - 1) / warps;
        grid = std::max(1u, std::min(grid, need));
    } else {
        k_forest_plan<<<1, 1024, 0, s>>>(f->d_tab, f->count, b, nb, nq, plan_ws);
        cs = plan_ws;
    }
    uint32_t npin = 0;
    for (uint32_t i = 0; i < f->count; ++i)
        if (f->h_tab[i].t.pin_levels > 0) npin = i + 1;
    kern<<<grid, threads, smem, s>>>(f->d_tab, f->count, npin, f->pin_total, b, nb, cs, static_cast<const K *>(q), nq,
                                     static_cast<V *>(ov), of, f->stage_bytes, done);
    return cudaGetLastError();
}

cudaError_t forest_run(const bt_forest *f, const bt_batch_desc *b, uint32_t nb, const uint32_t *cs,
                       uint32_t host_chunks, uint32_t *plan_ws, const void *q, uint64_t nq, void *ov, uint8_t *of,
                       uint32_t warps, cudaStream_t s, ForestDone done)
{
    if (f->key_bytes == 8) {
        if (f->val_bytes == 8) return forest_launch_t<uint64_t, uint64_t>(f, b, nb, cs, host_chunks, plan_ws, q, nq, ov, of, warps, s, done);
        return forest_launch_t<uint64_t, uint32_t>(f, b, nb, cs, host_chunks, plan_ws, q, nq, ov, of, warps, s, done);
    }
    if (f->val_bytes == 8) return forest_launch_t<uint32_t, uint64_t>(f, b, nb, cs, host_chunks, plan_ws, q, nq, ov, of, warps, s, done);
    return forest_launch_t<uint32_t, uint32_t>(f, b, nb, cs, host_chunks, plan_ws, q, nq, ov, of, warps, s, done);
}

void forest_chunks(const bt_forest *f, const bt_batch_desc *b, uint32_t nb, uint32_t *cs)
{
    uint32_t run = 0;
    for (uint32_t i = 0; i < nb; ++i) {
        cs[i] = run;
        run += forest_desc_chunks(b[i], f->count, ~0ull, b[i].tree < f->count ? f->h_tab[b[i].tree].lq : 1);
    }
    cs[nb] = run;
}

uint32_t forest_default_warps(const bt_forest *f) { return f->warps; }

// The forest's table from its trees, models and settings: each tree's tuned
// queries per lane and staging design unless overridden; its tuned pinned
// levels, trimmed (one level at a time from the tree pinning most) until
// all trees' pinned levels fit the forest's budget.
static void forest_table(bt_forest *f)
{
    const uint32_t n = f->count;
    f->h_tab.assign(n, ForestTree{});
    bool any_staged = false;
    uint64_t total = 0;
    for (uint32_t i = 0; i < n; ++i) {
        ForestTree &e = f->h_tab[i];
        const DevTree &t = f->trees[i]->dev;
        e.t = t;
        e.md = ModelDev{};
        e.md.kind = kModelNone;
        if (f->models[i]) e.md = f->models[i]->dev;
        e.lq = f->lane_mode ? static_cast<int>(f->lane_mode) : (t.lane_queries == 2 ? 2 : 1);
        const bool tuned_staged = t.staging != BT_STAGE_PIPELINED || t.inner_stage == 1;
        e.staged = (f->stage_mode == 0 ? tuned_staged : f->stage_mode == 2) ? 1 : 0;
        if (e.md.kind != kModelNone) e.staged = 0;  // learned lanes walk alone
        any_staged |= e.staged != 0;
        total += e.t.pin_levels > 0 ? e.t.pin_bytes : 0u;
    }
    while (total > f->pin_budget) {
        uint32_t big = 0;
        for (uint32_t i = 1; i < n; ++i)
            if (f->h_tab[i].t.pin_bytes > f->h_tab[big].t.pin_bytes) big = i;
        DevTree &t = f->h_tab[big].t;
        const uint32_t before = t.pin_levels > 0 ? t.pin_bytes : 0u;
        // drop the deepest pinned level
        const int L = t.pin_levels - 1;
        const bt_info &inf = f->trees[big]->info;
        t.pin_levels = L;
        t.pin_bytes = L > 0 ? static_cast<uint32_t>((inf.level_key_offset[L - 1] +
                                                     t.nodes[L - 1] * static_cast<uint64_t>(t.m) * t.key_bytes + 15) /
                                                    16 * 16)
                            : 0u;
        total -= before - t.pin_bytes;
    }
    uint32_t off = 0;
    for (uint32_t i = 0; i < n; ++i) {
        DevTree &t = f->h_tab[i].t;
        if (t.pin_levels == 0) t.pin_bytes = 0;
        f->h_tab[i].pin_off = off;
        off += t.pin_bytes;
    }
    f->pin_total = off;
    f->model_set = kModelNone;
    for (uint32_t i = 0; i < n; ++i) {
        const int k = f->h_tab[i].md.kind;
        if (k == kModelMLP) f->model_set = kModelMLP;
        if (k == kModelPL && f->model_set == kModelNone) f->model_set = kModelPL;
    }
    f->stage_bytes = any_staged ? static_cast<uint32_t>(kForestStageBytes) : 0u;
}

static bt_status forest_upload(bt_forest *f)
{
    forest_table(f);
    cudaError_t e = cudaDeviceSynchronize();  // no search may be reading the old table
    if (e == cudaSuccess)
        e = cudaMemcpy(f->d_tab, f->h_tab.data(), sizeof(ForestTree) * f->count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_error_detail("forest table", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}

}  // namespace btgb

using namespace btgb;

static bt_status forest_create(const bt_tree *const *trees, const bt_model *const *models, uint32_t count,
                               bt_forest **out)
{
    if (!trees || !out || count == 0) return BT_ERR_ARG;
    for (uint32_t i = 0; i < count; ++i) {
        if (!trees[i] || trees[i]->dev.key_bytes == 32 || trees[i]->dev.key_bytes != trees[0]->dev.key_bytes ||
            trees[i]->dev.val_bytes != trees[0]->dev.val_bytes)
            return BT_ERR_ARG;
        if (models && models[i] &&
            (trees[i]->dev.height == 0 || models[i]->dev.leaves != trees[i]->dev.nodes[trees[i]->dev.height - 1]))
            return BT_ERR_ARG;
    }
    bt_forest *f = new (std::nothrow) bt_forest;
    if (!f) return BT_ERR_NOMEM;
    f->d_tab = nullptr;
    f->count = count;
    f->trees.assign(trees, trees + count);
    f->models.assign(count, nullptr);
    if (models) f->models.assign(models, models + count);
    f->key_bytes = trees[0]->dev.key_bytes;
    f->val_bytes = trees[0]->dev.val_bytes;
    // defaults: the launch shape the largest tree was tuned with, each
    // tree's own design, and a pin budget that leaves room for several blocks per SM
    uint32_t big = 0;
    for (uint32_t i = 1; i < count; ++i)
        if (trees[i]->info.n > trees[big]->info.n) big = i;
    f->warps = static_cast<uint32_t>(trees[big]->dev.warps > 0 ? trees[big]->dev.warps : 8);
    f->pin_budget = 32768;
    f->lane_mode = 0;
    f->stage_mode = 0;
    cudaError_t e = cudaMalloc(&f->d_tab, sizeof(ForestTree) * count);
    if (e != cudaSuccess) {
        set_error_detail("forest table", e);
        delete f;
        return e == cudaErrorMemoryAllocation ? BT_ERR_NOMEM : BT_ERR_CUDA;
    }
    const bt_status st = forest_upload(f);
    if (st != BT_OK) {
        cudaFree(f->d_tab);
        delete f;
        return st;
    }
    *out = f;
    return BT_OK;
}

extern "C" bt_status bt_forest_create(const bt_tree *const *trees, uint32_t count, bt_forest **out)
{
    return forest_create(trees, nullptr, count, out);
}

extern "C" bt_status bt_forest_create_learned(const bt_tree *const *trees, const bt_model *const *models,
                                              uint32_t count, bt_forest **out)
{
    if (!models) return BT_ERR_ARG;
    return forest_create(trees, models, count, out);
}

extern "C" void bt_forest_free(bt_forest *f)
{
    if (!f) return;
    cudaFree(f->d_tab);
    delete f;
}

extern "C" uint64_t bt_forest_workspace_bytes(uint32_t nbatches) { return (static_cast<uint64_t>(nbatches) + 1) * 4; }

extern "C" bt_status bt_forest_set_launch(bt_forest *f, const bt_forest_tune *cfg)
{
    if (!f || !cfg || cfg->warps_per_block < 1 || cfg->warps_per_block > 16 || cfg->pin_budget > kForestPinMax ||
        cfg->lane_queries > 2 || cfg->staging > 2)
        return BT_ERR_ARG;
    f->warps = cfg->warps_per_block;
    f->pin_budget = cfg->pin_budget;
    f->lane_mode = cfg->lane_queries;
    f->stage_mode = cfg->staging;
    return forest_upload(f);
}

extern "C" bt_status bt_forest_get_launch(const bt_forest *f, bt_forest_tune *out)
{
    if (!f || !out) return BT_ERR_ARG;
    *out = bt_forest_tune{f->warps, f->pin_budget, f->lane_mode, f->stage_mode, f->pin_total, 0.0f};
    return BT_OK;
}

// Keeps the stream busy for a fixed number of clock cycles (the autotuner's
// timed calls queue behind it).
static __global__ void k_tune_spin(long long cycles)
{
    const long long t0 = clock64();
    while (clock64() - t0 < cycles) {
    }
}

// The work list, queries and values are aligned to their element sizes.
static bool forest_arrays_aligned(const bt_forest *f, const void *d_batches, const void *q, const void *v)
{
    const uintptr_t kb = static_cast<uintptr_t>(f->key_bytes), vb = static_cast<uintptr_t>(f->val_bytes);
    return (reinterpret_cast<uintptr_t>(d_batches) & 7u) == 0 && (reinterpret_cast<uintptr_t>(q) & (kb - 1)) == 0 &&
           (reinterpret_cast<uintptr_t>(v) & (vb - 1)) == 0;
}

extern "C" bt_status bt_forest_search(const bt_forest *f, const bt_batch_desc *d_batches, uint32_t nbatches,
                                      const void *d_queries, uint64_t nq, void *d_out_vals, uint8_t *d_out_found,
                                      void *d_workspace, uint64_t ws_bytes, uint32_t warps_per_block,
                                      bt_stream stream)
{
    if (!f) return BT_ERR_ARG;
    if (nbatches == 0) return BT_OK;
    if (!d_batches || !d_queries || !d_out_vals || !d_out_found) return BT_ERR_ARG;
    if (!forest_arrays_aligned(f, d_batches, d_queries, d_out_vals)) return BT_ERR_ARG;
    if (warps_per_block == 0) warps_per_block = f->warps;
    if (warps_per_block > 16) return BT_ERR_ARG;
    if (!d_workspace || ws_bytes < bt_forest_workspace_bytes(nbatches)) return BT_ERR_WORKSPACE;
    const cudaError_t e = forest_run(f, d_batches, nbatches, nullptr, 0, static_cast<uint32_t *>(d_workspace),
                                     d_queries, nq, d_out_vals, d_out_found, warps_per_block,
                                     reinterpret_cast<cudaStream_t>(stream), ForestDone{nullptr, nullptr, 0});
    if (e != cudaSuccess) {
        set_error_detail("forest search launch", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}

extern "C" bt_status bt_forest_autotune(bt_forest *f, const bt_batch_desc *d_batches, uint32_t nbatches,
                                        const void *d_queries, uint64_t nq, void *d_out_vals, uint8_t *d_out_found,
                                        void *d_workspace, uint64_t ws_bytes, bt_stream stream, bt_forest_tune *best)
{
    if (!f || !best || nbatches == 0 || !d_batches || !d_queries || !d_out_vals || !d_out_found) return BT_ERR_ARG;
    if (!forest_arrays_aligned(f, d_batches, d_queries, d_out_vals)) return BT_ERR_ARG;
    if (!d_workspace || ws_bytes < bt_forest_workspace_bytes(nbatches)) return BT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const uint32_t warps[] = {4, 8, 16};
    const uint32_t pins[] = {0, 16384, 49152, 98304};
    bt_forest_tune b{};
    bool have = false;
    for (uint32_t w : warps)
        for (uint32_t p : pins)
            for (uint32_t lm = 0; lm <= 2 && e == cudaSuccess; ++lm)
                for (uint32_t sm = 0; sm <= 2 && e == cudaSuccess; ++sm) {
                    const bt_forest_tune cfg{w, p, lm, sm, 0, 0.0f};
                    bt_status st = bt_forest_set_launch(f, &cfg);
                    if (st != BT_OK) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return st;
                    }
                    // two warm-up calls, then kReps runs of kCalls calls issued
                    // behind a spin of about 100 us (so that they run back to
                    // back on the device), timed together; median per call
                    constexpr int kCalls = 5, kReps = 3;
                    std::vector<float> ms;
                    for (int r = 0; r < 2 + kReps && e == cudaSuccess; ++r) {
                        const bool timed = r >= 2;
                        if (timed) {
                            k_tune_spin<<<1, 32, 0, s>>>(200000);
                            e = cudaGetLastError();
                            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                        }
                        for (int i = 0; i < (timed ? kCalls : 1) && e == cudaSuccess; ++i) {
                            st = bt_forest_search(f, d_batches, nbatches, d_queries, nq, d_out_vals, d_out_found,
                                                  d_workspace, ws_bytes, 0, stream);
                            if (st != BT_OK) {
                                cudaEventDestroy(e0);
                                cudaEventDestroy(e1);
                                return st;
                            }
                        }
                        if (timed) {
                            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                            float x = 0;
                            if (e == cudaSuccess) e = cudaEventElapsedTime(&x, e0, e1);
                            ms.push_back(x / kCalls);
                        }
                    }
                    if (e != cudaSuccess) break;
                    std::sort(ms.begin(), ms.end());
                    const float us = 1000.0f * ms[ms.size() / 2];
                    if (!have || us < b.us) {
                        b = cfg;
                        b.us = us;
                        have = true;
                    }
                }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        set_error_detail("forest autotune", e);
        return BT_ERR_CUDA;
    }
    const bt_status st = bt_forest_set_launch(f, &b);
    if (st != BT_OK) return st;
    b.pin_applied = f->pin_total;
    *best = b;
    return BT_OK;
}

extern "C" bt_status bt_forest_bad_batches(uint64_t *out)
{
    if (!out) return BT_ERR_ARG;
    unsigned long long v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_bt_bad_batches, sizeof(v));
    if (e == cudaSuccess && v) {
        const unsigned long long zero = 0;
        e = cudaMemcpyToSymbol(g_bt_bad_batches, &zero, sizeof(zero));
    }
    if (e != cudaSuccess) {
        set_error_detail("rejected-batch counter", e);
        return BT_ERR_CUDA;
    }
    *out = v;
    return BT_OK;
}
