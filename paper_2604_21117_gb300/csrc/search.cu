// Batched level-wise B+ tree point search on GB300 (sm_103a).
//
// One search is (Sec. IV-A, IV-F):
//   1. an on-device partition of (query, input position) pairs by a bucket
//      number monotone in the key (part_sort.cuh), so that queries routed
//      to the same node end up adjacent (the paper's sorted batch);
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
#include <cstring>
#include <type_traits>

#include "bt_internal.h"
#include "part_sort.cuh"

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

// ---- bulk asynchronous copies (TMA, non-tensor form) with an mbarrier ----

// Bounded waits that gave up (the results of that search are invalid);
// read and cleared by bt_check_timeouts.
__device__ unsigned int g_bt_timeouts;
constexpr uint32_t kMbarSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// -------------------------------------------- level-wise descent (a3-a5)
//
// Persistent blocks of a tunable number of warps.  Each block first copies the top
// levels of the tree (as many whole levels as fit the tree's pin budget, never
// the leaves) into shared memory once; a warp then loops over chunks of 32
// consecutive queries of the (sorted) batch, prefetching the next chunk's
// queries and output positions while it works on the current one.  Per
// level below the pinned ones, the warp's distinct nodes are staged into
// its shared-memory slots (rounds of `stage_slots` nodes) before the binary
// searches.

constexpr int kDescWarpsDefault = 8;
constexpr int kDescWarpsMax = 16;
constexpr int kPinBudgetMax = 49152;

template <typename K, int M>
constexpr int stage_slots()
{
    return (M * static_cast<int>(sizeof(K)) >= 2048) ? 4 : (M * static_cast<int>(sizeof(K)) >= 512) ? 8 : 16;
}

// Shared memory per warp: its stage slots, its node list and its mbarrier.
template <typename K, int M>
constexpr int desc_smem_per_warp()
{
    return stage_slots<K, M>() * M * static_cast<int>(sizeof(K)) + 32 * 4 + 8;
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

// First child of inner node `node` of level l plus rank r.  32-bit: an
// inner node has at most 64 children and every level has < 2^32 nodes.
__device__ __forceinline__ uint32_t child_of(const DevTree &t, int l, uint32_t node, int r)
{
    const uint32_t base = static_cast<uint32_t>(t.cbase[l]), rem = static_cast<uint32_t>(t.crem[l]);
    return node * base + (node < rem ? node : rem) + static_cast<uint32_t>(r);
}

// Stage nu node blocks of CH 16-byte chunks (block i of `src` array at
// list[i]) into consecutive shared-memory slots with 16-byte asynchronous
// copies: CH lanes per block when CH <= 32 (32 / CH blocks per round), else
// the warp walks each block.  `.cg` (L2 only) for leaves, `.ca` for inner
// levels.  Used by the paper-layout descent (whole nodes).
template <int CH>
__device__ __forceinline__ void stage_blocks(unsigned char *dst, const unsigned char *src, uint32_t blk_bytes,
                                             const uint32_t *list, int nu, int lane, bool leaf)
{
    if constexpr (CH <= 32) {
        constexpr int NPI = 32 / CH;
        const int part = lane % CH;
        for (int u = lane / CH; u < nu; u += NPI) {
            const unsigned char *s = src + static_cast<uint64_t>(list[u]) * blk_bytes + part * 16;
            unsigned char *d = dst + u * blk_bytes + part * 16;
            if (leaf)
                cp_async16_cg(d, s);
            else
                cp_async16_ca(d, s);
        }
    } else {
        for (int u = 0; u < nu; ++u)
            for (int part = lane; part < CH; part += 32) {
                const unsigned char *s = src + static_cast<uint64_t>(list[u]) * blk_bytes + part * 16;
                unsigned char *d = dst + u * blk_bytes + part * 16;
                if (leaf)
                    cp_async16_cg(d, s);
                else
                    cp_async16_ca(d, s);
            }
    }
}

// Leaf-max entries a warp can stage for its model windows.
constexpr int kLeafMaxCap = 128;
// PL models with at most this many segments are copied to shared memory.
constexpr uint32_t kModelSmemSegments = 512;

__host__ __device__ inline uint32_t model_smem_bytes(const ModelDev &m)
{
    if (m.kind == kModelPL) return m.segments <= kModelSmemSegments ? (m.segments * 20u + 15u) / 16u * 16u : 0u;
    if (m.kind == kModelMLP) return (kMlpParams * 4u + 15u) / 16u * 16u;
    return 0u;
}

template <typename K, typename V, int M, bool COUNT, bool LEARN>
__global__ void __launch_bounds__(kDescWarpsMax * 32) k_descend(
    const DevTree t, const RawOf<K> *__restrict__ q, const uint32_t *__restrict__ qidx, uint64_t nq,
    V *__restrict__ out_v, uint8_t *__restrict__ out_f, unsigned long long *__restrict__ fetch,
    const ModelDev md, unsigned long long *__restrict__ lstats)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int CH = M * static_cast<int>(sizeof(K)) / 16;  // 16-byte chunks per node block
    constexpr int SLOTS = stage_slots<K, M>();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t pin_bytes = t.pin_bytes;
    const uint32_t mbytes = LEARN ? model_smem_bytes(md) : 0u;
    unsigned char *pin = smem;
    unsigned char *msm = smem + pin_bytes;
    K *stage = reinterpret_cast<K *>(msm + mbytes) + warp * SLOTS * M;
    const int nw = blockDim.x >> 5;
    unsigned char *after_stage = msm + mbytes + nw * SLOTS * M * sizeof(K);
    uint32_t *list = reinterpret_cast<uint32_t *>(after_stage) + warp * 32;
    K *lmstage = reinterpret_cast<K *>(after_stage + nw * 32 * 4) + warp * kLeafMaxCap;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(after_stage + nw * 32 * 4 +
                                                  (LEARN ? nw * kLeafMaxCap * sizeof(K) : 0)) + warp;
    const bool tma = (t.staging == 1);  // stage node blocks with bulk copies (else 16-byte cp.async)
    uint32_t phase = 0;
    if (tma && lane == 0) mbar_init(mbar);
    __syncwarp();

    // Top levels, pinned once per block.
    const unsigned char *top = static_cast<const unsigned char *>(t.keys[0]);
    for (uint32_t i = threadIdx.x * 16u; i < pin_bytes; i += blockDim.x * 16u) cp_async16_ca(pin + i, top + i);
    // The model's parameters, copied once per block when they fit.
    const uint64_t *mb = md.b;
    const float *minv = md.inv_w, *mslope = md.slope, *micpt = md.icpt, *mmlp = md.mlp;
    if constexpr (LEARN) {
      if (mbytes) {
        if (md.kind == kModelPL) {
            const uint32_t S = md.segments;
            uint64_t *sb = reinterpret_cast<uint64_t *>(msm);
            float *sf = reinterpret_cast<float *>(msm + S * 8u);
            for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) {
                sb[i] = md.b[i];
                sf[i] = md.inv_w[i];
                sf[S + i] = md.slope[i];
                sf[2 * S + i] = md.icpt[i];
            }
            mb = sb;
            minv = sf;
            mslope = sf + S;
            micpt = sf + 2 * S;
        } else {
            float *sp = reinterpret_cast<float *>(msm);
            for (uint32_t i = threadIdx.x; i < static_cast<uint32_t>(kMlpParams); i += blockDim.x) sp[i] = md.mlp[i];
            mmlp = sp;
        }
      }
    }
    cp_async_wait_all();
    __syncthreads();

    const uint64_t nchunks = (nq + 31) / 32;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * nw;
    const int H = t.height, P = t.pin_levels;
    uint64_t c = static_cast<uint64_t>(blockIdx.x) * nw + warp;
    if (c >= nchunks) return;

    // Tail lanes follow lane 0's query so they never add a node fetch.
    K key_n;
    uint32_t dst_n;
    {
        const uint64_t pos = c * 32 + lane;
        const bool v = pos < nq;
        key_n = KeyOps<K>::load(q, v ? pos : c * 32);
        dst_n = v ? (qidx ? qidx[pos] : static_cast<uint32_t>(pos)) : 0u;
    }
    // The previous chunk's result: its value load is issued at its leaf
    // level and consumed (stored) only after this chunk's first staged level,
    // so the load's latency overlaps the next descent.
    V pend_val = 0;
    uint32_t pend_dst = 0;
    bool pend_store = false, pend_hit = false;
    for (;;) {
        const uint64_t pos = c * 32 + lane;
        const bool valid = pos < nq;
        const K key = key_n;
        const uint32_t dst = dst_n;
        const uint64_t cn = c + stride;
        if (cn < nchunks) {  // prefetch the next chunk
            const uint64_t pn = cn * 32 + lane;
            const bool vn = pn < nq;
            key_n = KeyOps<K>::load(q, vn ? pn : cn * 32);
            dst_n = vn ? (qidx ? qidx[pn] : static_cast<uint32_t>(pn)) : 0u;
        }

        uint32_t node = 0;
        int l = 0;
        if constexpr (LEARN) {
            // Predicted leaf and its error window; the warp stages the leaf
            // maxima covering all its windows (plus the leaf below) and every
            // lane proves its leaf: the first window leaf whose largest key
            // is >= the query, with the leaf below the window ending below
            // the query.  One unproven lane sends the warp down the tree.
            const uint32_t L = md.leaves;
            const uint32_t hat = model_leaf(md, mb, minv, mslope, micpt, mmlp, static_cast<uint64_t>(key));
            const uint32_t er = __ldg(md.errs + err_range(hat, L));  // bound of this prediction's range
            const uint32_t lo = hat > er ? hat - er : 0u;
            const uint32_t hi = (static_cast<uint64_t>(hat) + er < L) ? hat + er : L - 1;
            uint32_t wlo = __reduce_min_sync(0xffffffffu, lo);
            if (wlo > 0) --wlo;
            const uint32_t whi = __reduce_max_sync(0xffffffffu, hi);
            bool ok = false;
            uint32_t leaf = 0;
            if (whi - wlo < static_cast<uint32_t>(kLeafMaxCap)) {
                const K *lm = static_cast<const K *>(md.leaf_max);
                for (uint32_t j = lane; j <= whi - wlo; j += 32) lmstage[j] = lm[wlo + j];
                __syncwarp();
                const bool low_ok = (lo == 0) || (key > lmstage[lo - 1 - wlo]);
                uint32_t a = lo, e = hi + 1;  // first j in [lo, hi] with key <= leaf_max[j]
                while (a < e) {
                    const uint32_t mid = (a + e) >> 1;
                    if (lmstage[mid - wlo] < key)
                        a = mid + 1;
                    else
                        e = mid;
                }
                if (a <= hi) {
                    leaf = a;
                    ok = low_ok;
                } else if (hi == L - 1) {  // above every key: the last leaf
                    leaf = L - 1;
                    ok = low_ok;
                }
                __syncwarp();
            }
            const bool all_ok = __all_sync(0xffffffffu, ok);
            if (lstats && lane == 0) atomicAdd(lstats + (all_ok ? 0 : 1), 1ull);
            if (all_ok) {
                node = leaf;
                l = H - 1;
            }
        }
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
                if (tma) {
                    // one bulk copy per node block, completion counted in bytes
                    // on the warp's mbarrier; the wait is bounded
                    constexpr unsigned kBlk = M * sizeof(K);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    if (lane == 0) mbar_arrive_expect_tx(mbar, static_cast<unsigned>(nu) * kBlk);
                    __syncwarp();
                    if (lane < nu)
                        bulk_g2s(stage + lane * M, lk + static_cast<uint64_t>(list[rb + lane]) * M, kBlk, mbar);
                    bool gave_up = false;
                    for (uint32_t spins = 0; !mbar_try_wait(mbar, phase);)
                        if (++spins > kMbarSpinLimit) {
                            gave_up = true;
                            break;
                        }
                    if (__any_sync(0xffffffffu, gave_up)) {
                        // record it, give the copies in flight a second bounded
                        // wait to land, and leave: this warp's results are invalid
                        if (lane == 0) atomicAdd(&g_bt_timeouts, 1u);
                        for (uint32_t spins = 0; spins < kMbarSpinLimit && !mbar_try_wait(mbar, phase); ++spins) {
                        }
                        return;
                    }
                    phase ^= 1u;
                } else {
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
                }
                __syncwarp();
                if (slot >= rb && slot < rb + nu) {
                    const K *blk = stage + (slot - rb) * M;
                    r = block_rank<K, M>(blk, key);
                    eq = (blk[r] == key);
                }
                __syncwarp();
            }
            if (pend_store) {  // previous chunk's result, after this chunk's first staged level
                out_v[pend_dst] = pend_val;
                out_f[pend_dst] = pend_hit ? 1 : 0;
                pend_store = false;
            }
            if (!last) {
                node = child_of(t, l, node, r);
            } else {
                const uint64_t cnt = t.cbase[l] + (node < t.crem[l] ? 1u : 0u);
                const bool hit = (static_cast<uint64_t>(r) < cnt) && eq;
                pend_val = static_cast<V>(~static_cast<V>(0));
                if (hit) pend_val = static_cast<const V *>(t.vals)[static_cast<uint64_t>(node) * M + r];
                pend_hit = hit;
                pend_dst = dst;
                pend_store = valid;
            }
        }
        if (cn >= nchunks) break;
        c = cn;
    }
    if (pend_store) {
        out_v[pend_dst] = pend_val;
        out_f[pend_dst] = pend_hit ? 1 : 0;
    }
}

// ------------------------------- two queries per lane (64-query chunks)
//
// The same level-wise descent with each warp taking 64 consecutive queries
// of the batch (lane l holds queries l and 32 + l): every per-level warp
// step -- finding the distinct nodes, staging them, the synchronisations --
// is shared by twice as many queries, and each lane runs two independent
// binary searches.  Selected per tree with bt_tree_set_lane_queries.

// Distinct node ids among the warp's 64 (a, b) pairs, as warp_distinct.  A
// node range wider than 32 lists the distinct a's, then the distinct b's
// (a node in both sets is then listed, and staged, twice).
__device__ __forceinline__ void warp_distinct2(uint32_t a, uint32_t b, int lane, uint32_t *list, int &U, int &sa,
                                               int &sb)
{
    const uint32_t nmin = __reduce_min_sync(0xffffffffu, a < b ? a : b);
    const uint32_t nmax = __reduce_max_sync(0xffffffffu, a < b ? b : a);
    if (nmax - nmin < 32u) {
        const unsigned ba = 1u << (a - nmin), bb = 1u << (b - nmin);
        const unsigned mask = __reduce_or_sync(0xffffffffu, ba | bb);
        U = __popc(mask);
        sa = __popc(mask & (ba - 1u));
        sb = __popc(mask & (bb - 1u));
        if ((mask >> lane) & 1u) list[__popc(mask & ((1u << lane) - 1u))] = nmin + lane;
    } else {
        const unsigned same_a = __match_any_sync(0xffffffffu, a);
        const unsigned same_b = __match_any_sync(0xffffffffu, b);
        const int lead_a = __ffs(same_a) - 1, lead_b = __ffs(same_b) - 1;
        const unsigned leaders_a = __ballot_sync(0xffffffffu, lane == lead_a);
        const unsigned leaders_b = __ballot_sync(0xffffffffu, lane == lead_b);
        const int ua = __popc(leaders_a);
        U = ua + __popc(leaders_b);
        sa = __popc(leaders_a & ((1u << lead_a) - 1u));
        sb = ua + __popc(leaders_b & ((1u << lead_b) - 1u));
        if (lane == lead_a) list[sa] = a;
        if (lane == lead_b) list[sb] = b;
    }
}

template <typename K, int M>
constexpr int desc2_smem_per_warp()
{
    return stage_slots<K, M>() * M * static_cast<int>(sizeof(K)) + 64 * 4;
}

template <typename K, typename V, int M, bool COUNT>
__global__ void __launch_bounds__(kDescWarpsMax * 32) k_descend2(
    const DevTree t, const RawOf<K> *__restrict__ q, const uint32_t *__restrict__ qidx, uint64_t nq,
    V *__restrict__ out_v, uint8_t *__restrict__ out_f, unsigned long long *__restrict__ fetch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int CH = M * static_cast<int>(sizeof(K)) / 16;
    constexpr int SLOTS = stage_slots<K, M>();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t pin_bytes = t.pin_bytes;
    unsigned char *pin = smem;
    K *stage = reinterpret_cast<K *>(smem + pin_bytes) + warp * SLOTS * M;
    uint32_t *list =
        reinterpret_cast<uint32_t *>(smem + pin_bytes + static_cast<uint32_t>(nw) * SLOTS * M * sizeof(K)) + warp * 64;
    const unsigned char *top = static_cast<const unsigned char *>(t.keys[0]);
    for (uint32_t i = threadIdx.x * 16u; i < pin_bytes; i += blockDim.x * 16u) cp_async16_ca(pin + i, top + i);
    cp_async_wait_all();
    __syncthreads();

    const uint64_t nchunks = (nq + 63) / 64;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * nw;
    const int H = t.height, P = t.pin_levels;
    for (uint64_t c = static_cast<uint64_t>(blockIdx.x) * nw + warp; c < nchunks; c += stride) {
        // tail lanes follow the chunk's first query so they never add a node fetch
        const uint64_t pa = c * 64 + lane, pb = pa + 32;
        const bool va = pa < nq, vb = pb < nq;
        const K ka = KeyOps<K>::load(q, va ? pa : c * 64);
        const K kb = KeyOps<K>::load(q, vb ? pb : c * 64);
        const uint32_t da = va ? (qidx ? qidx[pa] : static_cast<uint32_t>(pa)) : 0u;
        const uint32_t db = vb ? (qidx ? qidx[pb] : static_cast<uint32_t>(pb)) : 0u;
        uint32_t na = 0, nb = 0;
        int l = 0;
        for (; l < P; ++l) {
            if (COUNT) {
                int U, sa, sb;
                warp_distinct2(na, nb, lane, list, U, sa, sb);
                __syncwarp();
                if (lane == 0) atomicAdd(fetch + l, static_cast<unsigned long long>(U));
            }
            const K *lvl = reinterpret_cast<const K *>(pin + (static_cast<const unsigned char *>(t.keys[l]) - top));
            const int r_a = block_rank<K, M>(lvl + static_cast<uint64_t>(na) * M, ka);
            const int r_b = block_rank<K, M>(lvl + static_cast<uint64_t>(nb) * M, kb);
            na = child_of(t, l, na, r_a);
            nb = child_of(t, l, nb, r_b);
        }
        for (; l < H; ++l) {
            const K *lk = static_cast<const K *>(t.keys[l]);
            const bool last = (l + 1 == H);
            int U, sa, sb;
            warp_distinct2(na, nb, lane, list, U, sa, sb);
            if (COUNT && lane == 0) atomicAdd(fetch + l, static_cast<unsigned long long>(U));
            __syncwarp();
            int r_a = 0, r_b = 0;
            bool e_a = false, e_b = false;
            for (int rb = 0; rb < U; rb += SLOTS) {
                const int nu = (U - rb < SLOTS) ? U - rb : SLOTS;
                for (int i = lane; i < nu * CH; i += 32) {
                    const int u = i / CH, part = i - u * CH;
                    const unsigned char *src =
                        reinterpret_cast<const unsigned char *>(lk + static_cast<uint64_t>(list[rb + u]) * M) + part * 16;
                    unsigned char *dp = reinterpret_cast<unsigned char *>(stage + u * M) + part * 16;
                    if (last)
                        cp_async16_cg(dp, src);
                    else
                        cp_async16_ca(dp, src);
                }
                cp_async_wait_all();
                __syncwarp();
                if (sa >= rb && sa < rb + nu) {
                    const K *blk = stage + (sa - rb) * M;
                    r_a = block_rank<K, M>(blk, ka);
                    e_a = (blk[r_a] == ka);
                }
                if (sb >= rb && sb < rb + nu) {
                    const K *blk = stage + (sb - rb) * M;
                    r_b = block_rank<K, M>(blk, kb);
                    e_b = (blk[r_b] == kb);
                }
                __syncwarp();
            }
            if (!last) {
                na = child_of(t, l, na, r_a);
                nb = child_of(t, l, nb, r_b);
            } else {
                const V *vals = static_cast<const V *>(t.vals);
                const bool hit_a = (static_cast<uint64_t>(r_a) < t.cbase[l] + (na < t.crem[l] ? 1u : 0u)) && e_a;
                const bool hit_b = (static_cast<uint64_t>(r_b) < t.cbase[l] + (nb < t.crem[l] ? 1u : 0u)) && e_b;
                const V v_a = hit_a ? vals[static_cast<uint64_t>(na) * M + r_a] : static_cast<V>(~static_cast<V>(0));
                const V v_b = hit_b ? vals[static_cast<uint64_t>(nb) * M + r_b] : static_cast<V>(~static_cast<V>(0));
                if (va) {
                    out_v[da] = v_a;
                    out_f[da] = hit_a ? 1 : 0;
                }
                if (vb) {
                    out_v[db] = v_b;
                    out_f[db] = hit_b ? 1 : 0;
                }
            }
        }
    }
}

// ---------------------------------------- the paper's node layout (Eq. 1)
//
// The same level-wise descent over the array-of-nodes layout of Eq. 1: the
// warp's distinct nodes (by node ordinal = byte address / node size) are
// staged whole -- header, keys and child addresses or data -- and each lane
// follows the child address of its rank, or at a leaf reads the data slot
// of its rank from the staged node.  Top levels (a prefix of the array) are
// pinned in shared memory as in k_descend.

template <typename K, int M>
struct PaperGeom {
    static constexpr uint32_t keys = (static_cast<uint32_t>((M - 1) * sizeof(K)) + 7u) / 8u * 8u;
    static constexpr uint32_t bytes = (32u + keys + 8u * M + 31u) / 32u * 32u;
    static constexpr int slots = bytes >= 2048 ? 2 : (bytes >= 1024 ? 4 : 8);
};

template <typename K, int M>
constexpr int paper_smem_per_warp()
{
    return PaperGeom<K, M>::slots * static_cast<int>(PaperGeom<K, M>::bytes) + 32 * 4;
}

template <typename K, typename V, int M>
__global__ void __launch_bounds__(kDescWarpsMax * 32) k_descend_paper(
    const PaperTree p, const RawOf<K> *__restrict__ q, const uint32_t *__restrict__ qidx, uint64_t nq,
    V *__restrict__ out_v, uint8_t *__restrict__ out_f)
{
    extern __shared__ __align__(16) unsigned char smem[];
    using G = PaperGeom<K, M>;
    constexpr uint32_t NB = G::bytes;
    constexpr int SLOTS = G::slots;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned char *pin = smem;
    unsigned char *stage = smem + p.pin_bytes + warp * (SLOTS * NB);
    uint32_t *list = reinterpret_cast<uint32_t *>(smem + p.pin_bytes + nw * (SLOTS * NB)) + warp * 32;
    for (uint32_t i = threadIdx.x * 16u; i < p.pin_bytes; i += blockDim.x * 16u) cp_async16_ca(pin + i, p.base + i);
    cp_async_wait_all();
    __syncthreads();

    const uint64_t nchunks = (nq + 31) / 32;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * nw;
    const int H = p.height, P = p.pin_levels;
    for (uint64_t c = static_cast<uint64_t>(blockIdx.x) * nw + warp; c < nchunks; c += stride) {
        const uint64_t pos = c * 32 + lane;
        const bool valid = pos < nq;
        // tail lanes follow lane 0's query so they never add a node fetch
        const K key = KeyOps<K>::load(q, valid ? pos : c * 32);
        const uint32_t dst = valid ? (qidx ? qidx[pos] : static_cast<uint32_t>(pos)) : 0u;
        uint64_t addr = 0;  // the root is the first node
        int l = 0;
        for (; l < P; ++l) {
            const unsigned char *node = pin + addr;
            const int r = block_rank<K, M>(reinterpret_cast<const K *>(node + 32), key);
            addr = *reinterpret_cast<const uint64_t *>(node + p.child_off + 8u * r);
        }
        for (; l < H; ++l) {
            const uint32_t ord = static_cast<uint32_t>(addr / NB);
            int U, slot;
            warp_distinct(ord, lane, list, U, slot);
            __syncwarp();
            uint64_t next = 0;
            bool hit = false;
            V val = static_cast<V>(~static_cast<V>(0));
            for (int rb = 0; rb < U; rb += SLOTS) {
                const int nu = (U - rb < SLOTS) ? U - rb : SLOTS;
                stage_blocks<NB / 16>(stage, p.base, NB, list + rb, nu, lane, true);
                cp_async_wait_all();
                __syncwarp();
                if (slot >= rb && slot < rb + nu) {
                    const unsigned char *node = stage + (slot - rb) * NB;
                    const K *keys = reinterpret_cast<const K *>(node + 32);
                    const int r = block_rank<K, M>(keys, key);
                    if (l + 1 < H) {
                        next = *reinterpret_cast<const uint64_t *>(node + p.child_off + 8u * r);
                    } else {
                        const uint32_t use = *reinterpret_cast<const uint32_t *>(node);
                        hit = (static_cast<uint32_t>(r) < use) && (keys[r] == key);
                        if (hit) val = static_cast<V>(*reinterpret_cast<const uint64_t *>(node + p.child_off + 8u * r));
                    }
                }
                __syncwarp();
            }
            if (l + 1 < H) {
                addr = next;
            } else if (valid) {
                out_v[dst] = val;
                out_f[dst] = hit ? 1 : 0;
            }
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

struct WsLayout {
    uint64_t qb, ib, counts, total;
};

// Bucket totals of the partition: at most 2^kMaxPartBits buckets, plus
// the ticket word, rounded to whole 16-byte groups.
constexpr uint64_t kPartCountWords = (1ull << kMaxPartBits) + 4;

// Workspace: the partitioned batch (queries, then input positions) and the
// partition's bucket counters.
static WsLayout ws_layout(int kb, uint64_t nq)
{
    WsLayout w;
    uint64_t o = 0;
    w.qb = o;
    o = align256(o + nq * kb);
    w.ib = o;
    o = align256(o + nq * 4);
    w.counts = o;
    o = align256(o + kPartCountWords * 4);
    w.total = nq ? o : 0;
    return w;
}

static int bitlen(uint64_t x) { return x ? 64 - __builtin_clzll(x) : 0; }

// Queries per batch from which the sort pays for itself by node reuse.
constexpr uint64_t kAutoSortMinBatch = 16384;
// Automatic bucket bits: about 16 queries per bucket, so that a warp's 32
// consecutive queries span about two buckets.
static int auto_part_bits(uint64_t nq)
{
    const int b = bitlen(nq) - 5;
    return b < 1 ? 1 : (b > kMaxPartBits ? kMaxPartBits : b);
}

// One search's descent launch: everything a kernel instantiation needs.
struct DescendArgs {
    const DevTree *t;
    const void *q;
    const uint32_t *qidx;
    uint64_t nq;
    void *out_v;
    uint8_t *out_f;
    unsigned long long *fetch;
    const ModelDev *md;  // non-null: learned descent
    unsigned long long *lstats;
};

template <typename K, typename V, int M, bool COUNT, bool LEARN>
static cudaError_t launch_descend(const DescendArgs &a, cudaStream_t s)
{
    const int nw = a.t->warps > 0 ? a.t->warps : kDescWarpsDefault;
    const int fixed = nw * desc_smem_per_warp<K, M>();
    const int learn_fixed = LEARN ? nw * kLeafMaxCap * static_cast<int>(sizeof(K)) : 0;
    constexpr int max_model = LEARN ? static_cast<int>(kModelSmemSegments) * 20 : 0;
    const int threads = nw * 32;
    auto kern = k_descend<K, V, M, COUNT, LEARN>;
    static const cudaError_t attr = cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
        kDescWarpsMax * (desc_smem_per_warp<K, M>() + (LEARN ? kLeafMaxCap * static_cast<int>(sizeof(K)) : 0)) +
            kPinBudgetMax + max_model);
    if (attr != cudaSuccess) return attr;
    ModelDev none;
    memset(&none, 0, sizeof(none));
    const ModelDev &md = a.md ? *a.md : none;
    const int smem = fixed + learn_fixed + static_cast<int>(a.t->pin_bytes) +
                     static_cast<int>(LEARN ? model_smem_bytes(md) : 0u);
    // resident blocks per SM for this block size and shared-memory size
    // (cached per warp count and 256 bytes of shared memory)
    constexpr int kCache = (kPinBudgetMax + max_model) / 256 + 2;
    static int occ_cache[kDescWarpsMax + 1][kCache] = {{0}};
    const int key = (smem - fixed - learn_fixed + 255) / 256;
    if (occ_cache[nw][key] == 0) {
        int b = 0;
        cudaError_t e =
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, fixed + learn_fixed + key * 256);
        if (e != cudaSuccess) return e;
        occ_cache[nw][key] = b > 0 ? b : 1;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const uint64_t chunks = (a.nq + 31) / 32;
    uint64_t grid = (chunks + nw - 1) / nw;
    const uint64_t cap = static_cast<uint64_t>(sms) * occ_cache[nw][key];
    if (grid > cap) grid = cap;
    kern<<<static_cast<unsigned>(grid), threads, smem, s>>>(*a.t, static_cast<const RawOf<K> *>(a.q), a.qidx, a.nq,
                                                           static_cast<V *>(a.out_v), a.out_f, a.fetch, md,
                                                           a.lstats);
    return cudaGetLastError();
}

template <typename K, typename V, int M, bool COUNT>
static cudaError_t launch_descend2(const DescendArgs &a, cudaStream_t s)
{
    const int nw = a.t->warps > 0 ? a.t->warps : kDescWarpsDefault;
    auto kern = k_descend2<K, V, M, COUNT>;
    const int smem = static_cast<int>(a.t->pin_bytes) + nw * desc2_smem_per_warp<K, M>();
    static const cudaError_t attr = cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kPinBudgetMax + kDescWarpsMax * desc2_smem_per_warp<K, M>());
    if (attr != cudaSuccess) return attr;
    constexpr int kCache = kPinBudgetMax / 256 + 2;
    static int occ_cache[kDescWarpsMax + 1][kCache] = {{0}};
    const int key = (static_cast<int>(a.t->pin_bytes) + 255) / 256;
    if (occ_cache[nw][key] == 0) {
        int b = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, nw * 32,
                                                                      key * 256 + nw * desc2_smem_per_warp<K, M>());
        if (e != cudaSuccess) return e;
        occ_cache[nw][key] = b > 0 ? b : 1;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    uint64_t grid = ((a.nq + 63) / 64 + nw - 1) / nw;
    const uint64_t cap = static_cast<uint64_t>(sms) * occ_cache[nw][key];
    if (grid > cap) grid = cap;
    kern<<<static_cast<unsigned>(grid), nw * 32, smem, s>>>(*a.t, static_cast<const RawOf<K> *>(a.q), a.qidx, a.nq,
                                                          static_cast<V *>(a.out_v), a.out_f, a.fetch);
    return cudaGetLastError();
}

template <typename K, typename V, int M>
static cudaError_t dispatch_mode(const DescendArgs &a, cudaStream_t s)
{
    if constexpr (!std::is_same<K, Key32>::value) {
        if (a.md) return launch_descend<K, V, M, false, true>(a, s);
    }
    if (a.t->lane_queries == 2) {
        if (a.fetch) return launch_descend2<K, V, M, true>(a, s);
        return launch_descend2<K, V, M, false>(a, s);
    }
    if (a.fetch) return launch_descend<K, V, M, true, false>(a, s);
    return launch_descend<K, V, M, false, false>(a, s);
}

template <typename K, typename V>
static cudaError_t dispatch_m(const DescendArgs &a, cudaStream_t s)
{
    switch (a.t->m) {
    case 8: return dispatch_mode<K, V, 8>(a, s);
    case 16: return dispatch_mode<K, V, 16>(a, s);
    case 32: return dispatch_mode<K, V, 32>(a, s);
    default: return dispatch_mode<K, V, 64>(a, s);
    }
}

static cudaError_t descend_any(const DescendArgs &a, cudaStream_t s)
{
    if (a.t->key_bytes == 8) {
        if (a.t->val_bytes == 8) return dispatch_m<uint64_t, uint64_t>(a, s);
        return dispatch_m<uint64_t, uint32_t>(a, s);
    }
    if (a.t->key_bytes == 32) {
        if (a.t->val_bytes == 8) return dispatch_m<Key32, uint64_t>(a, s);
        return dispatch_m<Key32, uint32_t>(a, s);
    }
    if (a.t->val_bytes == 8) return dispatch_m<uint32_t, uint64_t>(a, s);
    return dispatch_m<uint32_t, uint32_t>(a, s);
}

static cudaError_t descend(const DevTree &t, const void *q, const uint32_t *qidx, uint64_t nq,
                           void *out_v, uint8_t *out_f, unsigned long long *fetch, cudaStream_t s)
{
    const DescendArgs a{&t, q, qidx, nq, out_v, out_f, fetch, nullptr, nullptr};
    return descend_any(a, s);
}

template <typename K, typename V, int M>
static cudaError_t launch_paper(const PaperTree &p, const void *q, const uint32_t *qidx, uint64_t nq, void *out_v,
                                uint8_t *out_f, int nw, cudaStream_t s)
{
    auto kern = k_descend_paper<K, V, M>;
    const int smem = static_cast<int>(p.pin_bytes) + nw * paper_smem_per_warp<K, M>();
    static const cudaError_t attr = cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 + kDescWarpsMax * paper_smem_per_warp<K, M>());
    if (attr != cudaSuccess) return attr;
    int b = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, nw * 32, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    uint64_t grid = ((nq + 31) / 32 + nw - 1) / nw;
    const uint64_t cap = static_cast<uint64_t>(sms) * (b > 0 ? b : 1);
    if (grid > cap) grid = cap;
    kern<<<static_cast<unsigned>(grid), nw * 32, smem, s>>>(p, static_cast<const RawOf<K> *>(q), qidx, nq,
                                                          static_cast<V *>(out_v), out_f);
    return cudaGetLastError();
}

template <typename K, typename V>
static cudaError_t paper_m(const DevTree &t, const PaperTree &p, const void *q, const uint32_t *qidx, uint64_t nq,
                           void *out_v, uint8_t *out_f, cudaStream_t s)
{
    const int nw = t.warps > 0 ? t.warps : kDescWarpsDefault;
    switch (t.m) {
    case 8: return launch_paper<K, V, 8>(p, q, qidx, nq, out_v, out_f, nw, s);
    case 16: return launch_paper<K, V, 16>(p, q, qidx, nq, out_v, out_f, nw, s);
    case 32: return launch_paper<K, V, 32>(p, q, qidx, nq, out_v, out_f, nw, s);
    default: return launch_paper<K, V, 64>(p, q, qidx, nq, out_v, out_f, nw, s);
    }
}

static cudaError_t descend_paper(const DevTree &t, const PaperTree &p, const void *q, const uint32_t *qidx,
                                 uint64_t nq, void *out_v, uint8_t *out_f, cudaStream_t s)
{
    if (t.key_bytes == 32)
        return t.val_bytes == 8 ? paper_m<Key32, uint64_t>(t, p, q, qidx, nq, out_v, out_f, s)
                                : paper_m<Key32, uint32_t>(t, p, q, qidx, nq, out_v, out_f, s);
    if (t.key_bytes == 8)
        return t.val_bytes == 8 ? paper_m<uint64_t, uint64_t>(t, p, q, qidx, nq, out_v, out_f, s)
                                : paper_m<uint64_t, uint32_t>(t, p, q, qidx, nq, out_v, out_f, s);
    return t.val_bytes == 8 ? paper_m<uint32_t, uint64_t>(t, p, q, qidx, nq, out_v, out_f, s)
                            : paper_m<uint32_t, uint32_t>(t, p, q, qidx, nq, out_v, out_f, s);
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
// below the query) and the interpolation bits r make a bucket of `bits` bits.
struct PartPlan {
    int bits;       // 0: no partition
    int r;          // interpolation bits inside a splitter segment
    int cshift;     // right shift of c when bits < the splitter bits
    uint32_t nb;    // buckets, rounded up to a multiple of 4
};

// sort_bits < 0: auto_part_bits for batches of at least kAutoSortMinBatch
// queries, else none; sort_bits > 0: that many bits, at most kMaxPartBits.
static PartPlan plan_partition(const DevTree &t, int32_t sort_bits, uint64_t nq)
{
    PartPlan p{0, 0, 0, 0};
    int bits = sort_bits;
    if (bits < 0) bits = (nq >= kAutoSortMinBatch) ? auto_part_bits(nq) : 0;
    if (bits > kMaxPartBits) bits = kMaxPartBits;
    if (bits <= 0 || t.height == 0) return p;
    const int cbits = bitlen(t.nsplit);  // c is in [0, nsplit]
    p.bits = bits;
    p.r = bits > cbits ? bits - cbits : 0;
    p.cshift = cbits > bits ? cbits - bits : 0;
    const uint64_t nb = ((static_cast<uint64_t>(t.nsplit) >> p.cshift) + 1) << p.r;
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

template <typename K>
static cudaError_t part_sort(const DevTree &t, const RawOf<K> *q, uint64_t nq, const PartPlan &pp,
                             unsigned char *ws, const WsLayout &w, RawOf<K> *dst_q, uint32_t *dst_i, cudaStream_t s)
{
    PartNorm<K> pn;
    pn.split = static_cast<const K *>(t.split);
    pn.split_inv = t.split_inv;
    pn.split_off = t.split_off;
    tree_bounds<K>(t, &pn.kmin, &pn.kmax);
    pn.nsplit = t.nsplit;
    pn.r = pp.r;
    pn.cshift = pp.cshift;
    pn.scale = static_cast<float>(1u << pp.r);
    pn.split_R = t.split_R;
    pn.rshift = t.split_rshift;
    pn.p0 = t.split_p0;
    pn.wmin = t.split_wmin;
    uint32_t *total = reinterpret_cast<uint32_t *>(ws + w.counts);
    cudaError_t e = cudaMemsetAsync(total, 0, (static_cast<uint64_t>(pp.nb) + 4) * 4, s);
    if (e != cudaSuccess) return e;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    constexpr int kMaxDyn = (1 << kMaxPartBits) * 4;
    static const cudaError_t a1 =
        cudaFuncSetAttribute(k_part_hist<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
    static const cudaError_t a2 =
        cudaFuncSetAttribute(k_part_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn);
    if (a1 != cudaSuccess) return a1;
    if (a2 != cudaSuccess) return a2;
    const int dyn = static_cast<int>(pp.nb) * 4;
    // one wave: as many blocks as are resident at the largest bucket count
    static int occ_h = 0, occ_s = 0;
    if (occ_h == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_h, k_part_hist<K>, kPartThreads, kMaxDyn);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, k_part_scatter<K>, kPartThreads, kMaxDyn);
        if (e != cudaSuccess) return e;
        if (occ_h < 1) occ_h = 1;
        if (occ_s < 1) occ_s = 1;
    }
    // at least as many queries per block as buckets, so that clearing and
    // flushing the block's counters stays a small part of its work
    uint64_t gh = (nq + 8ull * kPartThreads - 1) / (8ull * kPartThreads);
    if (gh > static_cast<uint64_t>(occ_h) * sms) gh = static_cast<uint64_t>(occ_h) * sms;
    const uint64_t per_round = static_cast<uint64_t>(part_per_thread<K>()) * kPartThreads;
    uint64_t gs = (nq + per_round - 1) / per_round;
    if (gs > static_cast<uint64_t>(occ_s) * sms) gs = static_cast<uint64_t>(occ_s) * sms;
    k_part_hist<K><<<static_cast<unsigned>(gh), kPartThreads, dyn, s>>>(q, nq, pn, total, pp.nb);
    k_part_scatter<K><<<static_cast<unsigned>(gs), kPartThreads, dyn, s>>>(q, nq, pn, total, pp.nb, dst_q, dst_i);
    return cudaGetLastError();
}

// Where bt_search_batch puts the partitioned batch.
static void internal_sort_dst(unsigned char *ws, const WsLayout &w, void **dq, uint32_t **di)
{
    *dq = ws + w.qb;
    *di = reinterpret_cast<uint32_t *>(ws + w.ib);
}

static cudaError_t sort_any(const DevTree &t, const void *q, uint64_t nq, const PartPlan &pp,
                            unsigned char *ws, const WsLayout &w, void *dq, uint32_t *di,
                            cudaStream_t s)
{
    if (t.key_bytes == 32)
        return part_sort<Key32>(t, static_cast<const Raw32 *>(q), nq, pp, ws, w, static_cast<Raw32 *>(dq), di, s);
    if (t.key_bytes == 8)
        return part_sort<uint64_t>(t, static_cast<const uint64_t *>(q), nq, pp, ws, w,
                                   static_cast<uint64_t *>(dq), di, s);
    return part_sort<uint32_t>(t, static_cast<const uint32_t *>(q), nq, pp, ws, w,
                               static_cast<uint32_t *>(dq), di, s);
}

}  // namespace btgb

using namespace btgb;

extern "C" int32_t bt_sort_launches(const bt_tree *tree, uint64_t nq, int32_t sort_bits)
{
    if (!tree) return -1;
    if (tree->dev.height == 0 || nq == 0) return 0;
    return plan_partition(tree->dev, sort_bits, nq).bits ? 2 : 0;
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

    const PartPlan pp = plan_partition(t, opts ? opts->sort_bits : -1, nq);
    const void *q = d_queries;
    const uint32_t *qidx = nullptr;
    unsigned char *ws = static_cast<unsigned char *>(d_workspace);
    if (pp.bits > 0) {
        void *dq;
        uint32_t *di;
        internal_sort_dst(ws, w, &dq, &di);
        e = sort_any(t, d_queries, nq, pp, ws, w, dq, di, s);
        if (e != cudaSuccess) {
            set_error_detail("batch partition launch", e);
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
        e = sort_any(t, d_queries, nq, pp, static_cast<unsigned char *>(d_workspace), w, d_sorted_queries,
                     d_sorted_index, s);
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

extern "C" bt_status bt_learned_descend_sorted(const bt_tree *tree, const bt_model *model, const void *d_queries,
                                               const uint32_t *d_index, uint64_t nq, void *d_out_vals,
                                               uint8_t *d_out_found, unsigned long long *d_stats, bt_stream stream)
{
    if (!tree || !model) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    if (nq >= (1ull << 31)) return BT_ERR_ARG;
    if (!d_queries || !d_out_vals || !d_out_found) return BT_ERR_ARG;
    const DevTree &t = tree->dev;
    if (t.height == 0 || model->dev.leaves != t.nodes[t.height - 1]) return BT_ERR_ARG;
    const DescendArgs a{&t, d_queries, d_index, nq, d_out_vals, d_out_found, nullptr, &model->dev, d_stats};
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
    const DevTree &t = tree->dev;
    if (t.height == 0 || model->dev.leaves != t.nodes[t.height - 1]) return BT_ERR_ARG;
    const WsLayout w = ws_layout(t.key_bytes, nq);
    if (!d_workspace || ws_bytes < w.total || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return BT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const PartPlan pp = plan_partition(t, -1, nq);
    const void *q = d_queries;
    const uint32_t *qidx = nullptr;
    unsigned char *ws = static_cast<unsigned char *>(d_workspace);
    cudaError_t e;
    if (pp.bits > 0) {
        void *dq;
        uint32_t *di;
        internal_sort_dst(ws, w, &dq, &di);
        e = sort_any(t, d_queries, nq, pp, ws, w, dq, di, s);
        if (e != cudaSuccess) {
            set_error_detail("batch partition launch", e);
            return BT_ERR_CUDA;
        }
        q = dq;
        qidx = di;
    }
    const DescendArgs a{&t, q, qidx, nq, d_out_vals, d_out_found, nullptr, &model->dev, nullptr};
    e = descend_any(a, s);
    if (e != cudaSuccess) {
        set_error_detail("learned descent launch", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}

extern "C" bt_status bt_check_timeouts(void)
{
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_bt_timeouts, sizeof(v));
    if (e == cudaSuccess && v) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_bt_timeouts, &zero, sizeof(zero));
    }
    if (e != cudaSuccess) {
        set_error_detail("timeout counter", e);
        return BT_ERR_CUDA;
    }
    return v ? BT_ERR_TIMEOUT : BT_OK;
}

extern "C" bt_status bt_paper_descend_sorted(const bt_tree *tree, const void *d_queries, const uint32_t *d_index,
                                             uint64_t nq, void *d_out_vals, uint8_t *d_out_found, bt_stream stream)
{
    if (!tree) return BT_ERR_ARG;
    if (nq == 0) return BT_OK;
    if (nq >= (1ull << 31)) return BT_ERR_ARG;
    if (!d_queries || !d_out_vals || !d_out_found) return BT_ERR_ARG;
    if (tree->dev.height > 0 && !tree->d_paper) return BT_ERR_ARG;
    if (tree->dev.height == 0) return bt_descend_sorted(tree, d_queries, d_index, nq, d_out_vals, d_out_found,
                                                        nullptr, stream);
    const cudaError_t e = descend_paper(tree->dev, tree->paper, d_queries, d_index, nq, d_out_vals, d_out_found,
                                        reinterpret_cast<cudaStream_t>(stream));
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
    unsigned char *ws = static_cast<unsigned char *>(d_workspace);
    cudaError_t e;
    if (pp.bits > 0) {
        void *dq;
        uint32_t *di;
        internal_sort_dst(ws, w, &dq, &di);
        e = sort_any(t, d_queries, nq, pp, ws, w, dq, di, s);
        if (e != cudaSuccess) {
            set_error_detail("batch partition launch", e);
            return BT_ERR_CUDA;
        }
        q = dq;
        qidx = di;
    }
    e = descend_paper(t, tree->paper, q, qidx, nq, d_out_vals, d_out_found, s);
    if (e != cudaSuccess) {
        set_error_detail("paper-layout descent launch", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}
