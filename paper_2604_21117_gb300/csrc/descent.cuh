// Device helpers shared by the level-wise descent kernels, and the host-side
// interface between the search entry points (search.cu) and the kernel
// families (desc_pipe.cu: the pipelined descent; desc_sync.cu: the
// synchronous descents; desc_paper.cu: the descent over the paper's node
// layout).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "bt_internal.h"

namespace btgb {

// ---------------------------------------------------------------- copies

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

__device__ __forceinline__ void prefetch_l1(const void *p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the previous kernel of the stream is still
// running; pdl_wait() returns once that kernel has completed and its memory
// is visible (before it, a kernel touches only its own shared memory and
// read-only data).  pdl_trigger() lets the next such kernel start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---- bulk asynchronous copies (the TMA unit, non-tensor form) with an mbarrier ----

// Bounded waits that gave up (the results of that search are invalid), and
// give-ups after which the warp's copies had still not landed; read and
// cleared by bt_check_timeouts.  Device code is compiled per translation
// unit, so every kernel family has its own pair (see take_wait_counters).
static __device__ unsigned int g_bt_timeouts;
static __device__ unsigned int g_bt_copies_pending;
// Poll limit of the second wait after a give-up, which lets the copies in
// flight land before the warp leaves.
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

// An L2 cache policy that marks the lines it loads first in line for
// eviction: for data read once (leaf blocks, values), so that it does not
// push out what is read again (the partitioned batch, the inner levels).
__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Bulk copy global -> shared memory with an L2 cache policy.
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, unsigned bytes, uint64_t *bar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
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

// Bounded wait of the whole warp for phase `phase` of its mbarrier: false
// if some lane gave up after `polls` polls.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t phase, uint32_t polls)
{
    bool done = false;
    for (uint32_t i = 0; i < polls; ++i)
        if (mbar_try_wait(bar, phase)) {
            done = true;
            break;
        }
    return __all_sync(0xffffffffu, done);
}

// After a give-up: count it, then wait again (the full limit) so that the
// warp's copies land before it leaves and its block's shared memory is
// released; a second give-up is counted on its own.
__device__ __forceinline__ void mbar_give_up(uint64_t *bar, uint32_t phase, int lane)
{
    if (lane == 0) atomicAdd(&g_bt_timeouts, 1u);
    bool done = false;
    for (uint32_t i = 0; i < kMbarSpinLimit; ++i)
        if (mbar_try_wait(bar, phase)) {
            done = true;
            break;
        }
    if (!__all_sync(0xffffffffu, done) && lane == 0) atomicAdd(&g_bt_copies_pending, 1u);
}

// ------------------------------------------------------------ key access

// A key loaded from global memory through L1 (the tree is read-only).
template <typename K>
__device__ __forceinline__ K ld_key(const K *p)
{
    if constexpr (sizeof(K) == 8) {
        return static_cast<K>(__ldca(reinterpret_cast<const unsigned long long *>(p)));
    } else {
        return static_cast<K>(__ldca(reinterpret_cast<const unsigned int *>(p)));
    }
}

template <>
__device__ __forceinline__ Key32 ld_key<Key32>(const Key32 *p)
{
    const ulonglong2 *v = reinterpret_cast<const ulonglong2 *>(p);
    const ulonglong2 a = __ldca(v), b = __ldca(v + 1);
    Key32 k;
    k.w[0] = a.x;
    k.w[1] = a.y;
    k.w[2] = b.x;
    k.w[3] = b.y;
    return k;
}

template <typename K>
__device__ __forceinline__ K key_shfl(K k, int src)
{
    if constexpr (sizeof(K) == 8) {
        return static_cast<K>(__shfl_sync(0xffffffffu, static_cast<unsigned long long>(k), src));
    } else {
        return static_cast<K>(__shfl_sync(0xffffffffu, static_cast<unsigned int>(k), src));
    }
}

template <>
__device__ __forceinline__ Key32 key_shfl<Key32>(Key32 k, int src)
{
    Key32 r;
#pragma unroll
    for (int j = 0; j < 4; ++j) r.w[j] = __shfl_sync(0xffffffffu, static_cast<unsigned long long>(k.w[j]), src);
    return r;
}

// *p < key for a key read from global memory through L1; a 32-byte key's
// first word alone unless it ties.
template <typename K>
__device__ __forceinline__ bool ld_lt(const K *p, const K &key)
{
    return ld_key(p) < key;
}

template <>
__device__ __forceinline__ bool ld_lt<Key32>(const Key32 *p, const Key32 &key)
{
    const uint64_t w0 = __ldca(reinterpret_cast<const unsigned long long *>(p));
    if (w0 != key.w[0]) return w0 < key.w[0];
    return ld_key(p) < key;
}

// ------------------------------------------------------------- node math

constexpr int kDescWarpsDefault = 8;
constexpr int kDescWarpsMax = 16;
constexpr int kPinBudgetMax = 49152;

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
        if (mem_lt(blk + r + hlf - 1, key)) r += hlf;
    return r;
}

// The same rank read straight from a node block in global memory through
// L1: every 128-byte line of the block is prefetched first, so the probes
// wait for one round trip and then hit L1.  Lanes of a warp that share the
// node share its lines.
template <typename K, int M>
__device__ __forceinline__ int block_rank_l1(const K *blk, K key)
{
    constexpr int kLines = (M * static_cast<int>(sizeof(K)) + 127) / 128;
    if constexpr (kLines > 1) {
#pragma unroll
        for (int i = 0; i < kLines; ++i) prefetch_l1(reinterpret_cast<const unsigned char *>(blk) + 128 * i);
    }
    int r = 0;
#pragma unroll
    for (int hlf = M / 2; hlf >= 1; hlf >>= 1)
        if (ld_lt(blk + r + hlf - 1, key)) r += hlf;
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

// ------------------------------------------------------- host interface

// One search's descent launch: everything a kernel instantiation needs.
struct DescendArgs {
    const DevTree *t;
    const bt_tree *tree;  // for the L2 window; may be null
    const void *q;         // keys (with qidx, or identity positions), when recs is null
    const uint32_t *qidx;
    const void *recs;      // the partition's records (PartRec<K>), or null
    uint64_t nq;
    void *out_v;
    uint8_t *out_f;
    unsigned long long *fetch;
    const ModelDev *md;  // non-null: learned descent
    unsigned long long *lstats;
};

// Pipelined descent (staging mode BT_STAGE_PIPELINED, and every learned search).
cudaError_t descend_pipelined(const DescendArgs &a, cudaStream_t s);
// Synchronous descents: cp.async or bulk-copy staging, and two queries per lane.
cudaError_t descend_synchronous(const DescendArgs &a, cudaStream_t s);
// Level-wise descent over the paper's node layout (Eq. 1).
cudaError_t descend_paper_layout(const DevTree &t, const PaperTree &p, const void *q, const uint32_t *qidx,
                                 const void *recs, uint64_t nq, void *out_v, uint8_t *out_f, cudaStream_t s);

// Grid of a persistent descent: enough blocks for the chunks, at most one
// full wave of resident blocks.
cudaError_t persistent_grid(const void *kern, int threads, int smem, uint64_t units_per_block, uint64_t units,
                            unsigned *grid, int max_per_sm = 0);

// This translation unit's wait counters, read and cleared (synchronous).
static inline cudaError_t take_wait_counters(unsigned *timeouts, unsigned *pending)
{
    unsigned v[2] = {0, 0};
    cudaError_t e = cudaMemcpyFromSymbol(&v[0], g_bt_timeouts, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v[1], g_bt_copies_pending, sizeof(unsigned));
    const unsigned zero = 0;
    if (e == cudaSuccess && v[0]) e = cudaMemcpyToSymbol(g_bt_timeouts, &zero, sizeof(zero));
    if (e == cudaSuccess && v[1]) e = cudaMemcpyToSymbol(g_bt_copies_pending, &zero, sizeof(zero));
    *timeouts += v[0];
    *pending += v[1];
    return e;
}
cudaError_t take_wait_counters_pipelined(unsigned *timeouts, unsigned *pending);
cudaError_t take_wait_counters_synchronous(unsigned *timeouts, unsigned *pending);

}  // namespace btgb
