// Synchronous level-wise descents, kept as selectable alternatives to the
// pipelined one (bt_tree_set_staging, bt_tree_set_lane_queries) so that the
// designs can be measured against each other.
//
// k_descend_sync: each warp takes 32 consecutive queries of the sorted batch
// and walks them down together; at every level below the pinned ones it
// finds its distinct nodes, stages each node's key block into shared memory
// once (16-byte cp.async, or one bulk copy per block counted on an mbarrier
// with a bounded wait), waits for the copies, and every query binary-searches
// its node (Sec. IV-A, IV-E).  The leaf probe and the result store follow
// (the value load and store are deferred into the next chunk's first staged
// level).
// k_descend2: the same with two queries per lane (64-query chunks).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "descent.cuh"

namespace btgb {

template <typename K, int M>
constexpr int stage_slots()
{
    return (M * static_cast<int>(sizeof(K)) >= 2048) ? 4 : (M * static_cast<int>(sizeof(K)) >= 512) ? 8 : 16;
}

// Shared memory per warp: its stage slots, its node list (64 entries for
// two queries per lane) and its mbarrier.
template <typename K, int M>
constexpr int sync_smem_per_warp()
{
    return stage_slots<K, M>() * M * static_cast<int>(sizeof(K)) + 64 * 4 + 8;
}

template <typename K, typename V, int M, bool COUNT>
__global__ void __launch_bounds__(kDescWarpsMax * 32) k_descend_sync(
    const DevTree t, const RawOf<K> *__restrict__ q, const uint32_t *__restrict__ qidx,
    const PartRec<K> *__restrict__ recs, uint64_t nq, V *__restrict__ out_v, uint8_t *__restrict__ out_f,
    unsigned long long *__restrict__ fetch, uint32_t wait_polls)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int CH = M * static_cast<int>(sizeof(K)) / 16;  // 16-byte chunks per node block
    constexpr int SLOTS = stage_slots<K, M>();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t pin_bytes = t.pin_bytes;
    unsigned char *pin = smem;
    K *stage = reinterpret_cast<K *>(smem + pin_bytes) + warp * SLOTS * M;
    unsigned char *after_stage = smem + pin_bytes + nw * SLOTS * M * sizeof(K);
    uint32_t *list = reinterpret_cast<uint32_t *>(after_stage) + warp * 64;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(after_stage + nw * 64 * 4) + warp;
    const bool tma = (t.staging == BT_STAGE_BULK);
    uint32_t phase = 0;
    if (tma && lane == 0) mbar_init(mbar);
    __syncwarp();

    const unsigned char *top = static_cast<const unsigned char *>(t.keys[0]);
    for (uint32_t i = threadIdx.x * 16u; i < pin_bytes; i += blockDim.x * 16u) cp_async16_ca(pin + i, top + i);
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
        load_query<K>(q, qidx, recs, v ? pos : c * 32, key_n, dst_n);
        if (!v) dst_n = 0;
    }
    // The previous chunk's result: its value load is issued at its leaf
    // level and consumed (stored) only after this chunk's first staged level.
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
            load_query<K>(q, qidx, recs, vn ? pn : cn * 32, key_n, dst_n);
            if (!vn) dst_n = 0;
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
            const K *blk =
                reinterpret_cast<const K *>(pin + (static_cast<const unsigned char *>(t.keys[l]) - top)) +
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
                if (tma) {
                    // one bulk copy per node block, completion counted in
                    // bytes on the warp's mbarrier; the wait is bounded
                    constexpr unsigned kBlk = M * sizeof(K);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    if (lane == 0) mbar_arrive_expect_tx(mbar, static_cast<unsigned>(nu) * kBlk);
                    __syncwarp();
                    if (lane < nu)
                        bulk_g2s(stage + lane * M, lk + static_cast<uint64_t>(list[rb + lane]) * M, kBlk, mbar);
                    if (!mbar_wait_warp(mbar, phase, wait_polls)) {
                        // this warp's results are invalid; its copies land before it leaves
                        mbar_give_up(mbar, phase, lane);
                        return;
                    }
                    phase ^= 1u;
                } else {
                    for (int i = lane; i < nu * CH; i += 32) {
                        const int u = i / CH, part = i - u * CH;
                        const unsigned char *src =
                            reinterpret_cast<const unsigned char *>(lk + static_cast<uint64_t>(list[rb + u]) * M) +
                            part * 16;
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
                pend_store = valid && dst < nq;  // a position outside the batch is never written
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

template <typename K, typename V, int M, bool COUNT>
__global__ void __launch_bounds__(kDescWarpsMax * 32) k_descend2(
    const DevTree t, const RawOf<K> *__restrict__ q, const uint32_t *__restrict__ qidx,
    const PartRec<K> *__restrict__ recs, uint64_t nq, V *__restrict__ out_v, uint8_t *__restrict__ out_f,
    unsigned long long *__restrict__ fetch)
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
        K ka, kb;
        uint32_t da, db;
        load_query<K>(q, qidx, recs, va ? pa : c * 64, ka, da);
        load_query<K>(q, qidx, recs, vb ? pb : c * 64, kb, db);
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
                if (va && da < nq) {
                    out_v[da] = v_a;
                    out_f[da] = hit_a ? 1 : 0;
                }
                if (vb && db < nq) {
                    out_v[db] = v_b;
                    out_f[db] = hit_b ? 1 : 0;
                }
            }
        }
    }
}

template <typename K, typename V, int M, bool COUNT>
static cudaError_t launch_sync(const DescendArgs &a, cudaStream_t s)
{
    const DevTree &t = *a.t;
    const int nw = t.warps > 0 ? t.warps : kDescWarpsDefault;
    const int smem = static_cast<int>(t.pin_bytes) + nw * sync_smem_per_warp<K, M>();
    const bool two = t.lane_queries == 2;
    const void *kern = two ? reinterpret_cast<const void *>(k_descend2<K, V, M, COUNT>)
                           : reinterpret_cast<const void *>(k_descend_sync<K, V, M, COUNT>);
    cudaError_t e = ensure_dyn_smem(kern, kPinBudgetMax + kDescWarpsMax * sync_smem_per_warp<K, M>());
    if (e != cudaSuccess) return e;
    unsigned grid = 0;
    e = persistent_grid(kern, nw * 32, smem, static_cast<uint64_t>(nw) * (two ? 64 : 32), a.nq, &grid,
                        t.corun_descent_bps);
    if (e != cudaSuccess) return e;
    if (two)
        k_descend2<K, V, M, COUNT><<<grid, nw * 32, smem, s>>>(t, static_cast<const RawOf<K> *>(a.q), a.qidx,
                                                               static_cast<const PartRec<K> *>(a.recs), a.nq,
                                                               static_cast<V *>(a.out_v), a.out_f, a.fetch);
    else
        k_descend_sync<K, V, M, COUNT><<<grid, nw * 32, smem, s>>>(t, static_cast<const RawOf<K> *>(a.q), a.qidx,
                                                                   static_cast<const PartRec<K> *>(a.recs), a.nq,
                                                                   static_cast<V *>(a.out_v), a.out_f, a.fetch,
                                                                   first_wait_polls());
    return cudaGetLastError();
}

template <typename K, typename V>
static cudaError_t sync_m(const DescendArgs &a, cudaStream_t s)
{
    switch (a.t->m) {
    case 8: return a.fetch ? launch_sync<K, V, 8, true>(a, s) : launch_sync<K, V, 8, false>(a, s);
    case 16: return a.fetch ? launch_sync<K, V, 16, true>(a, s) : launch_sync<K, V, 16, false>(a, s);
    case 32: return a.fetch ? launch_sync<K, V, 32, true>(a, s) : launch_sync<K, V, 32, false>(a, s);
    default: return a.fetch ? launch_sync<K, V, 64, true>(a, s) : launch_sync<K, V, 64, false>(a, s);
    }
}

cudaError_t descend_synchronous(const DescendArgs &a, cudaStream_t s)
{
    const DevTree &t = *a.t;
    if (t.key_bytes == 8) return t.val_bytes == 8 ? sync_m<uint64_t, uint64_t>(a, s) : sync_m<uint64_t, uint32_t>(a, s);
    if (t.key_bytes == 32) return t.val_bytes == 8 ? sync_m<Key32, uint64_t>(a, s) : sync_m<Key32, uint32_t>(a, s);
    return t.val_bytes == 8 ? sync_m<uint32_t, uint64_t>(a, s) : sync_m<uint32_t, uint32_t>(a, s);
}

cudaError_t take_wait_counters_synchronous(unsigned *timeouts, unsigned *pending)
{
    return take_wait_counters(timeouts, pending);
}

}  // namespace btgb
