// The pipelined level-wise descent (default), plain and learned.
//
// Each warp walks chunks of 32 consecutive queries of the sorted batch down
// the tree (Sec. IV-A): at every level the warp's queries meet the node
// they are routed to, and the first separator a query is <= to gives its
// child (Sec. IV-E).  The leaf level carries almost all of the bytes (at
// 2^24 keys and 2^20 queries, 80% of the distinct node bytes), so its
// staging is overlapped with the next chunk's work:
//
//   iteration i:  chunk i walks the top levels (pinned in shared memory)
//                 and the inner levels (read through L1, or staged with
//                 16-byte cp.async: bt_tree_set_descent) down to its leaf;
//                 the result of chunk i-2 is stored (its value load has had
//                 a whole iteration to arrive);
//                 chunk i-1's leaf blocks, staged by bulk copies issued in
//                 iteration i-1, are awaited on the warp's mbarrier (bounded
//                 wait), every query ranks itself in its leaf (binary search,
//                 or warp ballot + popc), a hit issues its value load;
//                 chunk i's distinct leaves (each staged once, Sec. IV-A) are
//                 issued as bulk copies, one per leaf block, completing on the
//                 mbarrier while chunk i+1 walks its inner levels.
//
// A warp holding more distinct leaves than its slots stages the first
// slots' worth.  Over a partitioned batch (rarely more than the slots) the
// rest follow in further rounds, waited for at once; over a small batch
// searched as given (TAIL_L1: up to 32 leaves a chunk, at most 16 chunks per
// SM) the lanes whose leaf is beyond the slots prefetch its lines into L1
// when the copies are issued and rank in it from there, in the same
// iteration as the staged ones.  Learned searches start from the
// model's predicted leaf where its window proves the leaf, lane by lane; the
// other lanes walk the inner levels.  Everything is integer compares.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <type_traits>

#include "descent.cuh"

// Leaf blocks and values are loaded with an L2 evict-first policy (1), or
// with the default policy (0).
#ifndef BT_LEAF_EVICT_FIRST
#define BT_LEAF_EVICT_FIRST 1
#endif
// Register limit of the pipelined descent (0: the compiler's choice).
#ifndef BT_DESCEND_MAXNREG
#define BT_DESCEND_MAXNREG 0
#endif
// Inner-level slots per warp when inner levels are staged.
#ifndef BT_INNER_SLOTS
#define BT_INNER_SLOTS 4
#endif

namespace btgb {

// Leaf blocks a warp stages per round (about 4 KB), and inner-level slots.
template <typename K, int M>
constexpr int leaf_slots()
{
    return (M * static_cast<int>(sizeof(K)) >= 2048) ? 2
           : (M * static_cast<int>(sizeof(K)) >= 1024) ? 4
           : (M * static_cast<int>(sizeof(K)) >= 512)  ? 8
                                                        : 16;
}

template <typename K, int M>
constexpr int inner_slots()
{
    return leaf_slots<K, M>() * BT_INNER_SLOTS / 16 > 0 ? leaf_slots<K, M>() * BT_INNER_SLOTS / 16 : 1;
}

template <typename K, int M, bool LEARN>
inline int pipe_smem_per_warp(bool istage)
{
    constexpr int blk = M * static_cast<int>(sizeof(K));
    return leaf_slots<K, M>() * blk + (istage ? inner_slots<K, M>() * blk : 0) + 64 * 4 +
           (LEARN ? kLeafMaxCap * static_cast<int>(sizeof(K)) : 0) + 8;
}

// Issue one round of leaf blocks (list[0..nu)) as bulk copies into the
// warp's slots, completing on its mbarrier.
template <typename K, int M>
__device__ __forceinline__ void issue_leaf_round(K *stage, const K *lk, const uint32_t *lst, int nu, uint64_t *mbar,
                                                 int lane)
{
    constexpr unsigned kBlk = M * sizeof(K);
    // the slots' previous contents were read through the generic proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (lane == 0) mbar_arrive_expect_tx(mbar, static_cast<unsigned>(nu) * kBlk);
    __syncwarp();
    if (lane < nu) {
#if BT_LEAF_EVICT_FIRST
        bulk_g2s_hint(stage + lane * M, lk + static_cast<uint64_t>(lst[lane]) * M, kBlk, mbar, l2_evict_first_policy());
#else
        bulk_g2s(stage + lane * M, lk + static_cast<uint64_t>(lst[lane]) * M, kBlk, mbar);
#endif
    }
}

// A leaf value, read once.
template <typename V>
__device__ __forceinline__ V ld_value(const V *p)
{
#if BT_LEAF_EVICT_FIRST
    if constexpr (sizeof(V) == 8) {
        return static_cast<V>(__ldcs(reinterpret_cast<const unsigned long long *>(p)));
    } else {
        return static_cast<V>(__ldcs(reinterpret_cast<const unsigned int *>(p)));
    }
#else
    return *p;
#endif
}

// Rank (and equality) of each lane's key in its leaf, for the lanes whose
// leaf is in this round's slots [rb, rb + nu).  Binary search per lane, or
// (ballot) the Sec. IV-E comparator row: for each query in turn, lane j
// compares slot j (and j + 32) of that query's leaf, and the population
// count of the ballot is the number of keys below the query.
template <typename K, int M>
__device__ __forceinline__ void leaf_rank_round(const K *stage, int rb, int nu, int slot, const K &key, bool ballot,
                                                int lane, int &r, bool &eq)
{
    if (!ballot) {
        if (slot >= rb && slot < rb + nu) {
            const K *blk = stage + (slot - rb) * M;
            r = block_rank<K, M>(blk, key);
            eq = (blk[r] == key);
        }
        return;
    }
    for (int i = 0; i < 32; ++i) {
        const int si = __shfl_sync(0xffffffffu, slot, i);
        if (si < rb || si >= rb + nu) continue;  // uniform across the warp
        const K ki = key_shfl(key, i);
        const K *blk = stage + (si - rb) * M;
        int cnt = 0;
#pragma unroll
        for (int h = 0; h < (M + 31) / 32; ++h) {
            const int j = lane + 32 * h;
            const bool lt = (j < M) && (blk[j < M ? j : 0] < ki);
            cnt += __popc(__ballot_sync(0xffffffffu, lt));
        }
        if (lane == i) {
            r = cnt;
            eq = (blk[cnt] == ki);
        }
    }
}

#if BT_DESCEND_MAXNREG
#define BT_DESCEND_REGS __maxnreg__(BT_DESCEND_MAXNREG)
#else
#define BT_DESCEND_REGS __launch_bounds__(kDescWarpsMax * 32)
#endif

// MODEL: kModelNone for the plain descent, kModelPL or kModelMLP for the
// learned one (separate instantiations, so that the MLP's registers do not
// limit the others).
template <typename K, typename V, int M, bool COUNT, int MODEL, bool TAIL_L1 = false>
__global__ void BT_DESCEND_REGS k_descend(
    const DevTree t, const RawOf<K> *__restrict__ q, const uint32_t *__restrict__ qidx,
    const PartRec<K> *__restrict__ recs, uint64_t nq, V *__restrict__ out_v, uint8_t *__restrict__ out_f,
    unsigned long long *__restrict__ fetch, const ModelDev md,
    unsigned long long *__restrict__ lstats, uint32_t wait_polls)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int BLK = M * static_cast<int>(sizeof(K));
    constexpr int CH = BLK / 16;  // 16-byte pieces per node block
    constexpr int SL = leaf_slots<K, M>();
    constexpr int SI = inner_slots<K, M>();
    constexpr bool LEARN = MODEL != kModelNone;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool istage = !LEARN && t.inner_stage != 0;
    const bool ballot = t.rank_ballot != 0;
    const uint32_t pin_bytes = t.pin_bytes;
    const uint32_t mbytes = LEARN ? model_smem_bytes(md) : 0u;
    // shared memory: pinned levels | model | per warp: leaf slots, inner
    // slots, node lists, leaf-max window, mbarrier
    unsigned char *pin = smem;
    unsigned char *msm = smem + pin_bytes;
    unsigned char *p = msm + mbytes;
    K *lstage = reinterpret_cast<K *>(p) + warp * SL * M;
    p += nw * SL * BLK;
    K *istg = reinterpret_cast<K *>(p) + warp * SI * M;
    if (istage) p += nw * SI * BLK;
    uint32_t *list = reinterpret_cast<uint32_t *>(p) + warp * 64;  // leaf list of the chunk in flight
    uint32_t *ilist = list + 32;                                     // inner-level lists
    p += nw * 64 * 4;
    K *lmstage = reinterpret_cast<K *>(p) + warp * kLeafMaxCap;
    if (LEARN) p += nw * kLeafMaxCap * sizeof(K);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(p) + warp;
    if (lane == 0) mbar_init(mbar);
    __syncwarp();

    // Top levels, pinned once per block.
    const unsigned char *top = static_cast<const unsigned char *>(t.keys[0]);
    for (uint32_t i = threadIdx.x * 16u; i < pin_bytes; i += blockDim.x * 16u) cp_async16_ca(pin + i, top + i);
    // The model's parameters, copied once per block when they fit.
    const uint64_t *mb = md.b;
    const float *minv = md.inv_w, *mslope = md.slope, *micpt = md.icpt, *mmlp = md.mlp;
    if constexpr (LEARN) {
        if (mbytes) {
            if constexpr (MODEL == kModelPL) {
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
                for (uint32_t i = threadIdx.x; i < static_cast<uint32_t>(kMlpParams); i += blockDim.x)
                    sp[i] = md.mlp[i];
                mmlp = sp;
            }
        }
    }
    // the batch (and the outputs) belong to the previous kernel until it is
    // done; the copies above stay in flight meanwhile
    pdl_wait();

    const uint64_t nchunks = (nq + 31) / 32;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * nw;
    const int H = t.height, P = t.pin_levels, LEAF = H - 1;
    const K *lkeys = static_cast<const K *>(t.keys[LEAF]);
    const V *vals = static_cast<const V *>(t.vals);
    uint64_t c = static_cast<uint64_t>(blockIdx.x) * nw + warp;

    // The next chunk's queries, loaded one iteration ahead.  Tail lanes
    // follow lane 0's query so that they never add a node fetch.
    K key_n = KeyOps<K>::ones();
    uint32_t dst_n = 0;
    if (c < nchunks) {
        const uint64_t pos = c * 32 + lane;
        const bool v = pos < nq;
        load_query<K>(q, qidx, recs, v ? pos : c * 32, key_n, dst_n);
        if (!v) dst_n = 0;
    }
    // the pinned levels and the model, copied above (the first queries'
    // loads overlap the copies)
    cp_async_wait_all();
    __syncthreads();
    // Chunk A: its leaf round 0 is in flight.
    bool a_live = false, a_valid = false;
    K a_key = key_n;
    uint32_t a_dst = 0, a_node = 0;
    int a_slot = 0, a_U = 0;
    // The result of the chunk before A, stored one iteration late.
    V pend_val = 0;
    uint32_t pend_dst = 0;
    bool pend_store = false, pend_hit = false;
    uint32_t phase = 0;

    for (;;) {
        const bool b_live = c < nchunks;  // uniform across the warp
        const K key = key_n;
        const uint32_t dst = dst_n;
        bool valid = false;
        uint32_t node = 0;
        if (b_live) {
            valid = c * 32 + lane < nq;
            const uint64_t cn = c + stride;
            if (cn < nchunks) {
                const uint64_t pn = cn * 32 + lane;
                const bool vn = pn < nq;
                load_query<K>(q, qidx, recs, vn ? pn : cn * 32, key_n, dst_n);
                if (!vn) dst_n = 0;
            }
            bool proven = false;
            if constexpr (LEARN) {
                // Predicted leaf and its error window; a lane whose leaf is
                // proven (the leaf below the window ends below the query, and
                // the first window leaf whose largest key is >= the query is
                // the leaf) skips the inner levels.  A warp whose windows fit
                // kLeafMaxCap leaves stages their leaf maxima once; wider
                // windows (unsorted batches) are checked lane by lane in
                // global memory.
                const uint32_t L = md.leaves;
                uint32_t hat;
                if constexpr (MODEL == kModelPL)
                    hat = leaf_from_pred(pl_predict(mb, minv, mslope, micpt, md.segments, static_cast<uint64_t>(key)), L);
                else
                    hat = model_leaf(md, mb, minv, mslope, micpt, mmlp, static_cast<uint64_t>(key));
                const uint32_t er = __ldg(md.errs + err_range(hat, L));
                const uint32_t lo = hat > er ? hat - er : 0u;
                const uint32_t hi = (static_cast<uint64_t>(hat) + er < L) ? hat + er : L - 1;
                uint32_t wlo = __reduce_min_sync(0xffffffffu, lo);
                if (wlo > 0) --wlo;
                const uint32_t whi = __reduce_max_sync(0xffffffffu, hi);
                const K *lm = static_cast<const K *>(md.leaf_max);
                const bool staged = whi - wlo < static_cast<uint32_t>(kLeafMaxCap);
                if (staged) {
                    for (uint32_t j = lane; j <= whi - wlo; j += 32) lmstage[j] = lm[wlo + j];
                    __syncwarp();
                }
                if (!staged) {
                    // this lane's window, read through L1: prefetch its lines
                    // (up to four of 128 bytes), then search them
                    const uint32_t first = lo > 0 ? lo - 1 : 0;
                    const unsigned char *w0 = reinterpret_cast<const unsigned char *>(lm + first);
                    const unsigned char *w1 = reinterpret_cast<const unsigned char *>(lm + hi) + sizeof(K);
                    const uintptr_t l0 = reinterpret_cast<uintptr_t>(w0) & ~uintptr_t(127);
                    if (reinterpret_cast<uintptr_t>(w1) - l0 <= 4 * 128)
                        for (uintptr_t a = l0; a < reinterpret_cast<uintptr_t>(w1); a += 128)
                            prefetch_l1(reinterpret_cast<const void *>(a));
                }
                auto leaf_max = [&](uint32_t j) -> K { return staged ? lmstage[j - wlo] : ld_key(lm + j); };
                const bool low_ok = (lo == 0) || (leaf_max(lo - 1) < key);
                uint32_t a = lo, e = hi + 1;  // first j in [lo, hi] with key <= leaf_max[j]
                while (a < e) {
                    const uint32_t mid = (a + e) >> 1;
                    if (leaf_max(mid) < key)
                        a = mid + 1;
                    else
                        e = mid;
                }
                if (a <= hi) {
                    node = a;
                    proven = low_ok;
                } else if (hi == L - 1) {  // above every key: the last leaf
                    node = L - 1;
                    proven = low_ok;
                }
                if (staged) __syncwarp();
                if (lstats) {  // queries the window served, and queries that walk the inner levels
                    const unsigned served = __popc(__ballot_sync(0xffffffffu, proven && valid));
                    const unsigned all = __popc(__ballot_sync(0xffffffffu, valid));
                    if (lane == 0) {
                        atomicAdd(lstats + 0, static_cast<unsigned long long>(served));
                        atomicAdd(lstats + 1, static_cast<unsigned long long>(all - served));
                    }
                }
            }
            if (!proven) {
                node = 0;
                int l = 0;
                for (; l < P; ++l) {  // pinned levels: search the block's shared copy
                    if (COUNT) {
                        int U, slot;
                        warp_distinct(node, lane, ilist, U, slot);
                        if (lane == 0) atomicAdd(fetch + l, static_cast<unsigned long long>(U));
                        __syncwarp();
                    }
                    const K *blk =
                        reinterpret_cast<const K *>(pin + (static_cast<const unsigned char *>(t.keys[l]) - top)) +
                        static_cast<uint64_t>(node) * M;
                    node = child_of(t, l, node, block_rank<K, M>(blk, key));
                }
                for (; l < LEAF; ++l) {
                    const K *lk = static_cast<const K *>(t.keys[l]);
                    if (istage) {
                        // each distinct node's block staged once with 16-byte cp.async
                        int U, slot;
                        warp_distinct(node, lane, ilist, U, slot);
                        if (COUNT && lane == 0) atomicAdd(fetch + l, static_cast<unsigned long long>(U));
                        __syncwarp();
                        int r = 0;
                        for (int rb = 0; rb < U; rb += SI) {
                            const int nu = (U - rb < SI) ? U - rb : SI;
                            for (int i = lane; i < nu * CH; i += 32) {
                                const int u = i / CH, part = i - u * CH;
                                cp_async16_ca(reinterpret_cast<unsigned char *>(istg + u * M) + part * 16,
                                              reinterpret_cast<const unsigned char *>(
                                                  lk + static_cast<uint64_t>(ilist[rb + u]) * M) +
                                                  part * 16);
                            }
                            cp_async_wait_all();
                            __syncwarp();
                            if (slot >= rb && slot < rb + nu) r = block_rank<K, M>(istg + (slot - rb) * M, key);
                            __syncwarp();
                        }
                        node = child_of(t, l, node, r);
                    } else {
                        if (COUNT) {
                            int U, slot;
                            warp_distinct(node, lane, ilist, U, slot);
                            if (lane == 0) atomicAdd(fetch + l, static_cast<unsigned long long>(U));
                            __syncwarp();
                        }
                        node = child_of(t, l, node, block_rank_l1<K, M>(lk + static_cast<uint64_t>(node) * M, key));
                    }
                }
            }
        }
        if (pend_store) {
            out_v[pend_dst] = pend_val;
            out_f[pend_dst] = pend_hit ? 1 : 0;
            pend_store = false;
        }
        if (a_live) {
            if (!mbar_wait_warp(mbar, phase, wait_polls)) {
                mbar_give_up(mbar, phase, lane);
                return;
            }
            phase ^= 1u;
            int r = 0;
            bool eq = false;
            leaf_rank_round<K, M>(lstage, 0, a_U < SL ? a_U : SL, a_slot, a_key, ballot, lane, r, eq);
            if constexpr (TAIL_L1) {
                if (a_slot >= SL) {  // a leaf beyond the slots: its lines were prefetched into L1
                    const K *blk = lkeys + static_cast<uint64_t>(a_node) * M;
                    r = block_rank_l1<K, M>(blk, a_key);
                    eq = (ld_key(blk + r) == a_key);
                }
            } else {
                for (int rb = SL; rb < a_U; rb += SL) {  // further rounds, waited for at once
                    const int nu = (a_U - rb < SL) ? a_U - rb : SL;
                    __syncwarp();
                    issue_leaf_round<K, M>(lstage, lkeys, list + rb, nu, mbar, lane);
                    if (!mbar_wait_warp(mbar, phase, wait_polls)) {
                        mbar_give_up(mbar, phase, lane);
                        return;
                    }
                    phase ^= 1u;
                    leaf_rank_round<K, M>(lstage, rb, nu, a_slot, a_key, ballot, lane, r, eq);
                }
            }
            const uint64_t cnt = t.cbase[LEAF] + (a_node < t.crem[LEAF] ? 1u : 0u);
            const bool hit = (static_cast<uint64_t>(r) < cnt) && eq;
            pend_val = static_cast<V>(~static_cast<V>(0));
            if (hit) pend_val = ld_value(vals + static_cast<uint64_t>(a_node) * M + r);
            pend_hit = hit;
            pend_dst = a_dst;
            pend_store = a_valid && a_dst < nq;  // a position outside the batch is never written
            a_live = false;
            __syncwarp();  // every lane is done with the slots before they are refilled
        }
        if (!b_live) break;
        // This chunk's distinct leaves, staged once each; awaited next iteration.
        int U, slot;
        warp_distinct(node, lane, list, U, slot);
        if (COUNT && lane == 0) atomicAdd(fetch + LEAF, static_cast<unsigned long long>(U));
        __syncwarp();
        issue_leaf_round<K, M>(lstage, lkeys, list, U < SL ? U : SL, mbar, lane);
        if constexpr (TAIL_L1) {
            if (slot >= SL) {  // beyond the slots: into L1 now, ranked from there next iteration
                const unsigned char *b =
                    reinterpret_cast<const unsigned char *>(lkeys + static_cast<uint64_t>(node) * M);
#pragma unroll
                for (int i = 0; i < (BLK + 127) / 128; ++i) prefetch_l1(b + 128 * i);
            }
        }
        a_live = true;
        a_valid = valid;
        a_key = key;
        a_dst = dst;
        a_node = node;
        a_slot = slot;
        a_U = U;
        c += stride;
    }
    if (pend_store) {
        out_v[pend_dst] = pend_val;
        out_f[pend_dst] = pend_hit ? 1 : 0;
    }
}

// Launch through cudaLaunchKernelEx as a programmatic dependent launch, with
// the tree's L2 access-policy window (the non-pinned inner levels marked
// persisting) when it has one.
template <typename... KArgs, typename... Args>
static cudaError_t launch_with_window(void (*kern)(KArgs...), unsigned grid, int threads, int smem, cudaStream_t s,
                                      const bt_tree *tree, Args... args)
{
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(static_cast<unsigned>(threads));
    cfg.dynamicSmemBytes = static_cast<size_t>(smem);
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    memset(attr, 0, sizeof(attr));
    // may start while the previous kernel finishes (the kernel waits for it,
    // pdl_wait, before touching the batch or the outputs)
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    unsigned n = 1;
    if (tree && tree->l2_bytes) {
        attr[1].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[1].val.accessPolicyWindow.base_ptr = const_cast<void *>(tree->l2_base);
        attr[1].val.accessPolicyWindow.num_bytes = static_cast<size_t>(tree->l2_bytes);
        attr[1].val.accessPolicyWindow.hitRatio = tree->l2_hit_ratio;
        attr[1].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[1].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        n = 2;
    }
    cfg.attrs = attr;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename K, typename V, int M, bool COUNT, int MODEL, bool TAIL_L1 = false>
static cudaError_t launch_pipe(const DescendArgs &a, cudaStream_t s)
{
    // inner levels staged (1) or through L1 (0); "auto" (2) stages them for a
    // partitioned batch, whose warps meet one or two nodes per level, and not
    // for an unsorted one, whose warps meet up to 32
    constexpr bool LEARN = MODEL != kModelNone;
    DevTree t = *a.t;
    const bool istage = !LEARN && (t.inner_stage == 1 || (t.inner_stage == 2 && a.recs != nullptr));
    t.inner_stage = istage ? 1 : 0;
    int nw = t.warps > 0 ? t.warps : kDescWarpsDefault;
    // A batch with fewer 32-query chunks per SM than the tree's warps per
    // block would sit on a few SMs: its blocks get that many warps (at least
    // two), so that it spreads over more SMs (batch 1024: 6.3 us a call back
    // to back at 2 warps per block against 6.7 at 8).
    int sms = 0;
    cudaError_t e = dev_sm_count(&sms);
    if (e != cudaSuccess) return e;
    if (sms < 1) sms = 1;
    const uint64_t per_sm = ((a.nq + 31) / 32 + static_cast<uint64_t>(sms) - 1) / static_cast<uint64_t>(sms);
    if (per_sm < static_cast<uint64_t>(nw)) nw = per_sm < 2 ? (nw < 2 ? nw : 2) : static_cast<int>(per_sm);
    ModelDev none;
    memset(&none, 0, sizeof(none));
    const ModelDev &md = a.md ? *a.md : none;
    const int mbytes = LEARN ? static_cast<int>(model_smem_bytes(md)) : 0;
    const int smem = static_cast<int>(t.pin_bytes) + mbytes + nw * pipe_smem_per_warp<K, M, LEARN>(istage);
    auto kern = k_descend<K, V, M, COUNT, MODEL, TAIL_L1>;
    constexpr int max_model = LEARN ? static_cast<int>(kModelSmemSegments) * 20 : 0;
    e = ensure_dyn_smem(reinterpret_cast<const void *>(kern),
                        kPinBudgetMax + max_model + kDescWarpsMax * pipe_smem_per_warp<K, M, LEARN>(true));
    if (e != cudaSuccess) return e;
    unsigned grid = 0;
    e = persistent_grid(reinterpret_cast<const void *>(kern), nw * 32, smem, static_cast<uint64_t>(nw) * 32, a.nq,
                        &grid, t.corun_descent_bps);
    if (e != cudaSuccess) return e;
    return launch_with_window(kern, grid, nw * 32, smem, s, a.tree, t, static_cast<const RawOf<K> *>(a.q), a.qidx,
                              static_cast<const PartRec<K> *>(a.recs), a.nq, static_cast<V *>(a.out_v), a.out_f,
                              a.fetch, md, a.lstats, first_wait_polls());
}

template <typename K, typename V, int M>
static cudaError_t pipe_mode(const DescendArgs &a, cudaStream_t s)
{
    // A small batch searched as given: its chunks meet up to 32 leaves, more
    // than the slots, and rank the rest through L1.  From about 16 chunks per
    // SM the prefetched lines no longer stay in L1 until they are read (at
    // 2^20 queries on a 10^6-key tree: 67 us against 61 with the further
    // rounds), so larger batches keep the rounds.
    int sms = 0;
    const cudaError_t e = dev_sm_count(&sms);
    if (e != cudaSuccess) return e;
    const bool tail_l1 =
        !a.recs && !a.qidx && (a.nq + 31) / 32 <= 16ull * static_cast<uint64_t>(sms > 0 ? sms : 1);
    if constexpr (!std::is_same<K, Key32>::value) {
        if (a.md) {
            // PL windows on skewed keys span many leaves read through L1, and
            // the L1 path for the leaves cost them a step at batch 1024 (12.3
            // -> 14.3 us on lognormal keys); the MLP's gained (22.5 -> 18.4 us)
            if (a.md->kind == kModelPL) return launch_pipe<K, V, M, false, kModelPL>(a, s);
            return tail_l1 ? launch_pipe<K, V, M, false, kModelMLP, true>(a, s)
                           : launch_pipe<K, V, M, false, kModelMLP>(a, s);
        }
    }
    if (a.fetch) return launch_pipe<K, V, M, true, kModelNone>(a, s);
    if (tail_l1) return launch_pipe<K, V, M, false, kModelNone, true>(a, s);
    return launch_pipe<K, V, M, false, kModelNone>(a, s);
}

template <typename K, typename V>
static cudaError_t pipe_m(const DescendArgs &a, cudaStream_t s)
{
    switch (a.t->m) {
    case 8: return pipe_mode<K, V, 8>(a, s);
    case 16: return pipe_mode<K, V, 16>(a, s);
    case 32: return pipe_mode<K, V, 32>(a, s);
    default: return pipe_mode<K, V, 64>(a, s);
    }
}

cudaError_t descend_pipelined(const DescendArgs &a, cudaStream_t s)
{
    const DevTree &t = *a.t;
    if (t.key_bytes == 8) return t.val_bytes == 8 ? pipe_m<uint64_t, uint64_t>(a, s) : pipe_m<uint64_t, uint32_t>(a, s);
    if (t.key_bytes == 32) return t.val_bytes == 8 ? pipe_m<Key32, uint64_t>(a, s) : pipe_m<Key32, uint32_t>(a, s);
    return t.val_bytes == 8 ? pipe_m<uint32_t, uint64_t>(a, s) : pipe_m<uint32_t, uint32_t>(a, s);
}

cudaError_t take_wait_counters_pipelined(unsigned *timeouts, unsigned *pending)
{
    return take_wait_counters(timeouts, pending);
}

}  // namespace btgb
