// On-device partition of the query batch by approximate key rank.
//
// The paper sorts the query batch so that all queries routed to one node
// are adjacent and served by one node fetch (Sec. IV-A, Sec. IV-E).  What
// the warp-level descent needs is weaker: each run of 32 consecutive
// queries should cover a narrow key range.  A counting sort on a bucket
// number that is monotone in the key gives that in two passes over the
// batch:
//
//   bucket(q) = (c << r) | s      (or c >> cshift when fewer bits are asked
//                                   for than c has)
//     c  = how many of the tree's splitters are smaller than q.  The
//          splitters are the largest keys of evenly spaced leaves (at most
//          kSplitSlots of them, built with the tree), so c is q's rank among
//          the keys to within one segment, whatever the key distribution;
//     s  = q's position inside segment c on r bits, by linear interpolation
//          between the segment's bounds (fp32; monotone in q).  32-byte keys
//          interpolate on the 8 bytes that follow the bytes the segment's
//          bounds (hence all its keys) share.
//
//   k_part_hist     per block, the bucket counts of a slice of the batch in
//                   shared memory, added to the global totals once per
//                   non-zero bucket (a hot key costs one global atomic per
//                   block); the last block to finish (a ticket counter, no
//                   waiting) turns the totals into exclusive bucket starts.
//   k_part_scatter  per block and round of queries: shared-memory bucket
//                   counts, one global atomic per non-zero bucket to
//                   reserve its run, then each query's slot in the run from
//                   a shared-memory atomic; the query and its input position
//                   are written there.
//
// Result: the batch ordered by bucket; the order of queries within one
// bucket is unspecified (it depends on the order of the atomics).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "keys.cuh"

namespace btgb {

constexpr int kSplitSlots = 1023;   // splitters per tree, at most
constexpr int kRadixBits = 12;      // pre-index of the splitters by leading key bits
constexpr int kSplitBits = 10;      // bits of c with the full table
constexpr int kMaxPartBits = 13;    // bucket bits, at most (2^13 counters in shared memory)
constexpr int kPartThreads = 1024;

// Per-search view of the tree's splitter table.
template <typename K>
struct PartNorm {
    const K *split;         // nsplit splitters, ascending (device)
    const float *split_inv; // nsplit + 1 reciprocal segment widths (device)
    const unsigned char *split_off;  // 32-byte keys: per segment, bytes its keys share
    const uint16_t *split_R;         // R[j] = splitters whose leading bits are < j
    int rshift;                      // leading bits = (key - kmin) >> rshift
    int p0;                          // 32-byte keys: bytes every key shares; leading bits taken
    uint64_t wmin;                   //   from (8 bytes after them) - (the same of kmin)
    K kmin;                 // smallest key: lower bound of segment 0
    K kmax;                 // largest key: upper bound of the last segment
    uint32_t nsplit;
    int r;                  // interpolation bits within a segment
    int cshift;             // with r == 0: bucket = c >> cshift (fewer bits than c has)
    float scale;            // 2^r
};

// Shared-memory copy of the splitters, padded with all-ones keys so that a
// branchless binary search of kSplitBits probes finds c.
template <typename K>
struct PartSmem {
    K sp[kSplitSlots + 1];
    float inv[kSplitSlots + 1];
    unsigned char off[kSplitSlots + 1];
    uint16_t R[(1 << kRadixBits) + 1];
    uint32_t scan_tmp[32];
    uint32_t last;
};

template <typename K>
__device__ __forceinline__ void part_load_tables(PartSmem<K> &S, const PartNorm<K> &pn)
{
    for (int i = threadIdx.x; i <= kSplitSlots; i += blockDim.x) {
        S.sp[i] = i < static_cast<int>(pn.nsplit) ? pn.split[i] : KeyOps<K>::ones();
        S.inv[i] = i <= static_cast<int>(pn.nsplit) ? pn.split_inv[i] : 0.0f;
        S.off[i] = (pn.split_off && i <= static_cast<int>(pn.nsplit)) ? pn.split_off[i] : 0;
    }
    if (pn.split_R)
        for (int i = threadIdx.x; i <= (1 << kRadixBits); i += blockDim.x) S.R[i] = pn.split_R[i];
}

template <typename K>
__device__ __forceinline__ uint32_t part_bucket(const PartSmem<K> &S, const PartNorm<K> &pn, K q)
{
    uint32_t c;
    if (pn.split_R) {
        // the splitters whose leading bits equal q's bracket c; search only those
        const uint64_t d0 = q > pn.kmin ? static_cast<uint64_t>(q - pn.kmin) : 0ull;
        const uint64_t j64 = d0 >> pn.rshift;
        const uint32_t j = j64 < (1u << kRadixBits) ? static_cast<uint32_t>(j64) : (1u << kRadixBits) - 1u;
        uint32_t lo = S.R[j], hi = S.R[j + 1];
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (S.sp[mid] < q)
                lo = mid + 1;
            else
                hi = mid;
        }
        c = lo;
    } else {
        c = 0;
#pragma unroll
        for (uint32_t h = (kSplitSlots + 1) / 2; h >= 1; h >>= 1)
            if (S.sp[c + h - 1] < q) c += h;
    }
    if (pn.r == 0) return c >> pn.cshift;
    const K lo = c ? S.sp[c - 1] : pn.kmin;
    const float d = q > lo ? static_cast<float>(static_cast<uint64_t>(q - lo)) : 0.0f;
    const float top = pn.scale - 1.0f;
    const float x = fminf(__fmul_rn(__fmul_rn(d, S.inv[c]), pn.scale), top);
    return (c << pn.r) | static_cast<uint32_t>(x);
}

// 8 bytes of a 32-byte key from byte p on (p <= 24), as a big-endian number.
__device__ __forceinline__ uint64_t key32_window(const Key32 &k, int p)
{
    const int j = p >> 3, s = (p & 7) * 8;
    const uint64_t hi = k.w[j];
    const uint64_t lo = j < 3 ? k.w[j + 1] : 0ull;
    return s ? (hi << s) | (lo >> (64 - s)) : hi;
}

__device__ __forceinline__ uint32_t part_bucket(const PartSmem<Key32> &S, const PartNorm<Key32> &pn, const Key32 &q)
{
    uint32_t c = 0;
    if (pn.split_R) {
        if (pn.kmax < q) {
            c = pn.nsplit;
        } else if (!(q < pn.kmin)) {
            // inside [kmin, kmax] every key shares the first p0 bytes, so the
            // next 8 bytes order q among the splitters
            const uint64_t j64 = (key32_window(q, pn.p0) - pn.wmin) >> pn.rshift;
            const uint32_t j = j64 < (1u << kRadixBits) ? static_cast<uint32_t>(j64) : (1u << kRadixBits) - 1u;
            uint32_t lo = S.R[j], hi = S.R[j + 1];
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (S.sp[mid] < q)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            c = lo;
        }
    } else {
#pragma unroll
        for (uint32_t h = (kSplitSlots + 1) / 2; h >= 1; h >>= 1)
            if (S.sp[c + h - 1] < q) c += h;
    }
    if (pn.r == 0) return c >> pn.cshift;
    const uint32_t top = (1u << pn.r) - 1u;
    const Key32 lo = c ? S.sp[c - 1] : pn.kmin;
    if (!(lo < q)) return c << pn.r;
    if (c == pn.nsplit && pn.kmax < q) return (c << pn.r) | top;
    const int p = S.off[c];
    const float d = static_cast<float>(key32_window(q, p) - key32_window(lo, p));
    const float x = fminf(__fmul_rn(__fmul_rn(d, S.inv[c]), pn.scale), static_cast<float>(top));
    return (c << pn.r) | static_cast<uint32_t>(x);
}

__device__ __forceinline__ unsigned part_lanemask_lt()
{
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Block-wide exclusive scan of one value per thread; `tmp` holds 32 words.
__device__ __forceinline__ uint32_t part_block_excl_scan(uint32_t v, uint32_t *tmp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? tmp[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        tmp[lane] = w;
    }
    __syncthreads();
    const uint32_t r = x - v + (warp > 0 ? tmp[warp - 1] : 0u);
    __syncthreads();
    return r;
}

// Queries a block of k_part_scatter holds (in registers) per round.
template <typename K>
constexpr int part_per_thread()
{
    return sizeof(K) > 8 ? 4 : 8;
}

// Bucket histogram.  Each block counts the buckets of one contiguous slice
// of the batch in shared memory (dynamic, nb words), then adds its non-zero
// counts to total[] (nb words, zero on entry).  total[nb] is a ticket (zero
// on entry): the last block to finish turns total[] into exclusive bucket
// starts.  nb is a multiple of 4.
template <typename K>
__global__ void __launch_bounds__(kPartThreads) k_part_hist(const RawOf<K> *__restrict__ q, uint64_t nq, PartNorm<K> pn,
                                                            uint32_t *__restrict__ total, uint32_t nb)
{
    __shared__ PartSmem<K> S;
    extern __shared__ uint32_t cnt[];
    part_load_tables(S, pn);
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) cnt[j] = 0;
    __syncthreads();
    const uint64_t per = (nq + gridDim.x - 1) / gridDim.x;
    const uint64_t s0 = blockIdx.x * per, s1 = s0 + per < nq ? s0 + per : nq;
    constexpr int U = 4;
    for (uint64_t i0 = s0 + threadIdx.x; i0 < s1; i0 += static_cast<uint64_t>(U) * blockDim.x) {
        RawOf<K> key[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t i = i0 + static_cast<uint64_t>(u) * blockDim.x;
            if (i < s1) key[u] = q[i];
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + static_cast<uint64_t>(u) * blockDim.x < s1)
                atomicAdd(cnt + part_bucket(S, pn, KeyOps<K>::from_raw(key[u])), 1u);
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x)
        if (cnt[j]) atomicAdd(total + j, cnt[j]);
    // The last block to get here scans the totals (every other block's adds
    // are visible to it after their fences and its ticket).
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) S.last = (atomicAdd(total + nb, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!S.last) return;
    __threadfence();
    const uint32_t groups = nb / 4;
    const uint32_t per4 = (groups + blockDim.x - 1) / blockDim.x;  // uint4 groups per thread
    uint4 *t4 = reinterpret_cast<uint4 *>(total);
    const uint32_t g0 = threadIdx.x * per4;
    uint4 v[4];  // nb <= 2^13 and 1024 threads: at most 2 groups per thread
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t g = g0 + k;
        v[k] = (k < static_cast<int>(per4) && g < groups) ? __ldcg(t4 + g) : make_uint4(0, 0, 0, 0);
        sum += v[k].x + v[k].y + v[k].z + v[k].w;
    }
    uint32_t run = part_block_excl_scan(sum, S.scan_tmp);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t g = g0 + k;
        if (k < static_cast<int>(per4) && g < groups) {
            const uint32_t a0 = run, a1 = a0 + v[k].x, a2 = a1 + v[k].y, a3 = a2 + v[k].z;
            run = a3 + v[k].w;
            t4[g] = make_uint4(a0, a1, a2, a3);
        }
    }
}

// Scatter.  Each block takes up to part_per_thread * blockDim.x queries
// per round: counts their buckets in shared memory, reserves each
// non-zero bucket's run with one atomic on the global cursor (the bucket
// starts from k_part_hist), then places every query at its run's next slot
// (a shared-memory atomic) and writes it with its input position.
template <typename K>
__global__ void __launch_bounds__(kPartThreads) k_part_scatter(const RawOf<K> *__restrict__ q, uint64_t nq,
                                                               PartNorm<K> pn, uint32_t *__restrict__ cursor,
                                                               uint32_t nb, RawOf<K> *__restrict__ out_q,
                                                               uint32_t *__restrict__ out_i)
{
    __shared__ PartSmem<K> S;
    extern __shared__ uint32_t cnt[];
    constexpr int E = part_per_thread<K>();
    part_load_tables(S, pn);
    const uint64_t round = static_cast<uint64_t>(E) * blockDim.x;
    for (uint64_t base = blockIdx.x * round; base < nq; base += gridDim.x * round) {
        for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) cnt[j] = 0;
        __syncthreads();
        RawOf<K> key[E];
        uint32_t bk[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint64_t i = base + static_cast<uint64_t>(e) * blockDim.x + threadIdx.x;
            if (i < nq) key[e] = q[i];
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint64_t i = base + static_cast<uint64_t>(e) * blockDim.x + threadIdx.x;
            if (i < nq) {
                bk[e] = part_bucket(S, pn, KeyOps<K>::from_raw(key[e]));
                atomicAdd(cnt + bk[e], 1u);
            }
        }
        __syncthreads();
        {
            // reserve every non-zero bucket's run: all of a thread's atomics
            // are issued before any result is used (one round trip)
            constexpr int RPT = (1 << kMaxPartBits) / kPartThreads;
            uint32_t cv[RPT];
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const uint32_t j = threadIdx.x + k * kPartThreads;
                cv[k] = j < nb ? cnt[j] : 0u;
            }
#pragma unroll
            for (int k = 0; k < RPT; ++k)
                if (cv[k]) cv[k] = atomicAdd(cursor + threadIdx.x + k * kPartThreads, cv[k]);
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const uint32_t j = threadIdx.x + k * kPartThreads;
                if (j < nb) cnt[j] = cv[k];
            }
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint64_t i = base + static_cast<uint64_t>(e) * blockDim.x + threadIdx.x;
            if (i < nq) {
                const uint32_t pos = atomicAdd(cnt + bk[e], 1u);
                out_q[pos] = key[e];
                out_i[pos] = static_cast<uint32_t>(i);
            }
        }
        __syncthreads();
    }
}

}  // namespace btgb
