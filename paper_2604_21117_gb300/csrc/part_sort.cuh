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
//   k_part_count    per query: its bucket; warp-aggregated atomic counts
//                   (equal buckets within a warp are counted once, so a hot
//                   key costs one atomic per warp).  The last block to finish
//                   (a ticket counter, no waiting) turns the counts into
//                   exclusive bucket starts.
//   k_part_scatter  per query: a slot in its bucket from a warp-aggregated
//                   atomic cursor; the query and its input position are
//                   written there.
//
// Result: the batch ordered by bucket; the order of queries within one
// bucket is unspecified (it depends on the order of the atomics).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "keys.cuh"

namespace btgb {

constexpr int kSplitSlots = 1023;   // splitters per tree, at most
constexpr int kSplitBits = 10;      // bits of c with the full table
constexpr int kMaxPartBits = 16;    // bucket bits, at most (2^16 counters)
constexpr int kPartThreads = 1024;
constexpr int kPartUnroll = 4;

// Per-search view of the tree's splitter table.
template <typename K>
struct PartNorm {
    const K *split;         // nsplit splitters, ascending (device)
    const float *split_inv; // nsplit + 1 reciprocal segment widths (device)
    const unsigned char *split_off;  // 32-byte keys: per segment, bytes its keys share
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
}

template <typename K>
__device__ __forceinline__ uint32_t part_bucket(const PartSmem<K> &S, const PartNorm<K> &pn, K q)
{
    uint32_t c = 0;
#pragma unroll
    for (uint32_t h = (kSplitSlots + 1) / 2; h >= 1; h >>= 1)
        if (S.sp[c + h - 1] < q) c += h;
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
#pragma unroll
    for (uint32_t h = (kSplitSlots + 1) / 2; h >= 1; h >>= 1)
        if (S.sp[c + h - 1] < q) c += h;
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

// counts[0..nb) must be zero and counts[nb] (the ticket) zero on entry; on
// exit counts[b] is the first position of bucket b.  nb is a multiple of 4.
template <typename K>
__global__ void __launch_bounds__(kPartThreads) k_part_count(const RawOf<K> *__restrict__ q, uint64_t nq, PartNorm<K> pn,
                                                             uint32_t *__restrict__ counts, uint32_t nb)
{
    __shared__ PartSmem<K> S;
    part_load_tables(S, pn);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i0 = static_cast<uint64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u); i0 < nq;
         i0 += stride * kPartUnroll) {
        RawOf<K> key[kPartUnroll];
#pragma unroll
        for (int u = 0; u < kPartUnroll; ++u) {
            const uint64_t i = i0 + u * stride + lane;
            if (i < nq) key[u] = q[i];
        }
#pragma unroll
        for (int u = 0; u < kPartUnroll; ++u) {
            const uint64_t i = i0 + u * stride + lane;
            const unsigned vm = __ballot_sync(0xffffffffu, i < nq);
            if (i < nq) {
                const uint32_t b = part_bucket(S, pn, KeyOps<K>::from_raw(key[u]));
                const unsigned same = __match_any_sync(vm, b);
                if ((same & part_lanemask_lt()) == 0) atomicAdd(counts + b, static_cast<uint32_t>(__popc(same)));
            }
        }
    }
    // The last block to get here scans the counts (all other blocks' atomics
    // are visible to it after their fences and its ticket).
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) S.last = (atomicAdd(counts + nb, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!S.last) return;
    __threadfence();
    const uint32_t per = (nb / 4 + blockDim.x - 1) / blockDim.x;  // uint4 groups per thread
    uint4 *c4 = reinterpret_cast<uint4 *>(counts);
    const uint32_t g0 = threadIdx.x * per;
    uint32_t sum = 0;
#pragma unroll 4
    for (uint32_t g = g0; g < g0 + per && g < nb / 4; ++g) {
        const uint4 v = __ldcg(c4 + g);
        sum += v.x + v.y + v.z + v.w;
    }
    uint32_t run = part_block_excl_scan(sum, S.scan_tmp);
    for (uint32_t g = g0; g < g0 + per && g < nb / 4; ++g) {
        uint4 v = __ldcg(c4 + g);
        const uint32_t a = run, b = a + v.x, c = b + v.y, d = c + v.z;
        run = d + v.w;
        v.x = a;
        v.y = b;
        v.z = c;
        v.w = d;
        c4[g] = v;
    }
}

template <typename K>
__global__ void __launch_bounds__(kPartThreads) k_part_scatter(const RawOf<K> *__restrict__ q, uint64_t nq,
                                                               PartNorm<K> pn, uint32_t *__restrict__ cursor,
                                                               RawOf<K> *__restrict__ out_q,
                                                               uint32_t *__restrict__ out_i)
{
    __shared__ PartSmem<K> S;
    part_load_tables(S, pn);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i0 = static_cast<uint64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u); i0 < nq;
         i0 += stride * kPartUnroll) {
        RawOf<K> key[kPartUnroll];
#pragma unroll
        for (int u = 0; u < kPartUnroll; ++u) {
            const uint64_t i = i0 + u * stride + lane;
            if (i < nq) key[u] = q[i];
        }
#pragma unroll
        for (int u = 0; u < kPartUnroll; ++u) {
            const uint64_t i = i0 + u * stride + lane;
            const unsigned vm = __ballot_sync(0xffffffffu, i < nq);
            if (i < nq) {
                const uint32_t b = part_bucket(S, pn, KeyOps<K>::from_raw(key[u]));
                const unsigned same = __match_any_sync(vm, b);
                const int leader = __ffs(same) - 1;
                uint32_t base = 0;
                if (lane == leader) base = atomicAdd(cursor + b, static_cast<uint32_t>(__popc(same)));
                base = __shfl_sync(vm, base, leader);
                const uint32_t pos = base + __popc(same & part_lanemask_lt());
                out_q[pos] = key[u];
                out_i[pos] = static_cast<uint32_t>(i);
            }
        }
    }
}

}  // namespace btgb
