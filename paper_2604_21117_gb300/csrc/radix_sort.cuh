// On-device radix sort of (query, input position) pairs.
//
// The paper sorts the query batch so that all queries routed to one node
// are adjacent and served by one node fetch (Sec. IV-A, Sec. IV-E).  Here
// the sort key is the query's normalised offset above the tree's smallest
// key (see SortNorm); what the descent needs is that each run of 32
// consecutive queries covers a narrow key range, which this two-stage radix
// sort gives at the cost of one global distribution:
//
//   1. MSD distribution on the leading D bits (D = 0..12, about nq/4096
//      buckets, at most 2^20 (bucket, tile) pairs), counting sort style:
//        k_msd_hist     per-tile bucket histograms into a [bucket][tile]
//                       matrix (no atomics);
//        k_msd_offsets  one block: the matrix read bucket-major becomes the
//                       exclusive start of every (bucket, tile) run;
//        k_msd_scatter  per tile: the elements are regrouped by bucket in
//                       shared memory and written as contiguous runs at
//                       their (bucket, tile) starts.
//      No block waits on another (no look-back, no grid barrier).  Runs
//      keep tile order inside a bucket; inside a tile the order of one
//      bucket's elements is that of shared-memory atomics (unspecified).
//   2. k_local_sort: every aligned run of kSortTile positions is sorted
//      in shared memory by the leading `bits` bits (D bucket bits first),
//      stable LSD passes of 8 bits with warp multisplit ranking.
//
// Result: ordered on the leading D bits across the batch, and on the
// leading `bits` bits within every aligned run of kSortTile positions.
// Batches of at most kSortTile queries need only stage 2: a full sort on
// `bits` bits in one launch.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace btgb {

struct SortNorm {
    uint64_t kmin;
    uint64_t range;
    int rl;        // bit length of the key range
    int bits;      // leading bits ordered within a tile
    int dbits;     // leading bits of the global distribution (0 = none)
};

// Leading `nbits` bits of the normalised key: the offset above the smallest
// key, clamped to the key range, as a number with rl bits.  Monotone in q.
template <typename K>
__device__ __forceinline__ uint64_t sort_field(K q, const SortNorm &s, int nbits)
{
    const uint64_t x = static_cast<uint64_t>(q);
    uint64_t nk = (x <= s.kmin) ? 0 : x - s.kmin;
    if (nk > s.range) nk = s.range;
    const int sh = s.rl > nbits ? s.rl - nbits : 0;
    return nbits == 0 ? 0ull : (nk >> sh);
}

__device__ __forceinline__ unsigned sort_lanemask_lt()
{
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

constexpr int kSortTile = 4096;
constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortPerWarp = kSortTile / kSortWarps;  // 256 = 8 rounds of 32
constexpr int kMaxDistBits = 12;
constexpr int kMaxBuckets = 1 << kMaxDistBits;
constexpr uint64_t kMaxBucketTiles = 1ull << 20;  // cap on (bucket, tile) pairs

// Lanes (within `valid`) whose `nbits`-bit digit equals this lane's: the
// warp multisplit by one ballot per digit bit.  Every lane must call it.
__device__ __forceinline__ unsigned warp_match_bits(uint32_t d, unsigned valid, int nbits)
{
    unsigned same = valid;
    for (int b = 0; b < nbits; ++b) {
        const bool bit = (d >> b) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, bit);
        same &= bit ? bal : ~bal;
    }
    return same;
}

// Block-wide exclusive scan of one value per thread; `tmp` holds 32 words.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *tmp)
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
        tmp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const uint32_t r = x - v + (warp > 0 ? tmp[warp - 1] : 0u);
    __syncthreads();
    return r;
}

// ------------------------------------------------------ 1. distribution

// Per-tile bucket histogram, written to counts[bucket * ntiles + tile].
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_msd_hist(const K *__restrict__ q, uint64_t nq, SortNorm sn,
                                                           uint32_t *__restrict__ counts, uint32_t ntiles)
{
    __shared__ uint32_t h[kMaxBuckets];
    const int nb = 1 << sn.dbits;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
    __syncthreads();
    constexpr int R = kSortTile / kSortThreads;
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kSortTile;
    K key[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t pos = base + r * kSortThreads + threadIdx.x;
        if (pos < nq) key[r] = q[pos];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t pos = base + r * kSortThreads + threadIdx.x;
        const bool valid = pos < nq;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        const uint32_t d = valid ? static_cast<uint32_t>(sort_field(key[r], sn, sn.dbits)) : 0u;
        const unsigned same = warp_match_bits(d, vm, sn.dbits);
        if (valid && (same & sort_lanemask_lt()) == 0) atomicAdd(&h[d], __popc(same));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) counts[static_cast<uint64_t>(i) * ntiles + blockIdx.x] = h[i];
}

// One block: the [bucket][tile] count matrix, read bucket-major, becomes the
// exclusive offsets of every (bucket, tile) run.  Each warp owns a
// contiguous segment: it sums it, the warp sums are scanned, then the warp
// walks its segment in rows of 32 (8 rows loaded ahead), scanning each row.
__global__ void __launch_bounds__(1024) k_msd_offsets(uint32_t *__restrict__ counts, uint32_t total)
{
    __shared__ uint32_t tmp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t seg = ((total + nw - 1) / nw + 31) / 32 * 32;
    const uint32_t lo = warp * seg < total ? warp * seg : total;
    const uint32_t hi = lo + seg < total ? lo + seg : total;
    uint32_t sum = 0;
    for (uint32_t i = lo + lane; i < hi; i += 32) sum += counts[i];
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) tmp[warp] = sum;
    __syncthreads();
    uint32_t run = 0;
    for (int w = 0; w < warp; ++w) run += tmp[w];
    constexpr int kAhead = 8;
    for (uint32_t r0 = lo; r0 < hi; r0 += 32 * kAhead) {
        uint32_t v[kAhead];
#pragma unroll
        for (int k = 0; k < kAhead; ++k) {
            const uint32_t i = r0 + 32 * k + lane;
            v[k] = i < hi ? counts[i] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kAhead; ++k) {
            uint32_t x = v[k];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            const uint32_t i = r0 + 32 * k + lane;
            if (i < hi) counts[i] = run + x - v[k];
            run += __shfl_sync(0xffffffffu, x, 31);
        }
    }
}

template <typename K>
struct MsdSmem {
    uint32_t cnt[kMaxBuckets];    // tile bucket counts, then local starts
    uint32_t base[kMaxBuckets];   // reserved global start of the tile's run per bucket
    uint32_t scan_tmp[32];
    K sk[kSortTile];
    uint32_t si[kSortTile];
    uint32_t sd[kSortTile];
};

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_msd_scatter(const K *__restrict__ q, uint64_t nq, SortNorm sn,
                                                              const uint32_t *__restrict__ offsets, uint32_t ntiles,
                                                              K *__restrict__ out_q, uint32_t *__restrict__ out_i)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MsdSmem<K> &S = *reinterpret_cast<MsdSmem<K> *>(smem_raw);
    const int nb = 1 << sn.dbits;
    const int tid = threadIdx.x;
    for (int i = tid; i < nb; i += blockDim.x) S.cnt[i] = 0;
    __syncthreads();
    constexpr int R = kSortTile / kSortThreads;
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kSortTile;
    const uint32_t tile_n = static_cast<uint32_t>(nq - base < kSortTile ? nq - base : kSortTile);
    K key[R];
    uint32_t dig[R], rank[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t pos = base + r * kSortThreads + tid;
        if (pos < nq) key[r] = q[pos];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t pos = base + r * kSortThreads + tid;
        const bool valid = pos < nq;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        dig[r] = valid ? static_cast<uint32_t>(sort_field(key[r], sn, sn.dbits)) : 0u;
        const unsigned same = warp_match_bits(dig[r], vm, sn.dbits);
        const int leader = __ffs(same) - 1;
        uint32_t b0 = 0;
        if (valid && (tid & 31) == leader) b0 = atomicAdd(&S.cnt[dig[r]], __popc(same));
        b0 = __shfl_sync(0xffffffffu, b0, leader < 0 ? 0 : leader);
        if (valid) rank[r] = b0 + __popc(same & sort_lanemask_lt());
    }
    __syncthreads();
    // the tile's range in each bucket (scanned offsets), then local bucket starts
    for (int i = tid; i < nb; i += blockDim.x) S.base[i] = offsets[static_cast<uint64_t>(i) * ntiles + blockIdx.x];
    const int per = (nb + blockDim.x - 1) / blockDim.x;  // at most 8 buckets per thread
    uint32_t c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t sum = 0;
    for (int k = 0; k < per; ++k) {
        const int b = tid * per + k;
        if (b < nb) {
            c[k] = S.cnt[b];
            sum += c[k];
        }
    }
    __syncthreads();
    uint32_t run = block_excl_scan(sum, S.scan_tmp);
    for (int k = 0; k < per; ++k) {
        const int b = tid * per + k;
        if (b < nb) S.cnt[b] = run;
        run += c[k];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t pos = base + r * kSortThreads + tid;
        if (pos < nq) {
            const uint32_t lp = S.cnt[dig[r]] + rank[r];
            S.sk[lp] = key[r];
            S.si[lp] = static_cast<uint32_t>(pos);
            S.sd[lp] = dig[r];
        }
    }
    __syncthreads();
    for (uint32_t i = tid; i < tile_n; i += blockDim.x) {
        const uint32_t d = S.sd[i];
        const uint32_t g = S.base[d] + (i - S.cnt[d]);
        out_q[g] = S.sk[i];
        out_i[g] = S.si[i];
    }
}

// ---------------------------------------------------------- 2. local sort

template <typename K>
struct LocalSmem {
    uint32_t wh[kSortWarps][256];
    uint32_t tstart[256];
    uint32_t scan_tmp[32];
    K sk[2][kSortTile];
    uint32_t si[2][kSortTile];
};

// Sort every aligned run of kSortTile positions by the leading sn.bits bits,
// in place (src == dst allowed) or from src to dst.  iin == nullptr: the
// positions are the identity.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_local_sort(const K *src_q, const uint32_t *src_i, K *dst_q,
                                                             uint32_t *dst_i, uint64_t nq, SortNorm sn)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LocalSmem<K> &S = *reinterpret_cast<LocalSmem<K> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kSortTile;
    const uint32_t n = static_cast<uint32_t>(nq - base < kSortTile ? nq - base : kSortTile);
    {
        constexpr int RL = kSortTile / kSortThreads;  // all loads in flight before the stores
        K kk[RL];
        uint32_t ii[RL];
#pragma unroll
        for (int r = 0; r < RL; ++r) {
            const uint32_t i = r * kSortThreads + tid;
            if (i < n) {
                kk[r] = src_q[base + i];
                ii[r] = src_i ? src_i[base + i] : static_cast<uint32_t>(base + i);
            }
        }
#pragma unroll
        for (int r = 0; r < RL; ++r) {
            const uint32_t i = r * kSortThreads + tid;
            if (i < n) {
                S.sk[0][i] = kk[r];
                S.si[0][i] = ii[r];
            }
        }
    }
    __syncthreads();
    const int passes = (sn.bits + 7) / 8;
    int cur = 0;
    constexpr int R = kSortPerWarp / 32;
    for (int p = 0; p < passes; ++p) {
        const int lo = 8 * p;  // bit offset of this digit within the field
        const int w = sn.bits - lo < 8 ? sn.bits - lo : 8;
        for (int i = tid; i < kSortWarps * 256; i += blockDim.x) (&S.wh[0][0])[i] = 0;
        __syncthreads();
        uint32_t dig[R], rank[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t i = warp * kSortPerWarp + r * 32 + lane;
            const bool valid = i < n;
            const unsigned vm = __ballot_sync(0xffffffffu, valid);
            dig[r] = valid ? static_cast<uint32_t>((sort_field(S.sk[cur][i], sn, sn.bits) >> lo) & ((1u << w) - 1u)) : 0u;
            const unsigned same = warp_match_bits(dig[r], vm, w);
            if (valid) rank[r] = S.wh[warp][dig[r]] + __popc(same & sort_lanemask_lt());
            __syncwarp();
            if (valid && (same & sort_lanemask_lt()) == 0) S.wh[warp][dig[r]] += __popc(same);
            __syncwarp();
        }
        __syncthreads();
        uint32_t tcnt = 0;
        if (tid < 256) {
            for (int ww = 0; ww < kSortWarps; ++ww) {
                const uint32_t v = S.wh[ww][tid];
                S.wh[ww][tid] = tcnt;
                tcnt += v;
            }
        }
        const uint32_t ts = block_excl_scan(tcnt, S.scan_tmp);
        if (tid < 256) S.tstart[tid] = ts;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t i = warp * kSortPerWarp + r * 32 + lane;
            if (i < n) {
                const uint32_t lp = S.tstart[dig[r]] + S.wh[warp][dig[r]] + rank[r];
                S.sk[cur ^ 1][lp] = S.sk[cur][i];
                S.si[cur ^ 1][lp] = S.si[cur][i];
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    for (uint32_t i = tid; i < n; i += blockDim.x) {
        dst_q[base + i] = S.sk[cur][i];
        dst_i[base + i] = S.si[cur][i];
    }
}

template <typename K>
constexpr int msd_smem_bytes()
{
    return static_cast<int>(sizeof(MsdSmem<K>));
}

template <typename K>
constexpr int local_smem_bytes()
{
    return static_cast<int>(sizeof(LocalSmem<K>));
}

}  // namespace btgb
