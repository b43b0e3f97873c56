// On-device partition of the query batch by approximate key rank.
//
// The paper sorts the query batch so that all queries routed to one node
// are adjacent and served by one node fetch (Sec. IV-A, Sec. IV-E).  What
// the warp-level descent needs is that each run of 32 consecutive queries
// covers as narrow a key range as a sorted batch would.  A two-level
// counting sort on a bucket number that is monotone in the key gives that:
//
//   f(q) = (c << r) | s      (or c >> cshift when fewer bits are asked for
//                               than c has), on `bits` bits in all
//     c  = how many of the tree's splitters are smaller than q.  The
//          splitters are the largest keys of evenly spaced leaves (at most
//          kSplitSlots of them, built with the tree), so c is q's rank among
//          the keys to within one segment, whatever the key distribution;
//     s  = q's position inside segment c on r bits, by linear interpolation
//          between the segment's bounds (fp32; monotone in q).  32-byte keys
//          interpolate on the 8 bytes that follow the bytes the segment's
//          bounds (hence all its keys) share.
//   coarse(q) = f(q) >> lb,   digit(q) = f(q) & (2^lb - 1).
//
// One cooperative launch, k_partition (every block resident; two bounded
// grid barriers), with the batch cut into one slice per block:
//   count     the slice's coarse buckets in shared memory, added to global
//             totals with one atomic per bucket whose return value is the
//             block's offset inside that bucket;
//   scatter   bucket starts by a scan of the totals; every query goes to its
//             block's run in its bucket, at its rank there (taken while
//             counting), as one record (key, input position, digit) -- for
//             32-byte keys as an 8-byte (position, digit) pair;
//   sort      groups of threads order the coarse buckets by digit, in
//             place (32-byte keys: from the pairs into an array of the keys
//             and an array of their positions, each key read from the batch
//             once and written as one 32-byte sector), several buckets per
//             block at once.  Buckets of more
//             than part_tile<K>() queries (a hot key, or a coarse bucket far
//             above its average size) keep the scatter's order.
//
// Result: the batch ordered by coarse bucket, and inside every coarse bucket
// of at most part_tile<K>() queries by f; queries with equal f (and in the
// larger buckets, equal coarse buckets) come in an unspecified order.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "keys.cuh"

namespace btgb {

constexpr int kSplitSlots = 1023;   // splitters per tree, at most
constexpr int kRadixBits = 12;      // pre-index of the splitters by leading key bits
constexpr int kMaxCoarseBits = 12;  // coarse buckets: at most 2^12 counters in shared memory
constexpr int kLocalBits = 9;       // digit bits of the local sort: 2^9 counters
constexpr int kMaxPartBits = kMaxCoarseBits + kLocalBits;
constexpr int kPartThreads = 512;
// The local sort: groups of kSortThreads threads, each ordering one coarse
// bucket at a time.
constexpr int kSortThreads = 128;
constexpr int kSortGroups = kPartThreads / kSortThreads;

// Largest coarse bucket the local sort orders (one group of threads, the
// bucket's records in registers; larger buckets, a hot key, keep the
// scatter's order).
template <typename K>
__host__ __device__ constexpr int part_tile()
{
    return 1024;
}

// 32-byte keys scatter 8-byte (position, digit) pairs instead of 48-byte
// records; the local sort writes each query's record once, in its final
// place, reading the key from the batch.
template <typename K>
__host__ __device__ constexpr bool part_narrow()
{
    return sizeof(RawOf<K>) > 8;
}

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
    int cshift;             // with r == 0: f = c >> cshift (fewer bits than c has)
    int lb;                 // digit bits: coarse = f >> lb
    float scale;            // 2^r
};

// Shared-memory copy of the splitters, padded with all-ones keys so that a
// branchless binary search of ten probes finds c.
template <typename K>
struct __align__(16) PartSmem {
    K sp[kSplitSlots + 1];
    float inv[kSplitSlots + 1];
    unsigned char off[kSplitSlots + 1];
    uint16_t R[(1 << kRadixBits) + 8];  // whole 16-byte pieces
    uint32_t scan_tmp[32];
    uint32_t last;
};

__device__ __forceinline__ void part_cp_async16(void *smem_dst, const void *gsrc)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}

// Copy the splitter tables to shared memory in one round of 16-byte
// asynchronous copies (every table starts on a 256-byte boundary of the
// tree image, and the image pads each to the next such boundary, so whole
// 16-byte pieces stay inside it), then pad the splitters beyond nsplit with
// all-ones keys.  Ends with a block barrier.
template <typename K>
__device__ __forceinline__ void part_load_tables(PartSmem<K> &S, const PartNorm<K> &pn)
{
    const uint32_t ns = pn.nsplit;
    const uint32_t sp_pieces = (ns * static_cast<uint32_t>(sizeof(K)) + 15u) / 16u;
    const uint32_t inv_pieces = ((ns + 1u) * 4u + 15u) / 16u;
    const uint32_t off_pieces = pn.split_off ? ((ns + 1u) + 15u) / 16u : 0u;
    const uint32_t r_pieces = pn.split_R ? (((1u << kRadixBits) + 1u) * 2u + 15u) / 16u : 0u;
    const uint32_t total = sp_pieces + inv_pieces + off_pieces + r_pieces;
    for (uint32_t i = threadIdx.x; i < total; i += blockDim.x) {
        uint32_t j = i;
        if (j < sp_pieces) {
            part_cp_async16(reinterpret_cast<unsigned char *>(S.sp) + 16 * j,
                            reinterpret_cast<const unsigned char *>(pn.split) + 16 * j);
            continue;
        }
        j -= sp_pieces;
        if (j < inv_pieces) {
            part_cp_async16(reinterpret_cast<unsigned char *>(S.inv) + 16 * j,
                            reinterpret_cast<const unsigned char *>(pn.split_inv) + 16 * j);
            continue;
        }
        j -= inv_pieces;
        if (j < off_pieces) {
            part_cp_async16(S.off + 16 * j, pn.split_off + 16 * j);
            continue;
        }
        j -= off_pieces;
        part_cp_async16(reinterpret_cast<unsigned char *>(S.R) + 16 * j,
                        reinterpret_cast<const unsigned char *>(pn.split_R) + 16 * j);
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    for (uint32_t i = ns + threadIdx.x; i <= static_cast<uint32_t>(kSplitSlots); i += blockDim.x)
        S.sp[i] = KeyOps<K>::ones();
    __syncthreads();
}

// f(q) for integer keys.
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
            if (mem_lt(S.sp + mid, q))
                lo = mid + 1;
            else
                hi = mid;
        }
        c = lo;
    } else {
        c = 0;
#pragma unroll
        for (uint32_t h = (kSplitSlots + 1) / 2; h >= 1; h >>= 1)
            if (mem_lt(S.sp + c + h - 1, q)) c += h;
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

// f(q) for 32-byte keys.
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
                if (mem_lt(S.sp + mid, q))
                    lo = mid + 1;
                else
                    hi = mid;
            }
            c = lo;
        }
    } else {
#pragma unroll
        for (uint32_t h = (kSplitSlots + 1) / 2; h >= 1; h >>= 1)
            if (mem_lt(S.sp + c + h - 1, q)) c += h;
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

// In-place exclusive scan of n counters in shared memory (n a multiple of
// 4, at most 8 * blockDim.x); every thread of the block must call it.
__device__ __forceinline__ void part_scan_smem(uint32_t *cnt, uint32_t n, uint32_t *tmp)
{
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;  // at most 8
    const uint32_t j0 = threadIdx.x * per;
    uint32_t v[8];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t j = j0 + k;
        v[k] = (static_cast<uint32_t>(k) < per && j < n) ? cnt[j] : 0u;
        sum += v[k];
    }
    uint32_t run = part_block_excl_scan(sum, tmp);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t j = j0 + k;
        if (static_cast<uint32_t>(k) < per && j < n) {
            cnt[j] = run;
            run += v[k];
        }
    }
    __syncthreads();
}

// Blocks of the partition, at most.
constexpr uint32_t kMaxPartBlocks = 1024;

// Bounded waits of the partition's grid barrier that gave up (the results of
// that search are invalid); read and cleared by bt_check_timeouts.
static __device__ unsigned int g_part_timeouts;

// Queries of its slice a partition block keeps in shared memory between
// counting and scattering: f and the query's rank in its bucket, and for
// integer keys the key itself (32-byte keys are read again).
template <typename K>
__host__ __device__ constexpr uint32_t part_cache()
{
    return 4096u;
}

template <typename K>
__host__ __device__ constexpr bool part_cache_keys()
{
    return sizeof(RawOf<K>) <= 8;
}

template <typename K>
__host__ __device__ constexpr int part_cache_key_bytes()
{
    return part_cache_keys<K>() ? static_cast<int>(sizeof(RawOf<K>)) : 0;
}

// Dynamic shared memory of k_partition for nb coarse buckets: the block's
// counts / next positions (nb words), the bucket starts (nb + 4 words), then
// an area holding first the cached slice (keys, then f, then each query's
// rank among the slice's queries of its bucket) and later every sort group's
// digit counters.
template <typename K>
__host__ __device__ constexpr int part_area()
{
    return static_cast<int>(part_cache<K>()) * (part_cache_key_bytes<K>() + 6) > kSortGroups * ((1 << kLocalBits) + 8) * 4
               ? static_cast<int>(part_cache<K>()) * (part_cache_key_bytes<K>() + 6)
               : kSortGroups * ((1 << kLocalBits) + 8) * 4;
}

template <typename K>
__host__ __device__ constexpr int part_dyn(uint32_t nb)
{
    return static_cast<int>((nb + (nb + 4)) * 4u) + part_area<K>();
}

// A record read through L2 (written by another block of the same launch).
template <typename K>
__device__ __forceinline__ PartRec<K> ld_rec_cg(const PartRec<K> *p)
{
    static_assert(sizeof(PartRec<K>) % 16 == 0, "records are whole 16-byte pieces");
    PartRec<K> r;
    const uint4 *src = reinterpret_cast<const uint4 *>(p);
    uint4 *dst = reinterpret_cast<uint4 *>(&r);
#pragma unroll
    for (int i = 0; i < static_cast<int>(sizeof(PartRec<K>) / 16); ++i) dst[i] = __ldcg(src + i);
    return r;
}

// Grid-wide barrier of a cooperative launch (every block resident): thread 0
// counts its block's arrival on *ctr (zero before the launch) and waits, at
// most `polls` polls, until all gridDim.x blocks have arrived.  False if the
// wait gave up.
__device__ __forceinline__ bool part_grid_sync(unsigned int *ctr, uint32_t polls, uint32_t *flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        uint32_t ok = 0;
        for (uint32_t i = 0; i < polls; ++i) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
            if (v >= gridDim.x) {
                ok = 1;
                break;
            }
            __nanosleep(32);
        }
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

// Named barrier of sort group g (ids 1.. ; 0 is __syncthreads).
__device__ __forceinline__ void part_group_sync(uint32_t g)
{
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kSortThreads) : "memory");
}

// In-place exclusive scan of n counters (a multiple of 4, at most
// 8 * kSortThreads) by one sort group; tmp holds a word per warp of the group.
__device__ __forceinline__ void part_group_scan(uint32_t *cnt, uint32_t n, uint32_t *tmp, uint32_t g, uint32_t gtid)
{
    const uint32_t lane = gtid & 31, w = gtid >> 5;
    const uint32_t per = (n + kSortThreads - 1) / kSortThreads;
    const uint32_t j0 = gtid * per;
    uint32_t v[8];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t j = j0 + k;
        v[k] = (static_cast<uint32_t>(k) < per && j < n) ? cnt[j] : 0u;
        sum += v[k];
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= static_cast<uint32_t>(o)) x += y;
    }
    if (lane == 31) tmp[w] = x;
    part_group_sync(g);
    uint32_t run = x - sum;
    for (uint32_t k = 0; k < w; ++k) run += tmp[k];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t j = j0 + k;
        if (static_cast<uint32_t>(k) < per && j < n) {
            cnt[j] = run;
            run += v[k];
        }
    }
    part_group_sync(g);
}

// The whole partition in one cooperative launch; block g owns slice g of
// the batch (ceil(nq / gridDim.x) queries).
//   1. Count the slice's coarse buckets in shared memory (keeping each key,
//      its f and its rank among the slice's queries of its bucket -- the
//      counting atomic's return value -- in shared memory when the slice
//      fits part_cache).
//   2. Add every count to total[j] (nb words, zero on entry) with one atomic
//      whose return value -- the bucket's queries counted by blocks whose
//      atomic came first -- is the block's offset inside bucket j.
//   -- grid barrier on total[nb] --
//   3. Bucket starts: the exclusive scan of the totals (every block); the
//      block's next position in bucket j is start[j] + offset[j].
//   4. Every query of the slice goes to the block's next position in its
//      bucket plus its rank (or, uncached, the bucket's next position from a
//      shared-memory atomic) and is written there as one record.
//   -- grid barrier on total[nb + 1] --
//   5. Local sort, in place: groups of kSortThreads threads order the
//      coarse buckets of at most part_tile records by digit, one bucket per
//      group at a time (records in registers, ranks among equal digits from
//      shared-memory atomics, a scan of the digit counts).
// A barrier that gives up is counted (g_part_timeouts) and its block
// stops; that search's results are then invalid.
template <typename K>
__global__ void __launch_bounds__(kPartThreads, 2) k_partition(const RawOf<K> *__restrict__ q, uint64_t nq,
                                                               PartNorm<K> pn, unsigned int *__restrict__ total,
                                                               uint32_t nb, PartRec<K> *__restrict__ rec,
                                                               uint2 *__restrict__ pairs,
                                                               RawOf<K> *__restrict__ out_q,
                                                               uint32_t *__restrict__ out_i, uint32_t polls)
{
    __shared__ PartSmem<K> S;
    extern __shared__ __align__(16) unsigned char dsm[];
    constexpr int U = 4;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(dsm);
    uint32_t *st = cnt + nb;
    unsigned char *area = reinterpret_cast<unsigned char *>(st + nb + 4);  // nb is a multiple of 4
    RawOf<K> *ck = reinterpret_cast<RawOf<K> *>(area);
    uint32_t *cf = reinterpret_cast<uint32_t *>(area + part_cache<K>() * part_cache_key_bytes<K>());
    uint16_t *cr = reinterpret_cast<uint16_t *>(cf + part_cache<K>());
    part_load_tables(S, pn);
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) cnt[j] = 0;
    __syncthreads();
    const uint64_t per = (nq + gridDim.x - 1) / gridDim.x;
    const uint64_t s0 = blockIdx.x * per < nq ? blockIdx.x * per : nq;
    const uint64_t s1 = s0 + per < nq ? s0 + per : nq;
    const uint32_t ns = static_cast<uint32_t>(s1 - s0);
    const bool cached = ns <= part_cache<K>();

    // 1. counts
    for (uint32_t i0 = threadIdx.x; i0 < ns; i0 += U * blockDim.x) {
        RawOf<K> key[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t i = i0 + u * blockDim.x;
            if (i < ns) key[u] = q[s0 + i];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t i = i0 + u * blockDim.x;
            if (i < ns) {
                const uint32_t f = part_bucket(S, pn, KeyOps<K>::from_raw(key[u]));
                if (cached) {
                    // the query's rank in its bucket within the slice: its
                    // place in the bucket's run, so the scatter needs no atomics
                    if constexpr (part_cache_keys<K>()) ck[i] = key[u];
                    cf[i] = f;
                    cr[i] = static_cast<uint16_t>(atomicAdd(cnt + (f >> pn.lb), 1u));
                } else {
                    atomicAdd(cnt + (f >> pn.lb), 1u);
                }
            }
        }
    }
    __syncthreads();
    // 2. offsets: all of a thread's atomics are issued before any result is used
    {
        constexpr int RPT = (1 << kMaxCoarseBits) / kPartThreads;
        uint32_t cv[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const uint32_t j = threadIdx.x + k * blockDim.x;
            cv[k] = j < nb ? cnt[j] : 0u;
        }
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            if (cv[k]) cv[k] = atomicAdd(total + threadIdx.x + k * blockDim.x, cv[k]);
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const uint32_t j = threadIdx.x + k * blockDim.x;
            if (j < nb) cnt[j] = cv[k];
        }
    }
    if (!part_grid_sync(total + nb, polls, &S.last)) {
        if (threadIdx.x == 0) atomicAdd(&g_part_timeouts, 1u);
        return;
    }
    // 3. bucket starts and the block's next positions
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) st[j] = __ldcg(total + j);
    __syncthreads();
    part_scan_smem(st, nb, S.scan_tmp);
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) cnt[j] += st[j];
    if (threadIdx.x == 0) st[nb] = static_cast<uint32_t>(nq);
    __syncthreads();
    // 4. records
    const uint32_t dmask = (1u << pn.lb) - 1u;
    for (uint32_t i0 = threadIdx.x; i0 < ns; i0 += U * blockDim.x) {
        RawOf<K> key[U];
        uint32_t f[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t i = i0 + u * blockDim.x;
            if (i < ns) {
                if (cached) {
                    if constexpr (part_cache_keys<K>())
                        key[u] = ck[i];
                    else if constexpr (!part_narrow<K>())
                        key[u] = q[s0 + i];
                    f[u] = cf[i];
                } else {
                    key[u] = q[s0 + i];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t i = i0 + u * blockDim.x;
            if (i < ns) {
                if (!cached) f[u] = part_bucket(S, pn, KeyOps<K>::from_raw(key[u]));
                const uint32_t pos = cached ? cnt[f[u] >> pn.lb] + cr[i] : atomicAdd(cnt + (f[u] >> pn.lb), 1u);
                if (pos < nq) {  // always true when the counts agree; keeps a stray write in bounds
                    if constexpr (part_narrow<K>()) {
                        pairs[pos] = make_uint2(static_cast<uint32_t>(s0 + i), f[u] & dmask);
                    } else {
                        PartRec<K> r;
                        r.key = key[u];
                        r.idx = static_cast<uint32_t>(s0 + i);
                        r.digit = f[u] & dmask;
                        rec[pos] = r;
                    }
                }
            }
        }
    }
    if (pn.lb == 0 && !part_narrow<K>()) return;
    if (!part_grid_sync(total + nb + 1, polls, &S.last)) {
        if (threadIdx.x == 0) atomicAdd(&g_part_timeouts, 1u);
        return;
    }
    // the next kernel (the descent) may start launching; it waits for this
    // grid to finish before it reads the records
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // 5. local sorts, in place: the block's threads form kSortGroups groups
    // of kSortThreads, each ordering one coarse bucket of at most part_tile
    // records at a time by digit (records in registers, ranks among equal
    // digits from shared-memory atomics, a scan of the digit counts; the
    // group synchronises on its own named barrier).  Buckets go to the
    // groups group-major (bucket b to group b / gridDim.x of block
    // b % gridDim.x, then round after round), so that the buckets beyond the
    // first round spread over all blocks, and so over all SMs.
    const uint32_t nd = 1u << pn.lb;
    const uint32_t nscan = nd < 4 ? 4 : nd;  // the scan works on groups of 4 counters
    const uint32_t grp = threadIdx.x / kSortThreads, gtid = threadIdx.x % kSortThreads;
    uint32_t *gb = reinterpret_cast<uint32_t *>(area) + grp * ((1 << kLocalBits) + 8);
    uint32_t *gtmp = gb + (1 << kLocalBits);  // per-warp partial sums of the group's scan
    constexpr int EL = part_tile<K>() / kSortThreads;
    if constexpr (part_narrow<K>()) {
        // every bucket's pairs become keys and positions: sorted by digit
        // when the bucket fits the tile, else in scatter order
        for (uint32_t b = grp * gridDim.x + blockIdx.x; b < nb; b += gridDim.x * kSortGroups) {
            const uint32_t bs = st[b];
            const uint32_t n = st[b + 1] - bs;
            if (n == 0) continue;
            if (n > static_cast<uint32_t>(part_tile<K>()) || pn.lb == 0) {
                for (uint32_t i = gtid; i < n; i += kSortThreads) {
                    const uint2 pr = __ldcg(pairs + bs + i);
                    out_q[bs + i] = q[pr.x];
                    out_i[bs + i] = pr.x;
                }
                continue;
            }
            for (uint32_t j = gtid; j < nscan; j += kSortThreads) gb[j] = 0;
            part_group_sync(grp);
            uint2 pr[EL];
            uint32_t rk[EL];
#pragma unroll
            for (int e = 0; e < EL; ++e) {
                const uint32_t i = gtid + e * kSortThreads;
                if (i < n) pr[e] = __ldcg(pairs + bs + i);
            }
#pragma unroll
            for (int e = 0; e < EL; ++e) {
                const uint32_t i = gtid + e * kSortThreads;
                if (i < n) rk[e] = atomicAdd(gb + (pr[e].y & (nd - 1u)), 1u);
            }
            part_group_sync(grp);
            part_group_scan(gb, nscan, gtmp, grp, gtid);
#pragma unroll
            for (int e = 0; e < EL; ++e) {
                const uint32_t i = gtid + e * kSortThreads;
                if (i < n) {
                    const uint32_t p = gb[pr[e].y & (nd - 1u)] + rk[e];
                    if (p < n) {  // always true; keeps a stray write inside the bucket
                        out_q[bs + p] = q[pr[e].x];
                        out_i[bs + p] = pr[e].x;
                    }
                }
            }
            part_group_sync(grp);
        }
        return;
    }
    for (uint32_t b = grp * gridDim.x + blockIdx.x; b < nb; b += gridDim.x * kSortGroups) {
        const uint32_t bs = st[b];
        const uint32_t n = st[b + 1] - bs;
        if (n <= 1 || n > static_cast<uint32_t>(part_tile<K>())) continue;  // the same for the whole group
        for (uint32_t j = gtid; j < nscan; j += kSortThreads) gb[j] = 0;
        part_group_sync(grp);
        PartRec<K> r[EL];
        uint32_t rk[EL];
#pragma unroll
        for (int e = 0; e < EL; ++e) {
            const uint32_t i = gtid + e * kSortThreads;
            if (i < n) r[e] = ld_rec_cg(rec + bs + i);
        }
#pragma unroll
        for (int e = 0; e < EL; ++e) {
            const uint32_t i = gtid + e * kSortThreads;
            if (i < n) rk[e] = atomicAdd(gb + (r[e].digit & (nd - 1u)), 1u);
        }
        part_group_sync(grp);
        part_group_scan(gb, nscan, gtmp, grp, gtid);
#pragma unroll
        for (int e = 0; e < EL; ++e) {
            const uint32_t i = gtid + e * kSortThreads;
            if (i < n) {
                const uint32_t p = gb[r[e].digit & (nd - 1u)] + rk[e];
                if (p < n) rec[bs + p] = r[e];  // always true; keeps a stray write inside the bucket
            }
        }
        part_group_sync(grp);
    }
}

// The records split into a key array and a position array (bt_sort_batch,
// integer keys).
template <typename K>
__global__ void k_part_unpack(const PartRec<K> *__restrict__ rec, uint64_t nq, RawOf<K> *__restrict__ out_q,
                              uint32_t *__restrict__ out_i)
{
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < nq;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const PartRec<K> r = rec[i];
        out_q[i] = r.key;
        out_i[i] = r.idx;
    }
}

}  // namespace btgb
