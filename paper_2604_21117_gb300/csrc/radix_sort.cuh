// On-device stable LSD radix sort of (query, input position) pairs.
//
// The paper sorts the query batch so that all queries routed to one node
// are adjacent and served by one node fetch (Sec. IV-A, Sec. IV-E).  Here
// the sort key is the query's normalised offset above the tree's smallest
// key (see SortNorm), 8 bits per pass, least significant digit first.
//
// Single-pass ("onesweep") organisation, one kernel per digit pass plus one
// histogram kernel for all passes:
//   k_sort_hist      global digit histograms of every pass (one read);
//   k_sort_pass      per tile of kSortTile elements: stable local ranking
//                    (warp match + per-warp counters), publication of the
//                    tile's per-digit counts, decoupled look-back over the
//                    preceding tiles for the digit offsets (Merrill & Garland,
//                    "Single-pass Parallel Prefix Scan with Decoupled
//                    Look-back", 2016), a local reorder in shared memory and
//                    coalesced runs of writes.
// Tiles are claimed in order from an atomic counter, so a tile only ever
// waits on tiles whose blocks are already running.  Every wait is bounded:
// after kLookbackSpinLimit polls the block records BT_ERR_TIMEOUT in the
// workspace error word and carries on (the output is then wrong, and the
// error is reported by bt_workspace_status).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace btgb {

struct SortNorm {
    uint64_t kmin;
    uint64_t range;
    int shift;
    int passes;
};

// Normalised sort digit of a query: its offset above the smallest key,
// clamped to the key range, shifted so the used leading bits remain.
// Monotone in the query, so ordering by it agrees with the key order.
template <typename K>
__device__ __forceinline__ uint32_t sort_digit(K q, const SortNorm &s, int pass)
{
    const uint64_t x = static_cast<uint64_t>(q);
    uint64_t nk = (x <= s.kmin) ? 0 : x - s.kmin;
    if (nk > s.range) nk = s.range;
    return static_cast<uint32_t>((nk >> (s.shift + 8 * pass)) & 0xFFu);
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
constexpr int kMaxPasses = 8;
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagIncl = 2ull << 62;
constexpr uint32_t kLookbackSpinLimit = 1u << 24;  // with a 64 ns back-off: about a second
constexpr int kLookbackWindow = 16;

// Lanes (within `valid`) whose 8-bit digit equals this lane's: the warp
// multisplit by eight ballots, one per digit bit.  Every lane of the warp
// must call it.
__device__ __forceinline__ unsigned warp_match8(uint32_t d, unsigned valid)
{
    unsigned same = valid;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, bit);
        same &= bit ? bal : ~bal;
    }
    return same;
}

// Workspace block used by the sort besides the ping-pong buffers:
//   ghist[kMaxPasses][256] u32 | tile_ctr[kMaxPasses] u32 | err u32 | status
struct SortMeta {
    uint32_t *ghist;
    uint32_t *tile_ctr;
    uint32_t *err;
    unsigned long long *status;  // [passes][ntiles][256]
};

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const K *__restrict__ q, uint64_t nq,
                                                            SortNorm sn, uint32_t *__restrict__ ghist)
{
    __shared__ uint32_t h[kMaxPasses][256];
    for (int i = threadIdx.x; i < kMaxPasses * 256; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    constexpr int R = kSortTile / kSortThreads;
    const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kSortTile;
    K key[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {  // all loads in flight before any use
        const uint64_t pos = base + r * kSortThreads + threadIdx.x;
        if (pos < nq) key[r] = q[pos];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t pos = base + r * kSortThreads + threadIdx.x;
        const bool valid = pos < nq;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        for (int p = 0; p < sn.passes; ++p) {
            const uint32_t d = valid ? sort_digit(key[r], sn, p) : 0u;
            const unsigned same = warp_match8(d, vm);
            if (valid && (same & sort_lanemask_lt()) == 0) atomicAdd(&h[p][d], __popc(same));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < sn.passes * 256; i += blockDim.x) {
        const uint32_t v = (&h[0][0])[i];
        if (v) atomicAdd(ghist + i, v);
    }
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Exclusive scan of 256 values held one per thread by threads 0..255;
// all threads of the block must call it.  `tmp` holds 8 words.
__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t v, uint32_t *tmp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (warp < 8 && lane == 31) tmp[warp] = x;
    __syncthreads();
    uint32_t before = 0;
    if (warp < 8)
        for (int w = 0; w < warp; ++w) before += tmp[w];
    __syncthreads();
    return before + x - v;
}

template <typename K>
struct SortPassSmem {
    uint32_t wh[kSortWarps][256];
    uint32_t tstart[256];
    uint32_t gbase[256];
    uint32_t tpref[256];
    uint32_t scan_tmp[8];
    uint32_t tile;
    K sk[kSortTile];
    uint32_t si[kSortTile];
};

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_pass(
    const K *__restrict__ qin, const uint32_t *__restrict__ iin, K *__restrict__ qout,
    uint32_t *__restrict__ iout, uint64_t nq, SortNorm sn, int pass, SortMeta meta, uint32_t ntiles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortPassSmem<K> &S = *reinterpret_cast<SortPassSmem<K> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int i = tid; i < kSortWarps * 256; i += blockDim.x) (&S.wh[0][0])[i] = 0;
    if (tid == 0) S.tile = atomicAdd(meta.tile_ctr + pass, 1u);
    __syncthreads();
    const uint32_t tile = S.tile;
    const uint64_t tile_base = static_cast<uint64_t>(tile) * kSortTile;
    const uint32_t tile_n = static_cast<uint32_t>(nq - tile_base < kSortTile ? nq - tile_base : kSortTile);

    // 1. load this warp's 256 elements and rank them stably within the warp
    constexpr int R = kSortPerWarp / 32;
    K key[R];
    uint32_t idx[R], dig[R], rank[R];
    const uint64_t wbase = tile_base + warp * kSortPerWarp;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t pos = wbase + r * 32 + lane;
        if (pos < nq) {
            key[r] = qin[pos];
            idx[r] = iin ? iin[pos] : static_cast<uint32_t>(pos);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t pos = wbase + r * 32 + lane;
        const bool valid = pos < nq;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        dig[r] = valid ? sort_digit(key[r], sn, pass) : 0u;
        const unsigned same = warp_match8(dig[r], vm);
        if (valid) rank[r] = S.wh[warp][dig[r]] + __popc(same & sort_lanemask_lt());
        __syncwarp();
        if (valid && (same & sort_lanemask_lt()) == 0) S.wh[warp][dig[r]] += __popc(same);
        __syncwarp();
    }
    __syncthreads();

    // 2. per digit: prefix over warps, tile count, publication, offsets
    uint32_t tcnt = 0;
    if (tid < 256) {
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t v = S.wh[w][tid];
            S.wh[w][tid] = tcnt;
            tcnt += v;
        }
        unsigned long long *st = meta.status + (static_cast<uint64_t>(pass) * ntiles + tile) * 256u + tid;
        st_relaxed_u64(st, (tile == 0 ? kFlagIncl : kFlagAgg) | tcnt);
    }
    const uint32_t gh = (tid < 256) ? meta.ghist[pass * 256 + tid] : 0u;
    const uint32_t gb = block_excl_scan256(gh, S.scan_tmp);
    const uint32_t ts = block_excl_scan256(tcnt, S.scan_tmp);
    if (tid < 256) {
        S.gbase[tid] = gb;
        S.tstart[tid] = ts;
    }
    __syncthreads();

    // 3. reorder the tile by digit in shared memory (before the look-back,
    //    so the elements' registers are free while it runs)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint64_t pos = wbase + r * 32 + lane;
        if (pos < nq) {
            const uint32_t lp = S.tstart[dig[r]] + S.wh[warp][dig[r]] + rank[r];
            S.sk[lp] = key[r];
            S.si[lp] = idx[r];
        }
    }

    if (tid < 256) {
        // Decoupled look-back over the preceding tiles for this digit, a
        // window of kLookbackWindow tiles per round trip: walking down from
        // the nearest tile, add counts until a tile that already published
        // its inclusive prefix; a tile that has published nothing yet makes
        // the window be read again (bounded).
        uint32_t excl = 0;
        if (tile > 0) {
            const unsigned long long *col = meta.status + static_cast<uint64_t>(pass) * ntiles * 256u + tid;
            int64_t end = tile;
            uint32_t spins = 0;
            while (end > 0) {
                const int64_t lo = end > kLookbackWindow ? end - kLookbackWindow : 0;
                const int n = static_cast<int>(end - lo);
                unsigned long long v[kLookbackWindow];
#pragma unroll
                for (int k = 0; k < kLookbackWindow; ++k)
                    v[k] = (k < n) ? ld_relaxed_u64(col + static_cast<uint64_t>(lo + k) * 256u) : 0ull;
                uint32_t acc = 0;
                bool done = false, retry = false;
#pragma unroll
                for (int k = kLookbackWindow - 1; k >= 0; --k) {
                    if (k < n && !done && !retry) {
                        const unsigned long long flag = v[k] & (3ull << 62);
                        if (flag == 0) {
                            retry = true;
                        } else {
                            acc += static_cast<uint32_t>(v[k]);
                            done = (flag == kFlagIncl);
                        }
                    }
                }
                if (retry) {
                    if (++spins > kLookbackSpinLimit) {
                        atomicOr(meta.err, 1u);
                        break;
                    }
                    __nanosleep(64);
                    continue;
                }
                excl += acc;
                if (done) break;
                end = lo;
            }
            unsigned long long *st = meta.status + (static_cast<uint64_t>(pass) * ntiles + tile) * 256u + tid;
            st_relaxed_u64(st, kFlagIncl | (excl + tcnt));
        }
        S.tpref[tid] = excl;
    }
    __syncthreads();

    // 4. write runs of equal digits to consecutive output positions
    for (uint32_t i = tid; i < tile_n; i += blockDim.x) {
        const K k = S.sk[i];
        const uint32_t d = sort_digit(k, sn, pass);
        const uint32_t g = S.gbase[d] + S.tpref[d] + (i - S.tstart[d]);
        qout[g] = k;
        iout[g] = S.si[i];
    }
}

template <typename K>
constexpr int sort_pass_smem_bytes()
{
    return static_cast<int>(sizeof(SortPassSmem<K>));
}

}  // namespace btgb
