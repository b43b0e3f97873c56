// Many batches over several resident trees in one persistent launch.
//
// A "forest" is a device table of built trees sharing key and value widths
// (fanouts may differ).  A search takes a device work list of batches, each
// naming a tree, a count and an offset into flat query/result arrays, and
// runs all of them in one launch: a plan kernel turns the batch counts into
// 32-query chunk offsets, then persistent warps take chunks in turn and walk
// each chunk's queries down that chunk's tree level by level exactly as the
// single-tree descent does (distinct nodes per warp staged once, binary
// search per lane, leaf probe, result written at the query's position).
// Nothing is allocated and nothing is synchronised, so the whole call can be
// captured in a CUDA graph and replayed for every new work list.
#include <cuda_runtime.h>

#include <cstring>
#include <new>

#include "bt_internal.h"

struct bt_forest {
    btgb::DevTree *d_trees;
    uint32_t count;
    int key_bytes, val_bytes;
    int max_m;
};

namespace btgb {

// Work-list entries rejected by k_forest (tree out of range, or queries
// beyond the arrays); read and cleared by bt_forest_bad_batches.
__device__ unsigned long long g_bt_bad_batches;

__device__ __forceinline__ void fcp_async16(void *smem_dst, const void *gsrc)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void fcp_wait()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Slots below m (a power of two) holding a key smaller than `key`; slot m-1
// is always padding.
template <typename K>
__device__ __forceinline__ int rank_rt(const K *blk, int m, K key)
{
    int r = 0;
    for (int h = m >> 1; h >= 1; h >>= 1)
        if (blk[r + h - 1] < key) r += h;
    return r;
}

__device__ __forceinline__ void fwarp_distinct(uint32_t node, int lane, uint32_t *list, int &U, int &slot)
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

// chunk_start[b] = number of 32-query chunks in batches before b (one block).
__global__ void __launch_bounds__(1024) k_forest_plan(const bt_batch_desc *__restrict__ batches, uint32_t nb,
                                                      uint32_t *__restrict__ chunk_start)
{
    __shared__ uint32_t tmp[32];
    uint32_t run = 0;
    for (uint32_t base = 0; base < nb; base += blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t c = i < nb ? (batches[i].count + 31u) / 32u : 0u;
        // block exclusive scan of c
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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

constexpr int kForestSlots = 8;
constexpr int kForestMaxBlock = 512;  // bytes of the largest node block (m = 64, 8-byte keys)

template <typename K, typename V>
__global__ void __launch_bounds__(512) k_forest(const DevTree *__restrict__ trees, uint32_t ntrees,
                                                const bt_batch_desc *__restrict__ batches, uint32_t nb,
                                                const uint32_t *__restrict__ chunk_start, const K *__restrict__ q,
                                                uint64_t nq, V *__restrict__ out_v, uint8_t *__restrict__ out_f)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned char *stage = smem + warp * (kForestSlots * kForestMaxBlock + 32 * 4);
    uint32_t *list = reinterpret_cast<uint32_t *>(stage + kForestSlots * kForestMaxBlock);
    const uint32_t nchunks = chunk_start[nb];
    for (uint32_t c = blockIdx.x * nw + warp; c < nchunks; c += gridDim.x * nw) {
        // the batch holding chunk c: last b with chunk_start[b] <= c
        uint32_t lo = 0, hi = nb - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (chunk_start[mid] <= c)
                lo = mid;
            else
                hi = mid - 1;
        }
        const bt_batch_desc bd = batches[lo];
        // a descriptor naming a tree outside the forest, or queries beyond
        // the arrays, is skipped (nothing written) and counted
        if (bd.tree >= ntrees || bd.offset > nq || bd.count > nq - bd.offset) {
            if (lane == 0 && c == chunk_start[lo]) atomicAdd(&g_bt_bad_batches, 1ull);
            continue;
        }
        const uint32_t j = (c - chunk_start[lo]) * 32u + lane;
        const bool valid = j < bd.count;
        const DevTree &t = trees[bd.tree];
        const int H = t.height, m = t.m;
        const uint64_t pos = bd.offset + (valid ? j : (c - chunk_start[lo]) * 32u);
        const K key = q[pos];
        if (H == 0) {
            if (valid) {
                out_v[pos] = static_cast<V>(~static_cast<V>(0));
                out_f[pos] = 0;
            }
            continue;
        }
        const int CH = m * static_cast<int>(sizeof(K)) / 16;
        uint32_t node = 0;
        for (int l = 0; l < H; ++l) {
            const K *lk = static_cast<const K *>(t.keys[l]);
            int U, slot;
            fwarp_distinct(node, lane, list, U, slot);
            __syncwarp();
            int r = 0;
            bool eq = false;
            for (int rb = 0; rb < U; rb += kForestSlots) {
                const int nu = (U - rb < kForestSlots) ? U - rb : kForestSlots;
                for (int i = lane; i < nu * CH; i += 32) {
                    const int u = i / CH, part = i - u * CH;
                    fcp_async16(stage + u * kForestMaxBlock + part * 16,
                                reinterpret_cast<const unsigned char *>(lk + static_cast<uint64_t>(list[rb + u]) * m) +
                                    part * 16);
                }
                fcp_wait();
                __syncwarp();
                if (slot >= rb && slot < rb + nu) {
                    const K *blk = reinterpret_cast<const K *>(stage + (slot - rb) * kForestMaxBlock);
                    r = rank_rt<K>(blk, m, key);
                    eq = (blk[r] == key);
                }
                __syncwarp();
            }
            if (l + 1 < H) {
                const uint64_t base = t.cbase[l], rem = t.crem[l];
                node = static_cast<uint32_t>(node * base + (node < rem ? node : rem) + r);
            } else {
                const uint64_t cnt = t.cbase[l] + (node < t.crem[l] ? 1u : 0u);
                const bool hit = (static_cast<uint64_t>(r) < cnt) && eq;
                V val = static_cast<V>(~static_cast<V>(0));
                if (hit) val = static_cast<const V *>(t.vals)[static_cast<uint64_t>(node) * m + r];
                if (valid) {
                    out_v[pos] = val;
                    out_f[pos] = hit ? 1 : 0;
                }
            }
        }
    }
}

template <typename K, typename V>
static cudaError_t forest_launch(const bt_forest *f, const bt_batch_desc *d_b, uint32_t nb, uint32_t *chunk_start,
                                 const void *q, uint64_t nq, void *ov, uint8_t *of, uint32_t warps, cudaStream_t s)
{
    const int threads = static_cast<int>(warps) * 32;
    const int smem = static_cast<int>(warps) * (kForestSlots * kForestMaxBlock + 32 * 4);
    auto kern = k_forest<K, V>;
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(kern), 16 * (kForestSlots * kForestMaxBlock + 32 * 4));
    int per_sm = 0, sms = 0;
    if (e == cudaSuccess) e = blocks_per_sm(reinterpret_cast<const void *>(kern), threads, smem, &per_sm);
    if (e == cudaSuccess) e = dev_sm_count(&sms);
    if (e != cudaSuccess) return e;
    k_forest_plan<<<1, 1024, 0, s>>>(d_b, nb, chunk_start);
    const unsigned grid = static_cast<unsigned>(sms * (per_sm > 0 ? per_sm : 1));
    kern<<<grid, threads, smem, s>>>(f->d_trees, f->count, d_b, nb, chunk_start, static_cast<const K *>(q), nq,
                                     static_cast<V *>(ov), of);
    return cudaGetLastError();
}

}  // namespace btgb

using namespace btgb;

extern "C" bt_status bt_forest_create(const bt_tree *const *trees, uint32_t count, bt_forest **out)
{
    if (!trees || !out || count == 0) return BT_ERR_ARG;
    for (uint32_t i = 0; i < count; ++i)
        if (!trees[i] || trees[i]->dev.key_bytes == 32 || trees[i]->dev.key_bytes != trees[0]->dev.key_bytes ||
            trees[i]->dev.val_bytes != trees[0]->dev.val_bytes)
            return BT_ERR_ARG;
    bt_forest *f = new (std::nothrow) bt_forest;
    if (!f) return BT_ERR_NOMEM;
    f->count = count;
    f->key_bytes = trees[0]->dev.key_bytes;
    f->val_bytes = trees[0]->dev.val_bytes;
    DevTree *h = new (std::nothrow) DevTree[count];
    if (!h) {
        delete f;
        return BT_ERR_NOMEM;
    }
    for (uint32_t i = 0; i < count; ++i) h[i] = trees[i]->dev;
    cudaError_t e = cudaMalloc(&f->d_trees, sizeof(DevTree) * count);
    if (e == cudaSuccess) e = cudaMemcpy(f->d_trees, h, sizeof(DevTree) * count, cudaMemcpyHostToDevice);
    delete[] h;
    if (e != cudaSuccess) {
        set_error_detail("forest table", e);
        if (f->d_trees) cudaFree(f->d_trees);
        delete f;
        return e == cudaErrorMemoryAllocation ? BT_ERR_NOMEM : BT_ERR_CUDA;
    }
    *out = f;
    return BT_OK;
}

extern "C" void bt_forest_free(bt_forest *f)
{
    if (!f) return;
    cudaFree(f->d_trees);
    delete f;
}

extern "C" uint64_t bt_forest_workspace_bytes(uint32_t nbatches) { return (static_cast<uint64_t>(nbatches) + 1) * 4; }

extern "C" bt_status bt_forest_search(const bt_forest *f, const bt_batch_desc *d_batches, uint32_t nbatches,
                                      const void *d_queries, uint64_t nq, void *d_out_vals, uint8_t *d_out_found,
                                      void *d_workspace, uint64_t ws_bytes, uint32_t warps_per_block,
                                      bt_stream stream)
{
    if (!f) return BT_ERR_ARG;
    if (nbatches == 0) return BT_OK;
    if (!d_batches || !d_queries || !d_out_vals || !d_out_found) return BT_ERR_ARG;
    if (warps_per_block == 0) warps_per_block = 8;
    if (warps_per_block > 16) return BT_ERR_ARG;
    if (!d_workspace || ws_bytes < bt_forest_workspace_bytes(nbatches)) return BT_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t *cs = static_cast<uint32_t *>(d_workspace);
    cudaError_t e;
    if (f->key_bytes == 8) {
        if (f->val_bytes == 8)
            e = forest_launch<uint64_t, uint64_t>(f, d_batches, nbatches, cs, d_queries, nq, d_out_vals,
                                                  d_out_found, warps_per_block, s);
        else
            e = forest_launch<uint64_t, uint32_t>(f, d_batches, nbatches, cs, d_queries, nq, d_out_vals,
                                                  d_out_found, warps_per_block, s);
    } else {
        if (f->val_bytes == 8)
            e = forest_launch<uint32_t, uint64_t>(f, d_batches, nbatches, cs, d_queries, nq, d_out_vals,
                                                  d_out_found, warps_per_block, s);
        else
            e = forest_launch<uint32_t, uint32_t>(f, d_batches, nbatches, cs, d_queries, nq, d_out_vals,
                                                  d_out_found, warps_per_block, s);
    }
    if (e != cudaSuccess) {
        set_error_detail("forest search launch", e);
        return BT_ERR_CUDA;
    }
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
