// The level-wise descent over the paper's node layout (Eq. 1, Fig. 3), for
// comparison with the structure-of-arrays layout.  Same walk as the
// synchronous descent: per level the warp's distinct nodes are staged whole
// (16-byte cp.async) and each lane follows the child address of its rank,
// or at a leaf reads the data slot of its rank from the staged node.
#include <cuda_runtime.h>

#include <cstdint>

#include "descent.cuh"

namespace btgb {

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
    const PaperTree p, const RawOf<K> *__restrict__ q, const uint32_t *__restrict__ qidx,
    const PartRec<K> *__restrict__ recs, uint64_t nq, V *__restrict__ out_v, uint8_t *__restrict__ out_f)
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
        K key;
        uint32_t dst;
        load_query<K>(q, qidx, recs, valid ? pos : c * 32, key, dst);
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
            } else if (valid && dst < nq) {
                out_v[dst] = val;
                out_f[dst] = hit ? 1 : 0;
            }
        }
    }
}

template <typename K, typename V, int M>
static cudaError_t launch_paper(const PaperTree &p, const void *q, const uint32_t *qidx, const void *recs, uint64_t nq,
                                void *out_v, uint8_t *out_f, int nw, cudaStream_t s)
{
    auto kern = k_descend_paper<K, V, M>;
    const int smem = static_cast<int>(p.pin_bytes) + nw * paper_smem_per_warp<K, M>();
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(kern),
                                    16384 + kDescWarpsMax * paper_smem_per_warp<K, M>());
    if (e != cudaSuccess) return e;
    unsigned grid = 0;
    e = persistent_grid(reinterpret_cast<const void *>(kern), nw * 32, smem, static_cast<uint64_t>(nw) * 32, nq, &grid);
    if (e != cudaSuccess) return e;
    kern<<<grid, nw * 32, smem, s>>>(p, static_cast<const RawOf<K> *>(q), qidx, static_cast<const PartRec<K> *>(recs),
                                     nq, static_cast<V *>(out_v), out_f);
    return cudaGetLastError();
}

template <typename K, typename V>
static cudaError_t paper_m(const DevTree &t, const PaperTree &p, const void *q, const uint32_t *qidx, const void *recs,
                           uint64_t nq, void *out_v, uint8_t *out_f, cudaStream_t s)
{
    const int nw = t.warps > 0 ? t.warps : kDescWarpsDefault;
    switch (t.m) {
    case 8: return launch_paper<K, V, 8>(p, q, qidx, recs, nq, out_v, out_f, nw, s);
    case 16: return launch_paper<K, V, 16>(p, q, qidx, recs, nq, out_v, out_f, nw, s);
    case 32: return launch_paper<K, V, 32>(p, q, qidx, recs, nq, out_v, out_f, nw, s);
    default: return launch_paper<K, V, 64>(p, q, qidx, recs, nq, out_v, out_f, nw, s);
    }
}

cudaError_t descend_paper_layout(const DevTree &t, const PaperTree &p, const void *q, const uint32_t *qidx,
                                 const void *recs, uint64_t nq, void *out_v, uint8_t *out_f, cudaStream_t s)
{
    if (t.key_bytes == 32)
        return t.val_bytes == 8 ? paper_m<Key32, uint64_t>(t, p, q, qidx, recs, nq, out_v, out_f, s)
                                : paper_m<Key32, uint32_t>(t, p, q, qidx, recs, nq, out_v, out_f, s);
    if (t.key_bytes == 8)
        return t.val_bytes == 8 ? paper_m<uint64_t, uint64_t>(t, p, q, qidx, recs, nq, out_v, out_f, s)
                                : paper_m<uint64_t, uint32_t>(t, p, q, qidx, recs, nq, out_v, out_f, s);
    return t.val_bytes == 8 ? paper_m<uint32_t, uint64_t>(t, p, q, qidx, recs, nq, out_v, out_f, s)
                            : paper_m<uint32_t, uint32_t>(t, p, q, qidx, recs, nq, out_v, out_f, s);
}

}  // namespace btgb
