// Key types of the search kernels.
//
// Integer keys (uint32_t, uint64_t) are compared as unsigned integers and
// are stored in the tree and passed in queries as they are.
//
// 32-byte keys are the paper's key format: two keys compare byte by byte
// from the first byte, the first unequal byte deciding (Sec. IV-E: one
// comparator per byte, reduced by a priority cascade) -- lexicographic
// order.  Queries arrive as the raw 32 bytes (Raw32).  The tree stores each
// key as Key32: four 64-bit words, most significant first, word j being the
// big-endian value of key bytes 8j..8j+7, so that comparing the words in
// order, as unsigned integers, is comparing the bytes lexicographically.
// A query is converted to Key32 once, when it is loaded.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace btgb {

struct alignas(16) Raw32 {
    uint64_t b[4];  // the key's 32 bytes in memory order
};

struct alignas(16) Key32 {
    uint64_t w[4];  // w[0] = big-endian value of bytes 0..7, and so on
};

__host__ __device__ __forceinline__ bool operator<(const Key32 &a, const Key32 &b)
{
    // the first unequal word decides, as the first unequal byte does (distinct
    // keys nearly always differ in the first word: one compare, no divergence)
    if (a.w[0] != b.w[0]) return a.w[0] < b.w[0];
    if (a.w[1] != b.w[1]) return a.w[1] < b.w[1];
    if (a.w[2] != b.w[2]) return a.w[2] < b.w[2];
    return a.w[3] < b.w[3];
}

__host__ __device__ __forceinline__ bool operator==(const Key32 &a, const Key32 &b)
{
    return ((a.w[0] ^ b.w[0]) | (a.w[1] ^ b.w[1]) | (a.w[2] ^ b.w[2]) | (a.w[3] ^ b.w[3])) == 0;
}

__host__ __device__ __forceinline__ bool operator>(const Key32 &a, const Key32 &b) { return b < a; }

// Big-endian value of 8 bytes held in a little-endian 64-bit load.
__device__ __forceinline__ uint64_t bytes_be64(uint64_t x)
{
    const uint32_t lo = static_cast<uint32_t>(x), hi = static_cast<uint32_t>(x >> 32);
    return (static_cast<uint64_t>(__byte_perm(lo, 0, 0x0123)) << 32) | __byte_perm(hi, 0, 0x0123);
}

// How each key type is read from a query array, and its all-ones value.
template <typename K>
struct KeyOps {
    using Raw = K;
    __device__ static __forceinline__ K from_raw(const Raw &r) { return r; }
    __device__ static __forceinline__ K load(const Raw *q, uint64_t i) { return q[i]; }
    __host__ __device__ static constexpr K ones() { return static_cast<K>(~static_cast<K>(0)); }
};

template <>
struct KeyOps<Key32> {
    using Raw = Raw32;
    __device__ static __forceinline__ Key32 from_raw(const Raw32 &r)
    {
        Key32 k;
#pragma unroll
        for (int j = 0; j < 4; ++j) k.w[j] = bytes_be64(r.b[j]);
        return k;
    }
    __device__ static __forceinline__ Key32 load(const Raw32 *q, uint64_t i) { return from_raw(q[i]); }
    __host__ __device__ static Key32 ones() { return Key32{{~0ull, ~0ull, ~0ull, ~0ull}}; }
};

template <typename K>
using RawOf = typename KeyOps<K>::Raw;

// *p < key for a key in shared or global memory.  A 32-byte key's first word
// is read alone, and the other three only when it ties.
template <typename K>
__device__ __forceinline__ bool mem_lt(const K *p, const K &key)
{
    return *p < key;
}

template <>
__device__ __forceinline__ bool mem_lt<Key32>(const Key32 *p, const Key32 &key)
{
    const uint64_t w0 = p->w[0];
    if (w0 != key.w[0]) return w0 < key.w[0];
    return *p < key;
}

// One query of a partitioned batch of integer keys: the key as the caller
// gave it, its input position, and its local-sort digit, 16 bytes, so that
// each query moves with one vector store.  (32-byte keys are partitioned
// into separate key and position arrays.)
template <typename K>
struct alignas(16) PartRec {
    RawOf<K> key;
    uint32_t idx;
    uint32_t digit;
};

// Load query `pos` of a batch: from the partition's records when given,
// else from the key array and the optional position array (identity when
// absent).
template <typename K>
__device__ __forceinline__ void load_query(const RawOf<K> *q, const uint32_t *qidx, const PartRec<K> *recs,
                                           uint64_t pos, K &key, uint32_t &dst)
{
    if (recs) {
        const PartRec<K> r = recs[pos];
        key = KeyOps<K>::from_raw(r.key);
        dst = r.idx;
    } else {
        key = KeyOps<K>::load(q, pos);
        dst = qidx ? qidx[pos] : static_cast<uint32_t>(pos);
    }
}

}  // namespace btgb
