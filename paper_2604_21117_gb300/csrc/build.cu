// Host-side tree construction and bookkeeping (bt_build, bt_free, bt_tree_info).
//
// The tree is built once on the host and copied to device memory once
// (Sec. IV-B's BFS "mapper" flattens a pointer tree into a uniform node
// array; Sec. V-B treats that as one-time initialisation).  Here the levels
// are written directly in structure-of-arrays form from the sorted keys.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "bt_internal.h"

namespace btgb {

static thread_local char g_detail[256] = "";

void set_error_detail(const char *what, cudaError_t err)
{
    snprintf(g_detail, sizeof(g_detail), "%s: %s", what, cudaGetErrorString(err));
}

static inline uint64_t load_uint(const void *p, uint64_t i, int bytes)
{
    return bytes == 8 ? static_cast<const uint64_t *>(p)[i] : static_cast<const uint32_t *>(p)[i];
}

static inline void store_uint(void *p, uint64_t i, int bytes, uint64_t v)
{
    if (bytes == 8)
        static_cast<uint64_t *>(p)[i] = v;
    else
        static_cast<uint32_t *>(p)[i] = static_cast<uint32_t>(v);
}

static inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Big-endian value of 8 bytes.
static inline uint64_t be64(const unsigned char *b)
{
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i) v = (v << 8) | b[i];
    return v;
}

static inline const unsigned char *key_ptr(const void *h_keys, uint64_t i, int kb)
{
    return static_cast<const unsigned char *>(h_keys) + i * static_cast<uint64_t>(kb);
}

// Key i of the caller's array into device slot `slot` of a key array:
// integers as they are, 32-byte keys as four big-endian 64-bit words.
static inline void store_key(void *dst, uint64_t slot, int kb, const void *h_keys, uint64_t i)
{
    if (kb == 32) {
        uint64_t *w = static_cast<uint64_t *>(dst) + slot * 4;
        const unsigned char *b = key_ptr(h_keys, i, kb);
        for (int j = 0; j < 4; ++j) w[j] = be64(b + 8 * j);
    } else {
        store_uint(dst, slot, kb, load_uint(h_keys, i, kb));
    }
}

// All-ones padding slot (all-ones words for 32-byte keys).
static inline void store_pad(void *dst, uint64_t slot, int kb)
{
    memset(static_cast<unsigned char *>(dst) + slot * static_cast<uint64_t>(kb), 0xFF, static_cast<size_t>(kb));
}

// <0, 0, >0 as key a is below, equal to or above key b.
static inline int key_cmp(const void *h_keys, uint64_t a, uint64_t b, int kb)
{
    if (kb == 32) return memcmp(key_ptr(h_keys, a, kb), key_ptr(h_keys, b, kb), 32);
    const uint64_t x = load_uint(h_keys, a, kb), y = load_uint(h_keys, b, kb);
    return (x > y) - (x < y);
}

namespace {
std::mutex g_launch_mu;
std::map<int, int> g_sms;                                           // device -> SMs
// The same counts for the first devices, read without the lock on every
// launch (0 until known).
constexpr int kSmsFast = 64;
std::atomic<int> g_sms_fast[kSmsFast];
std::map<std::tuple<int, const void *, int, int>, int> g_occ;       // (device, kernel, threads, smem)
std::map<std::pair<int, const void *>, int> g_dyn;                  // (device, kernel) -> limit set
std::atomic<uint32_t> g_first_wait_polls{BT_DEFAULT_WAIT_POLLS};
}  // namespace

uint32_t first_wait_polls() { return g_first_wait_polls.load(std::memory_order_relaxed); }

cudaError_t dev_sm_count(int *sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kSmsFast) {
        const int v = g_sms_fast[dev].load(std::memory_order_relaxed);
        if (v > 0) {
            *sms = v;
            return cudaSuccess;
        }
    }
    std::lock_guard<std::mutex> lk(g_launch_mu);
    auto it = g_sms.find(dev);
    if (it == g_sms.end()) {
        int v = 0;
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        it = g_sms.emplace(dev, v).first;
    }
    *sms = it->second;
    if (dev >= 0 && dev < kSmsFast) g_sms_fast[dev].store(it->second, std::memory_order_relaxed);
    return cudaSuccess;
}

cudaError_t blocks_per_sm(const void *kern, int threads, int dyn_smem, int *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_launch_mu);
    const auto key = std::make_tuple(dev, kern, threads, dyn_smem);
    auto it = g_occ.find(key);
    if (it == g_occ.end()) {
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, static_cast<size_t>(dyn_smem));
        if (e != cudaSuccess) return e;
        it = g_occ.emplace(key, b > 0 ? b : 1).first;
    }
    *out = it->second;
    return cudaSuccess;
}

cudaError_t ensure_dyn_smem(const void *kern, int bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_launch_mu);
    const auto key = std::make_pair(dev, kern);
    auto it = g_dyn.find(key);
    if (it != g_dyn.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    g_dyn[key] = bytes;
    return cudaSuccess;
}

void set_pin_levels(DevTree &d, const bt_info &info, uint32_t budget)
{
    d.pin_levels = 0;
    d.pin_bytes = 0;
    for (int l = 0; l + 1 < d.height; ++l) {
        const uint64_t end = info.level_key_offset[l] + d.nodes[l] * static_cast<uint64_t>(d.m) * d.key_bytes;
        if (end > budget) break;
        d.pin_levels = l + 1;
        d.pin_bytes = static_cast<uint32_t>((end + 15) / 16 * 16);
    }
}

}  // namespace btgb

using namespace btgb;

extern "C" bt_status bt_tree_set_launch(bt_tree *t, uint32_t warps_per_block, uint32_t pin_bytes)
{
    if (!t || warps_per_block < 1 || warps_per_block > 16 || pin_bytes > 49152) return BT_ERR_ARG;
    t->dev.warps = static_cast<int>(warps_per_block);
    set_pin_levels(t->dev, t->info, pin_bytes);
    return BT_OK;
}

extern "C" bt_status bt_tree_set_lane_queries(bt_tree *t, uint32_t per_lane)
{
    if (!t || per_lane < 1 || per_lane > 2) return BT_ERR_ARG;
    t->dev.lane_queries = static_cast<int>(per_lane);
    return BT_OK;
}

extern "C" bt_status bt_tree_set_staging(bt_tree *t, uint32_t mode)
{
    if (!t || mode > BT_STAGE_PIPELINED) return BT_ERR_ARG;
    t->dev.staging = static_cast<int>(mode);
    return BT_OK;
}

extern "C" bt_status bt_tree_set_descent(bt_tree *t, uint32_t inner_staged, uint32_t rank_ballot)
{
    if (!t || inner_staged > 2 || rank_ballot > 1) return BT_ERR_ARG;
    t->dev.inner_stage = static_cast<int>(inner_staged);
    t->dev.rank_ballot = static_cast<int>(rank_ballot);
    return BT_OK;
}

extern "C" bt_status bt_tree_set_corun(bt_tree *t, uint32_t descent_blocks_per_sm, uint32_t partition_blocks_per_sm)
{
    if (!t || descent_blocks_per_sm > 32 || partition_blocks_per_sm > 32) return BT_ERR_ARG;
    t->dev.corun_descent_bps = static_cast<int>(descent_blocks_per_sm);
    t->dev.corun_partition_bps = static_cast<int>(partition_blocks_per_sm);
    return BT_OK;
}

extern "C" bt_status bt_tree_set_l2_window(bt_tree *t, uint64_t max_bytes)
{
    if (!t) return BT_ERR_ARG;
    t->l2_base = nullptr;
    t->l2_bytes = 0;
    t->l2_hit_ratio = 0.0f;
    const DevTree &d = t->dev;
    if (max_bytes == 0 || d.height < 2 || d.pin_levels >= d.height - 1) return BT_OK;
    // the inner levels below the pinned ones: contiguous from level pin_levels
    // to the start of the leaf level
    const uint64_t lo = t->info.level_key_offset[d.pin_levels];
    const uint64_t hi = t->info.level_key_offset[d.height - 1];
    int dev = 0, max_win = 0, max_persist = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev);
    if (e != cudaSuccess) {
        set_error_detail("L2 window attributes", e);
        return BT_ERR_CUDA;
    }
    uint64_t bytes = hi - lo;
    if (bytes > max_bytes) bytes = max_bytes;
    if (bytes > static_cast<uint64_t>(max_win)) bytes = static_cast<uint64_t>(max_win);
    if (bytes == 0 || max_persist <= 0) return BT_OK;
    // the context's persisting set-aside (this process only; it ends with it)
    size_t cur = 0;
    e = cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    const size_t want = bytes < static_cast<uint64_t>(max_persist) ? bytes : static_cast<size_t>(max_persist);
    if (e == cudaSuccess && cur < want) e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want);
    if (e == cudaSuccess) e = cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    if (e != cudaSuccess) {
        set_error_detail("persisting L2 limit", e);
        return BT_ERR_CUDA;
    }
    t->l2_base = static_cast<const unsigned char *>(t->d_image) + lo;
    t->l2_bytes = bytes;
    t->l2_hit_ratio = cur >= bytes ? 1.0f : static_cast<float>(cur) / static_cast<float>(bytes);
    return BT_OK;
}

extern "C" void bt_debug_set_wait_polls(uint32_t polls) { g_first_wait_polls.store(polls); }

extern "C" const char *bt_last_error_detail(void) { return g_detail; }

extern "C" const char *bt_status_str(bt_status s)
{
    switch (s) {
    case BT_OK: return "ok";
    case BT_ERR_ARG: return "invalid argument";
    case BT_ERR_UNSORTED: return "build keys are not in ascending order";
    case BT_ERR_DUPLICATE: return "build keys contain a duplicate";
    case BT_ERR_FANOUT: return "fanout must be 8, 16, 32 or 64";
    case BT_ERR_NOMEM: return "out of memory";
    case BT_ERR_CUDA: return "CUDA runtime error";
    case BT_ERR_TIMEOUT: return "bounded device wait timed out";
    case BT_ERR_WORKSPACE: return "workspace missing or too small";
    }
    return "unknown status";
}

extern "C" bt_status bt_build(const void *h_keys, const void *h_vals, uint64_t n, bt_width key_w,
                              bt_width val_w, uint32_t fanout, bt_stream stream, bt_tree **out)
{
    if (!out) return BT_ERR_ARG;
    if ((key_w != BT_U32 && key_w != BT_U64 && key_w != BT_B32) || (val_w != BT_U32 && val_w != BT_U64))
        return BT_ERR_ARG;
    if (fanout != 8 && fanout != 16 && fanout != 32 && fanout != 64) return BT_ERR_FANOUT;
    if (n > 0 && (!h_keys || !h_vals)) return BT_ERR_ARG;
    const int kb = static_cast<int>(key_w), vb = static_cast<int>(val_w);
    const uint64_t m = fanout, kmax_per_node = m - 1;

    for (uint64_t i = 1; i < n; ++i) {
        const int c = key_cmp(h_keys, i - 1, i, kb);
        if (c > 0) return BT_ERR_UNSORTED;
        if (c == 0) return BT_ERR_DUPLICATE;
    }

    // Level sizes, leaves first.
    std::vector<uint64_t> up;  // up[0] = leaves, up[k] = k levels above
    if (n > 0) {
        uint64_t c = (n + kmax_per_node - 1) / kmax_per_node;
        up.push_back(c);
        while (c > 1) {
            c = (c + m - 1) / m;
            up.push_back(c);
        }
    }
    const int h = static_cast<int>(up.size());
    if (h > BT_MAX_LEVELS) return BT_ERR_ARG;
    for (uint64_t c : up)
        if (c >= (1ull << 32)) return BT_ERR_ARG;

    bt_tree *t = new (std::nothrow) bt_tree;
    if (!t) return BT_ERR_NOMEM;
    memset(t, 0, sizeof(*t));
    DevTree &d = t->dev;
    d.height = h;
    d.m = static_cast<int>(m);
    d.key_bytes = kb;
    d.val_bytes = vb;
    t->info.height = static_cast<uint32_t>(h);
    t->info.fanout = fanout;
    t->info.key_bytes = static_cast<uint32_t>(kb);
    t->info.val_bytes = static_cast<uint32_t>(vb);
    t->info.n = n;
    if (n > 0 && kb == 32) {
        for (int j = 0; j < 4; ++j) {
            d.kmin32[j] = be64(key_ptr(h_keys, 0, kb) + 8 * j);
            d.kmax32[j] = be64(key_ptr(h_keys, n - 1, kb) + 8 * j);
        }
    } else if (n > 0) {
        d.kmin = load_uint(h_keys, 0, kb);
        d.kmax = load_uint(h_keys, n - 1, kb);
    }

    // Byte layout: level key arrays root first, then leaf values.
    uint64_t off = 0;
    for (int l = 0; l < h; ++l) {
        const uint64_t N = up[h - 1 - l];
        d.nodes[l] = N;
        t->info.level_nodes[l] = N;
        t->info.level_key_offset[l] = off;
        off = align_up(off + N * m * kb, 256);
    }
    t->info.leaf_val_offset = off;
    uint32_t nsplit = 0;
    uint64_t split_off_offset = 0, split_R_offset = 0;
    if (h > 0) {
        off = align_up(off + up[0] * m * vb, 256);
        nsplit = static_cast<uint32_t>(up[0] - 1 < 1023 ? up[0] - 1 : 1023);
        t->info.split_offset = off;
        off = align_up(off + static_cast<uint64_t>(nsplit) * kb, 256);
        t->info.split_inv_offset = off;
        off = align_up(off + (static_cast<uint64_t>(nsplit) + 1) * 4, 256);
        if (kb == 32) {
            split_off_offset = off;
            off = align_up(off + static_cast<uint64_t>(nsplit) + 1, 256);
        }
        split_R_offset = off;
        off = align_up(off + ((1ull << 12) + 1) * 2, 256);
    }
    t->info.nsplit = nsplit;
    d.nsplit = nsplit;
    t->info.device_bytes = off;

    // Descent launch defaults: 8 warps per block, top levels up to 16 KB
    // kept in shared memory (bt_tree_set_launch / bt_autotune change them).
    d.warps = 8;
    d.lane_queries = 1;
    d.staging = BT_STAGE_PIPELINED;
    d.inner_stage = 2;  // staged for partitioned batches, through L1 otherwise
    d.corun_descent_bps = 0;
    d.corun_partition_bps = 0;
    {
        int dev = 0, l2 = 0;
        const bool known = cudaGetDevice(&dev) == cudaSuccess &&
                           cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess && l2 > 0;
        d.sort_pays = (!known || off > static_cast<uint64_t>(l2) / 4) ? 1 : 0;
    }
    set_pin_levels(d, t->info, 16384);

    // Shape arithmetic: children (or keys, for leaves) per node.
    for (int l = 0; l < h; ++l) {
        const uint64_t N = d.nodes[l];
        const uint64_t below = (l + 1 < h) ? d.nodes[l + 1] : n;
        d.cbase[l] = below / N;
        d.crem[l] = below % N;
    }

    if (off == 0) {  // empty tree: nothing on the device
        *out = t;
        return BT_OK;
    }

    unsigned char *img = static_cast<unsigned char *>(malloc(off));
    if (!img) {
        delete t;
        return BT_ERR_NOMEM;
    }
    memset(img, 0, off);

    // Leaves: keys and values, padding key slots with all-ones.
    const int leaf = h - 1;
    const uint64_t L = d.nodes[leaf];
    void *lk = img + t->info.level_key_offset[leaf];
    void *lv = img + t->info.leaf_val_offset;
    std::vector<uint64_t> node_max(L);  // index of the largest key under each node
    {
        uint64_t first = 0;
        for (uint64_t i = 0; i < L; ++i) {
            const uint64_t cnt = d.cbase[leaf] + (i < d.crem[leaf] ? 1 : 0);
            for (uint64_t j = 0; j < m; ++j) {
                if (j < cnt) {
                    store_key(lk, i * m + j, kb, h_keys, first + j);
                    store_uint(lv, i * m + j, vb, load_uint(h_vals, first + j, vb));
                } else {
                    store_pad(lk, i * m + j, kb);
                }
            }
            node_max[i] = first + cnt - 1;
            first += cnt;
        }
    }
    // Partition splitters and the reciprocal widths of the segments they bound.
    {
        void *sk = img + t->info.split_offset;
        float *sinv = reinterpret_cast<float *>(img + t->info.split_inv_offset);
        std::vector<uint64_t> sidx(nsplit);  // key index of each splitter
        for (uint32_t j = 0; j < nsplit; ++j) {
            sidx[j] = node_max[(static_cast<uint64_t>(j) + 1) * L / (nsplit + 1) - 1];
            store_key(sk, j, kb, h_keys, sidx[j]);
        }
        for (uint32_t c = 0; c <= nsplit; ++c) {
            const uint64_t lo = c ? sidx[c - 1] : 0, hi = c < nsplit ? sidx[c] : n - 1;
            double width;
            if (kb == 32) {
                // 8 bytes after the bytes every key of the segment shares
                const unsigned char *a = key_ptr(h_keys, lo, kb), *b = key_ptr(h_keys, hi, kb);
                int p = 0;
                while (p < 24 && a[p] == b[p]) ++p;
                img[split_off_offset + c] = static_cast<unsigned char>(p);
                width = static_cast<double>(be64(b + p) - be64(a + p));
            } else {
                width = static_cast<double>(load_uint(h_keys, hi, kb) - load_uint(h_keys, lo, kb));
            }
            sinv[c] = static_cast<float>(1.0 / (width + 1.0));
        }
        // pre-index: R[j] = splitters whose leading 12 bits above the smallest
        // key are < j.  32-byte keys take those bits from the 8 bytes after
        // the p0 bytes every key shares.
        int p0 = 0;
        uint64_t wmin = d.kmin, wmax = d.kmax;
        if (kb == 32) {
            const unsigned char *a = key_ptr(h_keys, 0, kb), *b = key_ptr(h_keys, n - 1, kb);
            while (p0 < 24 && a[p0] == b[p0]) ++p0;
            wmin = be64(a + p0);
            wmax = be64(b + p0);
        }
        d.split_p0 = p0;
        d.split_wmin = wmin;
        const uint64_t range = wmax - wmin;
        int rl = 0;
        while (rl < 64 && (range >> rl) != 0) ++rl;
        d.split_rshift = rl > 12 ? rl - 12 : 0;
        uint16_t *R = reinterpret_cast<uint16_t *>(img + split_R_offset);
        uint32_t c = 0;
        for (uint32_t j = 0; j <= (1u << 12); ++j) {
            while (c < nsplit) {
                const uint64_t w = kb == 32 ? be64(key_ptr(h_keys, sidx[c], kb) + p0) : load_uint(sk, c, kb);
                if (((w - wmin) >> d.split_rshift) >= j) break;
                ++c;
            }
            R[j] = static_cast<uint16_t>(c);
        }
    }
    // Inner levels bottom-up: separator j = largest key under child j.
    for (int l = leaf - 1; l >= 0; --l) {
        const uint64_t N = d.nodes[l];
        void *ik = img + t->info.level_key_offset[l];
        std::vector<uint64_t> upper_max(N);
        uint64_t first = 0;
        for (uint64_t i = 0; i < N; ++i) {
            const uint64_t span = d.cbase[l] + (i < d.crem[l] ? 1 : 0);
            for (uint64_t j = 0; j < m; ++j) {
                if (j + 1 < span)
                    store_key(ik, i * m + j, kb, h_keys, node_max[first + j]);
                else
                    store_pad(ik, i * m + j, kb);
            }
            upper_max[i] = node_max[first + span - 1];
            first += span;
        }
        node_max.swap(upper_max);
    }

    cudaError_t e = cudaMalloc(&t->d_image, off);
    if (e != cudaSuccess) {
        set_error_detail("cudaMalloc(tree image)", e);
        free(img);
        delete t;
        return e == cudaErrorMemoryAllocation ? BT_ERR_NOMEM : BT_ERR_CUDA;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(t->d_image, img, off, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    free(img);
    if (e != cudaSuccess) {
        set_error_detail("copy of tree image to device", e);
        cudaFree(t->d_image);
        delete t;
        return BT_ERR_CUDA;
    }
    for (int l = 0; l < h; ++l)
        d.keys[l] = static_cast<unsigned char *>(t->d_image) + t->info.level_key_offset[l];
    d.vals = static_cast<unsigned char *>(t->d_image) + t->info.leaf_val_offset;
    d.split = static_cast<unsigned char *>(t->d_image) + t->info.split_offset;
    d.split_inv = reinterpret_cast<const float *>(static_cast<unsigned char *>(t->d_image) + t->info.split_inv_offset);
    d.split_off = kb == 32 ? static_cast<unsigned char *>(t->d_image) + split_off_offset : nullptr;
    d.split_R = reinterpret_cast<const uint16_t *>(static_cast<unsigned char *>(t->d_image) + split_R_offset);
    t->info.d_image = t->d_image;
    *out = t;
    return BT_OK;
}

extern "C" void bt_free(bt_tree *t)
{
    if (!t) return;
    if (t->d_image) cudaFree(t->d_image);
    if (t->d_paper) cudaFree(t->d_paper);
    delete t;
}

extern "C" uint32_t bt_paper_node_bytes(uint32_t fanout, bt_width key_w)
{
    const uint64_t w = static_cast<uint64_t>(key_w), m = fanout;
    if ((w != 4 && w != 8 && w != 32) || m < 3 || m > 64) return 0;
    const uint64_t keys = align_up(w * (m - 1), 8);
    return static_cast<uint32_t>(align_up(32 + keys + 8 * m, 32));
}

extern "C" bt_status bt_paper_layout_build(bt_tree *t, bt_stream stream)
{
    if (!t) return BT_ERR_ARG;
    if (t->d_paper || t->dev.height == 0) return BT_OK;
    const DevTree &d = t->dev;
    const int h = d.height, kb = d.key_bytes, vb = d.val_bytes;
    const uint64_t m = static_cast<uint64_t>(d.m);
    const uint32_t nb = bt_paper_node_bytes(static_cast<uint32_t>(m), static_cast<bt_width>(kb));
    const uint64_t child_off = 32 + align_up(static_cast<uint64_t>(kb) * (m - 1), 8);
    uint64_t first[BT_MAX_LEVELS + 1];
    first[0] = 0;
    for (int l = 0; l < h; ++l) first[l + 1] = first[l] + d.nodes[l];
    const uint64_t bytes = first[h] * nb;
    std::vector<unsigned char> soa(t->info.device_bytes);
    cudaError_t e = cudaMemcpy(soa.data(), t->d_image, soa.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_error_detail("copy of tree image to host", e);
        return BT_ERR_CUDA;
    }
    unsigned char *img = static_cast<unsigned char *>(calloc(bytes, 1));
    if (!img) return BT_ERR_NOMEM;
    for (int l = 0; l < h; ++l) {
        const bool leaf = (l + 1 == h);
        const unsigned char *lk = soa.data() + t->info.level_key_offset[l];
        for (uint64_t i = 0; i < d.nodes[l]; ++i) {
            unsigned char *node = img + (first[l] + i) * nb;
            const uint64_t span = d.cbase[l] + (i < d.crem[l] ? 1 : 0);  // children, or keys of a leaf
            const uint32_t use = static_cast<uint32_t>(leaf ? span : span - 1);
            const uint32_t depth = static_cast<uint32_t>(l);
            memcpy(node, &use, 4);
            memcpy(node + 4, &depth, 4);
            memcpy(node + 32, lk + i * m * kb, (m - 1) * kb);  // slots beyond `use` are all-ones already
            uint64_t *slots = reinterpret_cast<uint64_t *>(node + child_off);
            if (leaf) {
                const unsigned char *lv = soa.data() + t->info.leaf_val_offset + i * m * vb;
                for (uint64_t j = 0; j < span; ++j) slots[j] = load_uint(lv, j, vb);
            } else {
                const uint64_t c0 = i * d.cbase[l] + (i < d.crem[l] ? i : d.crem[l]);
                for (uint64_t j = 0; j < span; ++j) slots[j] = (first[l + 1] + c0 + j) * nb;
            }
        }
    }
    void *dp = nullptr;
    e = cudaMalloc(&dp, bytes);
    if (e != cudaSuccess) {
        free(img);
        set_error_detail("cudaMalloc(paper layout)", e);
        return e == cudaErrorMemoryAllocation ? BT_ERR_NOMEM : BT_ERR_CUDA;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(dp, img, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    free(img);
    if (e != cudaSuccess) {
        cudaFree(dp);
        set_error_detail("copy of paper layout to device", e);
        return BT_ERR_CUDA;
    }
    PaperTree &p = t->paper;
    p.base = static_cast<const unsigned char *>(dp);
    p.node_bytes = nb;
    p.child_off = static_cast<uint32_t>(child_off);
    p.height = h;
    p.pin_levels = 0;
    p.pin_bytes = 0;
    for (int l = 0; l + 1 < h && first[l + 1] * nb <= 16384; ++l) {
        p.pin_levels = l + 1;
        p.pin_bytes = static_cast<uint32_t>(first[l + 1] * nb);
    }
    t->d_paper = dp;
    return BT_OK;
}

extern "C" bt_status bt_tree_info(const bt_tree *t, bt_info *out)
{
    if (!t || !out) return BT_ERR_ARG;
    *out = t->info;
    return BT_OK;
}

extern "C" bt_status bt_tree_copy_image(const bt_tree *t, void *h_dst, uint64_t bytes)
{
    if (!t || (!h_dst && bytes)) return BT_ERR_ARG;
    if (bytes > t->info.device_bytes) return BT_ERR_ARG;
    if (bytes == 0) return BT_OK;
    cudaError_t e = cudaMemcpy(h_dst, t->d_image, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_error_detail("copy of tree image to host", e);
        return BT_ERR_CUDA;
    }
    return BT_OK;
}
