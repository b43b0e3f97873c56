// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "btree_gb300.h"
#include "keys.cuh"
#include "learned.cuh"

namespace btgb {

// Device-side description of a built tree, passed to kernels by value.
//
// Nodes of level l are numbered 0..nodes[l]-1 left to right.  The even bulk
// load makes the shape arithmetic: inner node i of level l owns children
// first_child(l, i) .. first_child(l, i) + span(l, i) - 1 of level l+1, with
// span(l, i) = cbase[l] + (i < crem[l]) and
// first_child(l, i) = i * cbase[l] + min(i, crem[l]).  For the leaf level the
// same two numbers split the n keys over the leaves, so leaf i holds
// cbase + (i < crem) keys.  No child pointers are stored (Sec. IV-B embeds
// child addresses in each node; here they follow from the node's index).
struct DevTree {
    const void *keys[BT_MAX_LEVELS];   // level key blocks, m slots per node
    uint64_t nodes[BT_MAX_LEVELS];
    uint64_t cbase[BT_MAX_LEVELS];
    uint64_t crem[BT_MAX_LEVELS];
    const void *vals;                  // leaf value blocks, m slots per leaf
    uint64_t kmin, kmax;               // smallest and largest key (integer keys)
    uint64_t kmin32[4], kmax32[4];     // the same for 32-byte keys, as Key32 words
    int height;
    int m;
    int key_bytes, val_bytes;
    int pin_levels;      // top levels copied to shared memory by the descent
    uint32_t pin_bytes;  // bytes from the root's block to the end of those levels
    int warps;           // warps per descent block
    int staging;         // BT_STAGE_*: pipelined (default), or synchronous with cp.async / bulk copies
    int lane_queries;    // queries per lane of the plain descent: 1 (32 per warp) or 2 (64 per warp)
    int inner_stage;     // pipelined descent: inner levels through L1 (0), staged with cp.async (1), or
                         // staged for partitioned batches and through L1 otherwise (2)
    int rank_ballot;     // pipelined descent: leaf rank by binary search (0) or warp ballot + popc (1)
    // Resident blocks per SM at most (0: as many as fit) of the descent and
    // of the partition, so that one batch's partition can run beside the
    // previous batch's descent (bt_tree_set_corun).
    int corun_descent_bps;
    int corun_partition_bps;
    // 1 when the tree's device image is larger than a quarter of the
    // device's L2: only then does the automatic choice partition large
    // batches (a smaller tree's leaves stay in the L2 between batches, and
    // the unsorted descent reads them from there faster than the partition
    // takes).
    int sort_pays;
    // Splitters of the batch partition: the largest keys of nsplit evenly
    // spaced leaves, and nsplit + 1 reciprocal widths of the key segments
    // they bound (part_sort.cuh).
    const void *split;
    const float *split_inv;
    const unsigned char *split_off;  // 32-byte keys: bytes shared within each segment
    const uint16_t *split_R;         // splitter pre-index by leading key bits
    int split_rshift;
    int split_p0;                    // 32-byte keys: bytes all keys share (leading bits follow them)
    uint64_t split_wmin;             // 32-byte keys: the 8 bytes after them in the smallest key
    uint32_t nsplit;
};

// The same tree in the paper's node layout (Eq. 1, Fig. 3): one array of
// equal-size nodes in BFS order (root first, level by level, left to
// right).  A node: a 32-byte header (uint32 slotUse = keys or separators in
// use, uint32 depth = level), then k_max = m - 1 key slots (device key form,
// unused slots all-ones) padded to 8 bytes, then for inner nodes m 8-byte
// child addresses (byte offsets from the array's start) and for leaves
// k_max 8-byte data slots (the value, zero-extended) plus 8 unused bytes;
// the node size is rounded up to whole 32-byte chunks (Sec. IV-B).
struct PaperTree {
    const unsigned char *base;
    uint32_t node_bytes;
    uint32_t child_off;   // byte offset of the child addresses / data slots in a node
    int height;
    int pin_levels;       // top levels copied to shared memory by the descent
    uint32_t pin_bytes;   // bytes of those levels (a prefix of the array)
};

// Whole top levels (never the leaves) whose bytes fit `budget`, root first.
void set_pin_levels(DevTree &d, const bt_info &info, uint32_t budget);

// Host-side launch facts, cached per device and safe to call from any
// thread: the current device's SM count, resident blocks per SM of a kernel
// at a block shape, and the kernel's dynamic shared-memory limit raised to
// `bytes` (once per device and kernel).
cudaError_t dev_sm_count(int *sms);
cudaError_t blocks_per_sm(const void *kern, int threads, int dyn_smem, int *out);
cudaError_t ensure_dyn_smem(const void *kern, int bytes);

// Poll limit of the first bounded wait in the descent (bt_debug_set_wait_polls).
uint32_t first_wait_polls();

}  // namespace btgb

struct bt_tree {
    btgb::DevTree dev;
    bt_info info;
    void *d_image;
    // L2 access-policy window of the descent (bt_tree_set_l2_window): the
    // non-pinned inner levels, marked persisting; 0 bytes = none.
    const void *l2_base;
    uint64_t l2_bytes;
    float l2_hit_ratio;
    btgb::PaperTree paper;  // valid once d_paper is set (bt_paper_layout_build)
    void *d_paper;
};

struct bt_model {
    btgb::ModelDev dev;
    bt_model_info info;
    void *d_mem;
};

namespace btgb {
void set_error_detail(const char *what, cudaError_t err);
}
