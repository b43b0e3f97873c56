/*
 * btree_gb300.h -- C ABI of the GB300 (sm_103a) batched B+ tree search library.
 *
 * The library answers batches of point queries against a static B+ tree by
 * the level-wise batch traversal of Tzschoppe et al., "Efficient Batch Search
 * Algorithm for B+ Tree Index Structures with Level-Wise Traversal on FPGAs":
 * the batch is sorted (Sec. IV-A; here partitioned by approximate key rank,
 * see bt_sort_batch), then descends the tree one level at a time;
 * every node needed at a level is fetched once per group of queries routed to
 * it and compared against all of them (Sec. IV-A, Sec. IV-F); a query goes to
 * the first slot whose separator it is less than or equal to (Sec. IV-E); at
 * the leaf an equal key yields its data, otherwise -1 (Sec. IV-D).
 *
 * Conventions for every call:
 *   - Keys are unsigned integers of 4 or 8 bytes, compared as unsigned
 *     integers, or the paper's 32-byte keys compared byte by byte (Sec. IV-E;
 *     BT_B32).  Values are unsigned integers of 4 or 8 bytes.
 *   - "d_" pointers are device (GPU global memory) pointers owned by the
 *     caller; "h_" pointers are host pointers owned by the caller.  Nothing the
 *     caller passes is freed or retained after a call returns, except that a
 *     search reads and writes its device buffers asynchronously on `stream`
 *     until the stream reaches that point.
 *   - `stream` is a CUDA runtime stream (cudaStream_t); NULL is the legacy
 *     default stream.  The header declares it as `struct CUstream_st *`, which
 *     is what cudaStream_t is, so that it needs no CUDA header.
 *   - Device key, position and value arrays of the search, sort and descent
 *     calls are aligned to their element size (32-byte keys: to 16 bytes);
 *     a misaligned one is an argument error (BT_ERR_ARG).
 *   - Argument errors are returned synchronously and leave outputs untouched.
 *     Launch and runtime failures of the CUDA runtime are returned as
 *     BT_ERR_CUDA; bt_last_error_detail() then names the failing call.
 *   - A built tree is immutable: searches on different streams with separate
 *     workspaces may run concurrently against one tree.
 */
#ifndef BTREE_GB300_H
#define BTREE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *bt_stream;

/* Key and value widths in bytes.  BT_B32 (keys only) is the paper's 32-byte key
 * (Sec. IV-B, IV-E): a string of 32 bytes compared byte by byte from the
 * first, the first unequal byte deciding (lexicographic order, as memcmp);
 * key arrays and query arrays hold 32 bytes per key, as they are. */
typedef enum bt_width { BT_U32 = 4, BT_U64 = 8, BT_B32 = 32 } bt_width;

typedef enum bt_status {
    BT_OK = 0,
    BT_ERR_ARG = 1,        /* null pointer, bad width, size out of range */
    BT_ERR_UNSORTED = 2,   /* build keys not in ascending order */
    BT_ERR_DUPLICATE = 3,  /* two equal build keys */
    BT_ERR_FANOUT = 4,     /* fanout not in {8, 16, 32, 64} */
    BT_ERR_NOMEM = 5,      /* host or device allocation failed */
    BT_ERR_CUDA = 6,       /* a CUDA runtime call failed */
    BT_ERR_TIMEOUT = 7,    /* a bounded device wait gave up */
    BT_ERR_WORKSPACE = 8   /* workspace missing or smaller than required */
} bt_status;

#define BT_MAX_LEVELS 24

/* Opaque, immutable after bt_build. */
typedef struct bt_tree bt_tree;

/* Opaque learned leaf predictor of one tree (see bt_model_train). */
typedef struct bt_model bt_model;

/* Shape of a built tree.  Level 0 is the root, level height-1 the leaves. */
typedef struct bt_info {
    uint32_t height;                       /* number of levels; 0 for an empty tree */
    uint32_t fanout;                       /* m: max children of an inner node */
    uint32_t key_bytes;                    /* 4, 8 or 32 */
    uint32_t val_bytes;                    /* 4 or 8 */
    uint64_t n;                            /* keys stored */
    uint64_t level_nodes[BT_MAX_LEVELS];   /* nodes per level */
    uint64_t level_key_offset[BT_MAX_LEVELS]; /* byte offset of the level's key blocks */
    uint64_t leaf_val_offset;              /* byte offset of the leaf value blocks */
    uint64_t device_bytes;                 /* size of the device image */
    uint64_t split_offset;                 /* byte offset of the partition splitters */
    uint64_t split_inv_offset;             /* byte offset of their fp32 segment reciprocals */
    uint32_t nsplit;                       /* number of splitters (0..1023) */
    uint32_t reserved;
    const void *d_image;                   /* device address of the image (read-only) */
} bt_info;

/*
 * bt_build -- bulk-load a static tree from sorted keys (Sec. IV-B: the tree
 * is built on the host once and transferred to device memory once; Sec. V-B).
 *
 *   h_keys   n keys of key_w bytes, strictly ascending (host, read only).
 *   h_vals   n values of val_w bytes, value i belongs to key i (host).
 *   n        number of keys; 0 builds an empty tree in which every query
 *            misses.  Every level must hold fewer than 2^32 nodes.
 *   key_w    BT_U32, BT_U64 or BT_B32.
 *   val_w    BT_U32 or BT_U64.
 *   fanout   m in {8, 16, 32, 64}: inner nodes hold up to m children and
 *            m-1 separators, leaves up to m-1 keys (Sec. III).
 *   stream   stream for the one host-to-device copy; the call synchronizes
 *            it before returning.
 *   out      receives the tree; free it with bt_free.
 *
 * Fill rule (the paper does not state one): L = ceil(n/(m-1)) leaves with the
 * keys spread as evenly as possible (larger leaves first), parents likewise
 * over ceil(C/m) nodes until one is left; separator i of an inner node is the
 * largest key under its child i.
 *
 * Device layout (structure of arrays, one allocation): for each level, root
 * first, a block of m key slots per node (m * key_w bytes), then for the
 * leaves a block of m value slots per leaf; every level array starts on a
 * 256-byte boundary, so blocks of 128 bytes or more start on a 128-byte line.
 * Unused key slots hold all-ones and are excluded from leaf matches by the
 * leaf's key count, so the all-ones key itself is legal.  A 32-byte key
 * slot holds four 64-bit words, most significant first, word j the
 * big-endian value of key bytes 8j..8j+7 (comparing the words in order as
 * unsigned integers compares the bytes lexicographically).  After the values
 * (each 256-byte aligned): the batch partition's splitters, nsplit =
 * min(L - 1, 1023) keys, splitter j the largest key of leaf
 * floor((j + 1) L / (nsplit + 1)) - 1; then nsplit + 1 fp32 values,
 * 1 / (hi - lo + 1) for each key segment (lo, hi] the splitters bound
 * (segment 0 starts at the smallest key, the last ends at the largest); for
 * 32-byte keys lo and hi are the big-endian values of the 8 bytes after the
 * p bytes the segment's bounds share (p <= 24), and nsplit + 1 bytes p
 * follow; then 4097 uint16 R[j] = the number of splitters whose leading 12
 * bits above the smallest key are below j (32-byte keys: bits of the 8 bytes
 * after the bytes all keys share).
 *
 * Errors: BT_ERR_ARG, BT_ERR_FANOUT, BT_ERR_UNSORTED, BT_ERR_DUPLICATE,
 * BT_ERR_NOMEM, BT_ERR_CUDA.  *out is set only on BT_OK.
 */
bt_status bt_build(const void *h_keys, const void *h_vals, uint64_t n, bt_width key_w,
                   bt_width val_w, uint32_t fanout, bt_stream stream, bt_tree **out);

/* Release a tree and its device memory (NULL is a no-op).  The caller must
 * make sure no search using it is still running.  No counterpart in the
 * paper (its tree lives for the whole run). */
void bt_free(bt_tree *tree);

/* Copy the tree's shape into *out (levels and node counts as in Sec. III:
 * height h, nodes per level).  BT_ERR_ARG on null pointers. */
bt_status bt_tree_info(const bt_tree *tree, bt_info *out);

/* Copy the first `bytes` of the device image into host memory (for layout
 * checks); synchronous.  BT_ERR_ARG if bytes exceeds the image. */
bt_status bt_tree_copy_image(const bt_tree *tree, void *h_dst, uint64_t bytes);

/* Bytes of device workspace bt_search_batch needs for a batch of nq queries
 * (the partitioned batch, its local-sort digits and the partition's bucket
 * counters).  Depends only on the tree's key width and nq; 0 for a NULL tree
 * or nq = 0.  No counterpart in the paper (its batch lives in on-chip BRAM,
 * Sec. IV-C). */
uint64_t bt_search_workspace_bytes(const bt_tree *tree, uint64_t nq);

/* Options for bt_search_batch_ex. */
typedef struct bt_search_opts {
    /* Bits of the bucket number the batch is partitioned on before the
     * descent (Sec. IV-A sorts the batch so that queries for one node are
     * adjacent; see bt_sort_batch for the order obtained): -1 lets the
     * library choose (none below 786432 queries -- 393216 for 32-byte
     * keys -- and none for a tree whose device image is at most a quarter of
     * the L2: the partition pays for itself only when the batch is large and
     * leaf blocks do not stay in the L2 between batches), 0 skips the
     * partition, 1..21 forces that many bits (larger values mean 21). */
    int32_t sort_bits;
    /* If non-NULL: device array of `height` counters to which the search
     * adds, per level, how many node key blocks it fetched -- the quantity
     * the paper's method keeps near the number of distinct nodes (Sec. IV-A).
     * Counting adds one atomic per warp and level. */
    unsigned long long *d_fetch_counts;
    /* If non-NULL: a CUDA event (cudaEvent_t) recorded on the stream between
     * the partition and the descent, so that a caller can time the two phases
     * of one call with its own events around it. */
    void *phase_event;
} bt_search_opts;

/*
 * bt_search_batch -- point lookups for a batch of queries, results in input
 * order (Sec. IV-D: the data of the equal key, or -1).
 *
 *   d_queries    nq keys of the tree's key width (device).
 *   nq           batch size, 0 <= nq < 2^31; 0 returns BT_OK and does nothing.
 *   d_out_vals   nq values of the tree's value width (device): the value of
 *                the equal key, or all-ones on a miss.
 *   d_out_found  nq bytes (device): 1 on a hit, 0 on a miss (a stored
 *                all-ones value stays distinguishable from a miss).
 *   d_workspace  at least bt_search_workspace_bytes(tree, nq) bytes of device
 *                memory, 256-byte aligned; contents need not be initialised
 *                and are clobbered.  It may be NULL only if that size is 0.
 *   ws_bytes     size of d_workspace.
 *
 * Asynchronous on `stream`; allocates nothing, so it may be captured in a
 * CUDA graph.  Queries and outputs must not overlap the workspace.
 * Errors: BT_ERR_ARG, BT_ERR_WORKSPACE, BT_ERR_CUDA.
 */
bt_status bt_search_batch(const bt_tree *tree, const void *d_queries, uint64_t nq,
                          void *d_out_vals, uint8_t *d_out_found, void *d_workspace,
                          uint64_t ws_bytes, bt_stream stream);

/* bt_search_batch with options (opts may be NULL = defaults). */
bt_status bt_search_batch_ex(const bt_tree *tree, const void *d_queries, uint64_t nq,
                             void *d_out_vals, uint8_t *d_out_found, void *d_workspace,
                             uint64_t ws_bytes, const bt_search_opts *opts,
                             bt_stream stream);

/*
 * bt_sort_batch -- the first step of a search on its own: the on-device
 * partition of the batch (Sec. IV-A: queries are sorted so that those
 * routed to one node are adjacent).  Writes the reordered queries and, for
 * each, its input position.  The order is that of a bucket number f monotone
 * in the key, on `bits` bits: sort_bits when positive (values above 21 mean
 * 21), none for 0 (the queries are copied and the index is the identity),
 * and for -1 the library's choice, which bt_sort_bits reports (none below
 * 786432 queries (393216 for 32-byte keys) or for a tree whose device image
 * is at most a quarter of the L2; otherwise coarse buckets of 512 to 1023
 * queries on average):
 *   f(q) = (c << r) | s, where c = the number of the tree's splitters
 *   (bt_info.nsplit keys, see bt_build) smaller than q, and s = the fp32
 *   product (q - lo) * inv_c * 2^r truncated and clamped to [0, 2^r - 1],
 *   with (lo, hi] the splitter segment holding q and inv_c its stored
 *   reciprocal width (32-byte keys: q - lo over the 8 bytes after the
 *   segment's shared prefix); r = bits - bitlen(nsplit) when positive,
 *   else f = c >> (bitlen(nsplit) - bits).
 * The batch is ordered by the coarse bucket f >> lb, lb = min(9, bits - 1),
 * and inside every coarse bucket of at most 1024 queries (the local sort's
 * tile) by f.  The order of queries with equal f, and inside larger coarse
 * buckets (a hot key, or automatic bits on batches from about 2^22 queries,
 * where the 2^12 coarse buckets grow past the tile) the order of queries
 * with equal coarse buckets, is
 * unspecified (it follows device atomics and may differ between calls).
 * One cooperative kernel (coarse counts, scatter, per-bucket local sort,
 * with two bounded grid barriers; see bt_check_timeouts) after one memset of
 * the coarse-bucket counters; for integer keys bt_sort_batch adds one kernel
 * that writes the two output arrays (32-byte keys are written into them by
 * the partition itself).
 *
 *   d_queries         nq keys (device).
 *   d_sorted_queries  nq keys (device), must not overlap d_queries.
 *   d_sorted_index    nq uint32 input positions (device).
 *   d_workspace       bt_search_workspace_bytes(tree, nq) bytes, 256-aligned.
 * Asynchronous on `stream`; allocates nothing.
 * Errors: BT_ERR_ARG, BT_ERR_WORKSPACE, BT_ERR_CUDA.
 */
bt_status bt_sort_batch(const bt_tree *tree, const void *d_queries, uint64_t nq, int32_t sort_bits,
                        void *d_sorted_queries, uint32_t *d_sorted_index, void *d_workspace,
                        uint64_t ws_bytes, bt_stream stream);

/* Number of kernels the partition of bt_sort_batch / bt_search_batch
 * launches for this tree, batch size and sort_bits (0 = no partition; it
 * also issues one cudaMemsetAsync of its bucket counters).  -1 on a NULL
 * tree. */
int32_t bt_sort_launches(const bt_tree *tree, uint64_t nq, int32_t sort_bits);

/* Bits of the bucket number f that bt_sort_batch / bt_search_batch order a
 * batch of nq queries on, for this sort_bits (-1 = the library's choice);
 * 0 = no partition.  -1 on a NULL tree.  No counterpart in the paper. */
int32_t bt_sort_bits(const bt_tree *tree, uint64_t nq, int32_t sort_bits);

/*
 * bt_descend_sorted -- the remaining steps on their own: the level-wise
 * descent (Sec. IV-A, IV-E, IV-F), the leaf probe (Sec. IV-D) and the
 * scatter of every result to position d_index[i] of the outputs.
 *
 *   d_queries     nq keys (device), ideally the output of bt_sort_batch;
 *                 any order gives the same results, sorting only buys node
 *                 reuse.
 *   d_index       nq uint32 output positions (device), a permutation of
 *                 0..nq-1, or NULL for the identity.
 *   d_out_vals, d_out_found   as in bt_search_batch.
 *   d_fetch_counts   NULL, or `height` device counters (see bt_search_opts).
 * Asynchronous on `stream`; needs no workspace.
 * Errors: BT_ERR_ARG, BT_ERR_CUDA.
 */
bt_status bt_descend_sorted(const bt_tree *tree, const void *d_queries, const uint32_t *d_index,
                            uint64_t nq, void *d_out_vals, uint8_t *d_out_found,
                            unsigned long long *d_fetch_counts, bt_stream stream);

/* Workspace for bt_search_batch_host: device room for the queries and
 * results plus bt_search_workspace_bytes. */
uint64_t bt_search_host_workspace_bytes(const bt_tree *tree, uint64_t nq);

/*
 * bt_search_batch_host -- the same lookup from host buffers: copies h_queries
 * to the device, searches, and copies the results back, all enqueued on
 * `stream` (the paper's per-batch host write, kernel, host read; Sec. V-B).
 * The call returns once the work is enqueued: synchronize `stream` before
 * reading h_out_vals / h_out_found.  Page-locked host buffers make the
 * copies asynchronous; pageable ones work but the copies then block.
 *
 *   h_queries, h_out_vals, h_out_found   host buffers of nq entries.
 *   d_workspace  bt_search_host_workspace_bytes(tree, nq) bytes of device
 *                memory, 256-byte aligned.
 * Errors: as bt_search_batch.
 */
bt_status bt_search_batch_host(const bt_tree *tree, const void *h_queries, uint64_t nq,
                               void *h_out_vals, uint8_t *h_out_found, void *d_workspace,
                               uint64_t ws_bytes, bt_stream stream);

/*
 * bt_search_batch_noalloc -- bt_search_batch without a caller workspace and
 * without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory, such as a
 * query engine or plugin host that owns every device buffer through its own
 * arena and hands a library only input and output pointers, or a latency-
 * critical request path that must not call cudaMalloc/cudaFree (they can
 * synchronize the whole device).
 *
 * Scratch space (the partitioned batch and the bucket counters) is a 4 MiB
 * file-scope device array inside the library; every GPU that loads the
 * library holds it until the process exits.  The caller still passes the
 * queries and the outputs, as for bt_search_batch.
 *
 *   nq   at most BT_NOALLOC_MAX_QUERIES; larger batches are rejected with
 *        BT_ERR_ARG (bt_last_error_detail says why) -- use bt_search_batch
 *        with a workspace for them.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  All calls share the one array
 * and it keeps the last call's contents (each search clears what must start
 * at zero), so calls whose work overlaps on the GPU -- on different streams,
 * or from different threads -- race and must be serialised by the caller.
 * Errors: as bt_search_batch, plus BT_ERR_ARG for nq > BT_NOALLOC_MAX_QUERIES
 * and BT_ERR_WORKSPACE when the batch's scratch would exceed the array (it
 * does not at up to BT_NOALLOC_MAX_QUERIES queries: 65536 32-byte-key
 * queries need 2.9 MB, integer keys 1.1 MB).
 */
#define BT_NOALLOC_MAX_QUERIES 65536
bt_status bt_search_batch_noalloc(const bt_tree *tree, const void *d_queries, uint64_t nq,
                                  void *d_out_vals, uint8_t *d_out_found, bt_stream stream);

/* ------------------------------------------------------------------------
 * Many batches over several resident trees in one launch.  Not in the paper
 * as such: it extends the paper's use of several kernel instances, each
 * serving a share of the work (Sec. IV-G), to many small batches of uneven
 * size addressed to different trees, served by one persistent launch.
 * ------------------------------------------------------------------------ */

/* One batch of a work list: `count` queries at d_queries[offset ..], whose
 * results go to the same positions of the result arrays, searched in tree
 * number `tree` of the forest. */
typedef struct bt_batch_desc {
    uint32_t tree;
    uint32_t count;
    uint64_t offset;
} bt_batch_desc;

typedef struct bt_forest bt_forest;

/* A table of `count` built trees with equal key and value widths (fanouts
 * may differ; integer keys only: BT_ERR_ARG for 32-byte keys).  Each tree
 * brings its own launch settings as bt_autotune (or bt_tree_set_launch,
 * bt_tree_set_staging, bt_tree_set_lane_queries, bt_tree_set_descent) left
 * them: its pinned top levels (trimmed, deepest level of the tree pinning
 * most first, until all trees' pinned levels fit the forest's shared-memory
 * budget), its queries per lane, and whether the levels below the pinned
 * ones are staged per warp (the synchronous designs and inner-staged
 * pipelined design) or read lane by lane through L1 (the pipelined design).
 * Warps per block default to the setting of the tree with the most keys,
 * the pin budget to 32 KB.  The trees must outlive the forest.
 * Errors: BT_ERR_ARG, BT_ERR_NOMEM, BT_ERR_CUDA. */
bt_status bt_forest_create(const bt_tree *const *trees, uint32_t count, bt_forest **out);

/* The same with a learned leaf predictor per tree: models[i] NULL (plain
 * descent) or a model trained on trees[i] (BT_ERR_ARG otherwise, or for a
 * model on an empty tree).  A query whose model window proves its leaf
 * skips the inner levels, the others walk them (bt_learned_search_batch's
 * rule, applied lane by lane); trees with a model are read through L1.
 * Models must outlive the forest. */
bt_status bt_forest_create_learned(const bt_tree *const *trees, const bt_model *const *models, uint32_t count,
                                   bt_forest **out);
void bt_forest_free(bt_forest *forest);

/* Launch settings of a forest. */
typedef struct bt_forest_tune {
    uint32_t warps_per_block; /* 1..16 */
    uint32_t pin_budget;      /* shared-memory bytes for all trees' pinned levels, 0..98304 */
    uint32_t lane_queries;    /* 0: each tree's own, 1 or 2: that many queries per lane for all trees */
    uint32_t staging;         /* 0: each tree's own design, 1: all read through L1, 2: all staged per warp */
    uint32_t pin_applied;     /* out: bytes of pinned levels the budget admitted */
    float us;                 /* out (bt_forest_autotune): device time per call of the work list */
} bt_forest_tune;

/* Replace a forest's launch settings (synchronizes the device; CUDA graphs
 * captured before keep the old shape and must be captured again).
 * Errors: BT_ERR_ARG (null or out-of-range values), BT_ERR_CUDA. */
bt_status bt_forest_set_launch(bt_forest *forest, const bt_forest_tune *settings);
bt_status bt_forest_get_launch(const bt_forest *forest, bt_forest_tune *out);

/* Device workspace for a work list of nbatches batches. */
uint64_t bt_forest_workspace_bytes(uint32_t nbatches);

/*
 * bt_forest_search -- every batch of the device work list d_batches[0..n) in
 * one persistent launch: the batches' chunks (32 queries, or 64 for a tree
 * at two queries per lane) are shared out over resident warps; each chunk
 * descends its tree level by level (Sec. IV-A) -- pinned levels from the
 * block's shared copy, the others staged per warp (each distinct node of the
 * chunk loaded once) or read through L1 (lanes sharing a node share its
 * lines) -- and writes value and found flag at its queries' positions.
 * Batches are not sorted (they are small, and unsorted chunks meet many
 * nodes per level).
 *   d_queries        nq keys (device); results go to the same positions of
 *                    d_out_vals / d_out_found (nq entries each).
 *   nq               length of those three arrays.
 *   warps_per_block  1..16, 0 = the forest's setting.
 * Each work-list entry must name a tree below the forest's count and lie
 * inside the arrays (offset + count <= nq).  The kernel checks both: an
 * entry that breaks either is skipped (nothing is written for it) and
 * counted (bt_forest_bad_batches).
 * Asynchronous, allocates nothing, may be captured in a CUDA graph.
 * Errors: BT_ERR_ARG, BT_ERR_WORKSPACE, BT_ERR_CUDA.
 */
bt_status bt_forest_search(const bt_forest *forest, const bt_batch_desc *d_batches, uint32_t nbatches,
                           const void *d_queries, uint64_t nq, void *d_out_vals, uint8_t *d_out_found,
                           void *d_workspace, uint64_t ws_bytes, uint32_t warps_per_block, bt_stream stream);

/*
 * bt_forest_autotune -- time the work list (arguments as bt_forest_search)
 * under every combination of warps per block {4, 8, 16}, pin budget
 * {0, 16384, 49152, 98304}, queries per lane {each tree's, 1, 2} and
 * staging {each tree's, all through L1, all staged}; keep the fastest (after 2
 * untimed calls, 3 runs of 5 calls issued back to back behind a short device
 * spin, timed together with CUDA events on `stream`; the median per call) as
 * the forest's settings and return it in *best.  Synchronizes the device.  No counterpart
 * in the paper (its kernel's shape is fixed by the FPGA build).
 * Errors: as bt_forest_search.
 */
bt_status bt_forest_autotune(bt_forest *forest, const bt_batch_desc *d_batches, uint32_t nbatches,
                             const void *d_queries, uint64_t nq, void *d_out_vals, uint8_t *d_out_found,
                             void *d_workspace, uint64_t ws_bytes, bt_stream stream, bt_forest_tune *best);

/* Work-list entries that bt_forest_search skipped since the last call (a
 * tree index outside the forest, or queries beyond the arrays), read and
 * cleared; synchronous.  No counterpart in the paper.
 * Errors: BT_ERR_ARG (null out), BT_ERR_CUDA. */
bt_status bt_forest_bad_batches(uint64_t *out);

/* Launch parameters of a tree's single-tree searches. */
typedef struct bt_tune {
    uint32_t fanout;          /* m the tree was built with */
    uint32_t warps_per_block; /* descent blocks: 4, 8 or 16 warps */
    uint32_t pin_bytes;       /* budget for top levels kept in shared memory (0..49152) */
    uint32_t staging;         /* BT_STAGE_PIPELINED, BT_STAGE_CP_ASYNC or BT_STAGE_BULK */
    uint32_t lane_queries;    /* queries per lane of the descent: 1 or 2 */
    uint32_t inner_staged;    /* pipelined descent: inner levels staged (1) or read through L1 (0) */
    float us_per_batch;       /* device time per call of the sample batch with these settings (10 calls
                               * issued back to back, median of 5 runs) */
} bt_tune;

/* Set the descent launch parameters of a built tree (not thread-safe with
 * searches running on it): warps per descent block (1..16) and the bytes of
 * top levels each block keeps in shared memory (0..49152).  The pipelined
 * descent gives a batch with fewer 32-query chunks per SM than
 * warps_per_block smaller blocks (that many warps, at least 2), so that a
 * small batch spreads over more SMs.  BT_ERR_ARG on unsupported values. */
bt_status bt_tree_set_launch(bt_tree *tree, uint32_t warps_per_block, uint32_t pin_bytes);

/* How the descent stages node blocks into shared memory (Sec. IV-A: every
 * node a group of queries needs is loaded once):
 *   BT_STAGE_PIPELINED (the default): leaf blocks are staged by one
 *     asynchronous bulk copy each (the TMA unit), completing on the warp's
 *     mbarrier while the warp walks the next 32 queries down the inner
 *     levels; the wait is bounded (see bt_check_timeouts);
 *   BT_STAGE_CP_ASYNC: every level below the pinned ones is staged with
 *     16-byte cp.async pieces and waited for before the search, one chunk
 *     of 32 queries at a time;
 *   BT_STAGE_BULK: as BT_STAGE_CP_ASYNC with one bulk copy per node block
 *     counted on an mbarrier (bounded wait).
 * Results are identical; speed differs.  BT_ERR_ARG on other values. */
#define BT_STAGE_CP_ASYNC 0
#define BT_STAGE_BULK 1
#define BT_STAGE_PIPELINED 2
bt_status bt_tree_set_staging(bt_tree *tree, uint32_t mode);

/* Two choices of the pipelined descent (no counterpart in the paper beyond
 * Sec. IV-E's comparator row, which rank_ballot = 1 follows):
 *   inner_staged  0: each lane reads its inner-level node block through L1
 *                 (every 128-byte line of the block prefetched first; lanes
 *                 that share a node share its lines);
 *                 1: each distinct inner node block is staged into shared
 *                 memory once with 16-byte cp.async, then searched there;
 *                 2 (default): 1 for partitioned batches (a warp meets one or
 *                 two nodes per level), 0 for unsorted ones (up to 32).
 *   rank_ballot   0 (default): each query finds its leaf rank by binary
 *                 search in the staged block; 1: the rank is the population
 *                 count of a warp ballot, lane j comparing slot j (and j+32)
 *                 of the query's leaf, one query after another.
 * Results are identical; speed differs.  BT_ERR_ARG on inner_staged above 2
 * or rank_ballot above 1. */
bt_status bt_tree_set_descent(bt_tree *tree, uint32_t inner_staged, uint32_t rank_ballot);

/* An L2 access-policy window for the tree's searches: the inner levels below
 * the shared-memory-pinned ones (at most max_bytes, and at most the device's
 * window size) are marked persisting in L2 on every descent launch, so that
 * the stream of leaf blocks does not evict them between batches.  Sets this
 * process's persisting-L2 set-aside (cudaLimitPersistingL2CacheSize) to at
 * least the window's size if it is smaller; the set-aside belongs to this
 * process's CUDA context and ends with it.  0 removes the window.  No
 * counterpart in the paper (its top levels stay on chip, Sec. IV-A).
 * Errors: BT_ERR_ARG, BT_ERR_CUDA. */
bt_status bt_tree_set_l2_window(bt_tree *tree, uint64_t max_bytes);

/* Batches in flight side by side: at most descent_blocks_per_sm resident
 * blocks of the tree's descent and partition_blocks_per_sm of its partition
 * on every SM (0: as many as fit, the default).  With the partition at one
 * block per SM (descent_blocks_per_sm 0, partition_blocks_per_sm 1 with the
 * default launch settings), a caller that alternates two streams -- each
 * with its own workspace and outputs -- gets batch i+1's partition running
 * beside batch i's descent: the paper's pipelining of successive batches
 * (Sec. V-B, Fig. 7), here on the device.  Results do not change; a single
 * stream runs slower with the caps.  The partition stays one cooperative
 * launch (all of its blocks resident before any passes a grid barrier).
 * Not thread-safe with searches running on the tree.  No counterpart in
 * the paper's kernel.  BT_ERR_ARG above 32. */
bt_status bt_tree_set_corun(bt_tree *tree, uint32_t descent_blocks_per_sm, uint32_t partition_blocks_per_sm);

/* Test hook: poll limit of the first bounded wait of the descents' bulk-copy
 * staging, BT_DEFAULT_WAIT_POLLS unless changed; 0 makes every such wait
 * give up at once.  After a wait gives up, the warp counts it
 * (bt_check_timeouts then returns BT_ERR_TIMEOUT), waits once more with the
 * default limit so that its copies land, and stops: the outputs of that
 * search are invalid.  Process-wide; takes effect for launches made after
 * the call.  No counterpart in the paper. */
#define BT_DEFAULT_WAIT_POLLS (1u << 22)
void bt_debug_set_wait_polls(uint32_t polls);

/* Queries each lane carries through the plain descent: 1 (a warp walks 32
 * consecutive queries of the batch down the tree together, the default) or
 * 2 (64 per warp: the per-level warp work -- finding the distinct nodes,
 * staging them -- is shared by twice as many queries; cp.async staging).
 * Results are identical; speed differs.  Not used by the learned descent.
 * BT_ERR_ARG on other values. */
bt_status bt_tree_set_lane_queries(bt_tree *tree, uint32_t per_lane);

/* BT_ERR_TIMEOUT if a bounded device wait of a search gave up since the
 * last call (the results of such a search are invalid), else BT_OK; clears
 * the counters.  Synchronous (reads device counters).  No counterpart in the
 * paper (its kernel has no waits that can fail). */
bt_status bt_check_timeouts(void);

/*
 * bt_autotune -- build the tree at every fanout in {8, 16, 32, 64} and time
 * a sample batch (d_sample, nsample device queries) through bt_search_batch
 * for every combination of warps per block {4, 8, 16}, pinned bytes
 * {0, 16384, 49152} and descent design (pipelined with inner levels read
 * through L1 or staged; synchronous with cp.async or bulk-copy staging; two
 * queries per lane); keep the fastest.  *out receives the tree built with
 * the best fanout and launch parameters applied, *best the choice and its
 * time.  A sample with fewer 32-query chunks per SM than a warps-per-block
 * setting runs the pipelined descent in smaller blocks whatever that setting
 * is (see bt_tree_set_launch), so such settings are not tried for it and the
 * pipelined designs keep 8 warps per block: tune on a batch of the size the
 * tree will serve.  Synchronizes `stream`.  Errors: as bt_build, plus
 * BT_ERR_ARG.
 * No counterpart in the paper (its fanout is fixed by the key size).
 */
bt_status bt_autotune(const void *h_keys, const void *h_vals, uint64_t n, bt_width key_w, bt_width val_w,
                      const void *d_sample, uint64_t nsample, bt_stream stream, bt_tree **out, bt_tune *best);

/* ------------------------------------------------------------------------
 * Range-partitioned trees.  The paper runs several kernel instances on one
 * batch (Sec. IV-G), each holding the whole tree; split by key range instead,
 * each holds one part: P subtrees over contiguous key ranges, every query
 * routed to the part whose range holds it and every result routed back to
 * its input position.  Across GPUs each part lives on its own GPU and the
 * routing is an exchange of queries and one of results
 * (paper_2604_21117_gb300/range_split.py holds that host-side exchange); on
 * one GPU, bt_range_search does both routings itself.
 * ------------------------------------------------------------------------ */
typedef struct bt_range bt_range;

/*
 * bt_range_build -- P = `parts` subtrees (1..64) over n sorted keys
 * (integer keys only): part p holds the keys of rank floor(p n / P) ..
 * floor((p+1) n / P) - 1 with their values, built with bt_build at `fanout`;
 * splitter p (p < P - 1) is the largest key of part p.  n must be >= P.
 * Synchronizes `stream`.  Errors: as bt_build, BT_ERR_ARG for P or n out of
 * range or 32-byte keys.
 */
bt_status bt_range_build(const void *h_keys, const void *h_vals, uint64_t n, bt_width key_w, bt_width val_w,
                         uint32_t fanout, uint32_t parts, bt_stream stream, bt_range **out);
void bt_range_free(bt_range *range);

/* The number of parts; optionally (non-NULL) the P - 1 splitters (as
 * uint64) and the number of keys of every part.  BT_ERR_ARG on nulls. */
bt_status bt_range_info(const bt_range *range, uint32_t *parts, uint64_t *h_splitters, uint64_t *h_part_keys);

/* Part p's tree (owned by the range; NULL if p is out of range). */
const bt_tree *bt_range_part(const bt_range *range, uint32_t p);

/* Device workspace of bt_range_search for nq queries. */
uint64_t bt_range_workspace_bytes(const bt_range *range, uint64_t nq);

/*
 * bt_range_search -- point lookups over the range-partitioned key set,
 * results in input order (as bt_search_batch over all the keys).  Every query
 * goes to the first part whose splitter is >= the query (the last part when
 * none is); each part's queries are searched with bt_search_batch on that
 * part's tree; results return to their input positions.  Reads the part
 * sizes back to the host once (it synchronizes `stream`).  Not thread-safe
 * for one range (the part sizes are staged in the range).
 * Errors: as bt_search_batch.
 */
bt_status bt_range_search(const bt_range *range, const void *d_queries, uint64_t nq, void *d_out_vals,
                          uint8_t *d_out_found, void *d_workspace, uint64_t ws_bytes, bt_stream stream);

/* ------------------------------------------------------------------------
 * The paper's node layout (Sec. IV-B, Eq. 1, Fig. 3), for comparison with
 * the structure-of-arrays layout above.  The same tree as one array of
 * equal-size nodes in BFS order (root first, then level by level, left to
 * right).  A node is:
 *   a 32-byte header: uint32 slotUse (keys in a leaf, separators in an
 *     inner node), uint32 depth (level, root = 0), 24 zero bytes;
 *   k_max = m - 1 key slots in the device key form (unused slots all-ones),
 *     padded to a multiple of 8 bytes;
 *   inner nodes: m 8-byte child addresses, byte offsets from the start of
 *     the array (slots beyond slotUse + 1 are zero);
 *   leaves: k_max 8-byte data slots (the value, zero-extended) and 8 unused
 *     bytes;
 *   rounded up to whole 32-byte chunks (the paper's memory access unit).
 * For 32-byte keys this is Eq. 1's N_size = 32 + 32 k_max + 32 (k_max+1)/4
 * = 40 m bytes.
 * ------------------------------------------------------------------------ */

/* Node size of the paper layout for fanout m and key width (0 if either is
 * unsupported).  Pure function, no device. */
uint32_t bt_paper_node_bytes(uint32_t fanout, bt_width key_w);

/* Build the paper layout of `tree` in a second device allocation (freed by
 * bt_free); copies the tree image to the host and back, synchronizes
 * `stream`.  A no-op if already built or if the tree is empty.
 * Errors: BT_ERR_ARG, BT_ERR_NOMEM, BT_ERR_CUDA. */
bt_status bt_paper_layout_build(bt_tree *tree, bt_stream stream);

/* bt_search_batch over the paper layout: the same partition, then the
 * level-wise descent over whole staged nodes, following child addresses
 * (results identical to bt_search_batch).  BT_ERR_ARG if the layout has not
 * been built.  Other errors as bt_search_batch. */
bt_status bt_paper_search_batch(const bt_tree *tree, const void *d_queries, uint64_t nq, void *d_out_vals,
                                uint8_t *d_out_found, void *d_workspace, uint64_t ws_bytes, bt_stream stream);

/* bt_descend_sorted over the paper layout. */
bt_status bt_paper_descend_sorted(const bt_tree *tree, const void *d_queries, const uint32_t *d_index, uint64_t nq,
                                  void *d_out_vals, uint8_t *d_out_found, bt_stream stream);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of small lookup requests.  The paper times a
 * host that writes a batch, runs the kernel and reads the results, and
 * notes that a pipelined host overlaps its transfers with the kernel
 * (Sec. V-B, Fig. 7).  A server keeps trees resident and serves requests
 * from many callers.  A submission copies the request's keys into its
 * tree's ring of lookups in page-locked, device-mapped host memory.  A
 * worker thread forms a batch when the oldest waiting request has waited
 * deadline_us or max_batch lookups are waiting: it takes waiting requests of
 * every tree (oldest tree first) and runs them as one multi-tree launch
 * (bt_forest_search's kernel, each tree with its own launch settings and
 * model) on a free slot (its own stream); the kernel reads the keys from the
 * rings, writes the results back into them and raises the slot's flag in
 * host memory -- one API call per batch, no copies.  Up to `slots` batches
 * are in flight at once, so their work overlaps on the device while new
 * requests are admitted into later batches as slots free up; batches retire
 * in issue order, their results copied into the requests' buffers.  A
 * batch is issued only while the bytes (keys, values, flags) of all batches
 * in flight stay within mem_cap_bytes; submissions beyond pending_cap_bytes
 * of waiting requests, or beyond a tree's ring (max_batch * (slots + 2)
 * lookups, at least 2 * max_batch, at most 2^22 unless 2 * max_batch is
 * more), are refused with BT_ERR_NOMEM (back-pressure).
 * ------------------------------------------------------------------------ */
typedef struct bt_server bt_server;

typedef struct bt_server_opts {
    uint32_t slots;             /* batches in flight at once, 1..64 */
    uint32_t max_batch;         /* queries per batch, 1..2^24 (also the largest request) */
    double deadline_us;         /* longest a request waits to be batched */
    uint64_t mem_cap_bytes;     /* bytes (keys, values, flags) of batches in flight (0 = unlimited) */
    uint64_t pending_cap_bytes; /* bytes of waiting requests before refusal (0 = unlimited) */
} bt_server_opts;

typedef struct bt_server_stats {
    uint64_t submitted, completed, lookups, batches;
    uint32_t max_inflight;      /* most batches seen in flight at once */
    float p50_us, p99_us, max_us; /* request latency, submission to results in place */
} bt_server_stats;

/* Start a server over `ntrees` resident trees (equal integer key and value
 * widths; BT_ERR_ARG for 32-byte keys).  models: NULL, or one entry per
 * tree, NULL or a model trained on that tree (its lookups then take the
 * learned path of bt_forest_create_learned; a model for an empty tree is
 * BT_ERR_ARG).  Trees and models must outlive the server.  Allocates the
 * rings and slots and starts the worker on the current device.
 * Errors: BT_ERR_ARG, BT_ERR_NOMEM, BT_ERR_CUDA. */
bt_status bt_server_create(const bt_tree *const *trees, const bt_model *const *models, uint32_t ntrees,
                           const bt_server_opts *opts, bt_server **out);

/* Queue one request of `count` keys (host memory, copied before the call
 * returns) for tree number `tree`; the results are written to h_out_vals /
 * h_out_found (host) before the request's ticket is reported done.  Buffers
 * must stay valid until then.  Thread-safe.  BT_ERR_NOMEM: the pending cap
 * or the tree's ring is full now (retry later); BT_ERR_ARG: count is 0 or
 * above max_batch, or the request alone exceeds pending_cap_bytes.  If a batch cannot be issued
 * (a failing CUDA call), its requests are never reported done and every
 * later call returns the error. */
bt_status bt_server_submit(bt_server *server, uint32_t tree, const void *h_keys, uint32_t count,
                           void *h_out_vals, uint8_t *h_out_found, uint64_t *ticket);

/* Up to `max` tickets completed since the last poll. */
bt_status bt_server_poll(bt_server *server, uint64_t *tickets, uint32_t max, uint32_t *n);

/* Wait until every submitted request is complete (BT_ERR_TIMEOUT after timeout_s). */
bt_status bt_server_drain(bt_server *server, double timeout_s);

/* Counters and latency percentiles since creation or the last reset. */
bt_status bt_server_get_stats(bt_server *server, bt_server_stats *out, int reset);

/* Finish all accepted requests, stop the worker, free the slots. */
void bt_server_destroy(bt_server *server);

/* Load replay for measurements: submit request i at t_arrival_s[i] seconds
 * after the call starts (tree[i], count[i] keys at h_keys[key_offset[i]..],
 * results at the same offsets of h_out_vals / h_out_found), then drain.
 * *wall_s receives the elapsed time. */
bt_status bt_server_run_trace(bt_server *server, uint64_t n, const double *t_arrival_s, const uint32_t *tree,
                              const uint32_t *count, const uint64_t *key_offset, const void *h_keys,
                              void *h_out_vals, uint8_t *h_out_found, double *wall_s);

/* ------------------------------------------------------------------------
 * Learned leaf predictor.  Not in the paper: an extension in which a small
 * fp32 model, fitted or trained on the GPU on the tree's own (stored key,
 * leaf index) pairs, predicts a key's leaf directly so the search can skip
 * the inner levels.  The model's maximum error over the stored keys, kept
 * per range of predicted leaf (BT_ERR_RANGES ranges; the same device code
 * computes it), bounds a window of leaves around each prediction; the
 * window's boundaries are checked with exact integer
 * compares against the leaves' largest keys, and a warp any of whose queries
 * is not proven to lie in its window takes the plain level-wise descent.
 * Results are therefore always exactly those of bt_search_batch.
 *
 * Models (fp32 steps as listed; the CPU oracle reproduces the PL ones
 * bit for bit):
 *   BT_MODEL_PL  S segments split at key quantiles b_s = key of rank
 *                floor(s*n/S); x = fp32(fp64(q - b_s)) * inv_w_s with
 *                inv_w_s = fp32(1/fp64(b_{s+1} - b_s)) (the last width runs
 *                one past the largest key); a least-squares line per segment
 *                fitted in fp64 and stored in fp32; pred = fp32(fp32(slope_s *
 *                x) + icpt_s), separately rounded.
 *   BT_MODEL_MLP 1 -> 32 -> 32 -> 1 with ReLU on a rank coordinate (two
 *                stages): the first stage is 64 breakpoints b_s at key
 *                quantiles with inv_w_s as for PL; x = fp32(fp32(s) +
 *                min(fp32(fp64(q - b_s)) * inv_w_s, 1)) * (1/64), which follows
 *                the key's rank whatever the key distribution; trained with
 *                Adam on the mean squared error against leaf / (L - 1); pred =
 *                output * (L - 1).  Parameters (BT_MLP_PARAMS floats): W1[32],
 *                b1[32], W2[32][32] (row = output unit), b2[32], w3[32], b3.
 *   leaf_hat = rint(clamp(pred, 0, L - 1)).
 * ------------------------------------------------------------------------ */
#define BT_MLP_PARAMS 1153
typedef enum bt_model_kind { BT_MODEL_PL = 1, BT_MODEL_MLP = 2 } bt_model_kind;

typedef struct bt_learn_opts {
    int32_t kind;          /* BT_MODEL_PL or BT_MODEL_MLP */
    uint32_t segments;     /* PL: S, 1..65536 (capped at n) */
    const float *h_init;   /* MLP: BT_MLP_PARAMS initial parameters (host, read only) */
    uint32_t steps;        /* MLP: Adam steps (>= 1) */
    uint32_t batch;        /* MLP: samples per step, 1..2^22, ranks drawn by splitmix64 */
    float lr;              /* MLP: Adam learning rate (> 0) */
    uint64_t seed;         /* MLP: sampling seed */
} bt_learn_opts;

typedef struct bt_model_info {
    int32_t kind;
    uint32_t segments;     /* PL: S actually used */
    uint32_t leaves;       /* L of the tree it was trained on */
    uint32_t max_err;      /* max |leaf_hat - leaf| over every stored key */
    float final_loss;      /* MLP: mean squared error of the last training step */
    uint64_t device_bytes; /* device memory held by the model */
} bt_model_info;

/* Fit (PL) or train (MLP) a model for `tree` on the GPU and compute its
 * error bound; synchronizes `stream`.  The model is only valid with this tree.
 * Integer keys only.
 * Errors: BT_ERR_ARG (empty tree, 32-byte keys, bad options), BT_ERR_NOMEM, BT_ERR_CUDA. */
bt_status bt_model_train(const bt_tree *tree, const bt_learn_opts *opts, bt_stream stream, bt_model **out);
void bt_model_free(bt_model *model);
bt_status bt_model_get_info(const bt_model *model, bt_model_info *out);
/* Copy the parameters to host memory (synchronous).  PL: b[S] (uint64),
 * inv_w[S], slope[S], icpt[S] (float), 20*S bytes; MLP: BT_MLP_PARAMS
 * floats.  BT_ERR_ARG if `bytes` is too small. */
bt_status bt_model_copy_params(const bt_model *model, void *h_dst, uint64_t bytes);

/* The error bound per range of prediction: entry r is the largest
 * |leaf_hat - leaf| over the stored keys whose leaf_hat lies in
 * [r*L/BT_ERR_RANGES, (r+1)*L/BT_ERR_RANGES); the search uses the bound of
 * each query's own range.  h_dst needs n >= BT_ERR_RANGES entries. */
#define BT_ERR_RANGES 256
bt_status bt_model_copy_err_bounds(const bt_model *model, uint32_t *h_dst, uint32_t n);

/* Mean-squared-error gradient of an MLP over n given samples, the training
 * kernel's own forward and backward pass: writes d_grad[BT_MLP_PARAMS] and
 * d_loss[0] = mean((f(x_i) - t_i)^2).  d_params, d_x, d_t, d_grad, d_loss are
 * device float arrays.  Asynchronous on `stream`. */
bt_status bt_mlp_grad(const float *d_params, const float *d_x, const float *d_t, uint32_t n,
                      float *d_grad, float *d_loss, bt_stream stream);

/* bt_descend_sorted with the model: same arguments and results, plus
 * d_stats (NULL or 2 device counters): warps that the model window served,
 * warps that fell back to the plain descent. */
bt_status bt_learned_descend_sorted(const bt_tree *tree, const bt_model *model, const void *d_queries,
                                    const uint32_t *d_index, uint64_t nq, void *d_out_vals,
                                    uint8_t *d_out_found, unsigned long long *d_stats, bt_stream stream);

/* bt_search_batch with the model (sort, then the learned descent); same
 * workspace, results identical to bt_search_batch. */
bt_status bt_learned_search_batch(const bt_tree *tree, const bt_model *model, const void *d_queries,
                                  uint64_t nq, void *d_out_vals, uint8_t *d_out_found, void *d_workspace,
                                  uint64_t ws_bytes, bt_stream stream);

/* Static text for a status code (never NULL; "unknown status" for values
 * outside bt_status).  No counterpart in the paper. */
const char *bt_status_str(bt_status status);

/* Thread-local detail of the last BT_ERR_CUDA on this thread ("" if none).
 * No counterpart in the paper. */
const char *bt_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* BTREE_GB300_H */
