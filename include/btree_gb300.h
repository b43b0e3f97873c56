/*
 * btree_gb300.h -- C ABI of the GB300 (sm_103a) batched B+ tree search library.
 *
 * The library answers batches of point queries against a static B+ tree by
 * the level-wise batch traversal of Tzschoppe et al., "Efficient Batch Search
 * Algorithm for B+ Tree Index Structures with Level-Wise Traversal on FPGAs":
 * the batch is sorted (Sec. IV-A), then descends the tree one level at a time;
 * every node needed at a level is fetched once per group of queries routed to
 * it and compared against all of them (Sec. IV-A, Sec. IV-F); a query goes to
 * the first slot whose separator it is less than or equal to (Sec. IV-E); at
 * the leaf an equal key yields its data, otherwise -1 (Sec. IV-D).
 *
 * Conventions for every call:
 *   - Keys and values are unsigned integers of 4 or 8 bytes, compared as
 *     unsigned integers (the paper's 32-byte keys compared byte by byte,
 *     Sec. IV-E, are replaced by native integer compares).
 *   - "d_" pointers are device (GPU global memory) pointers owned by the
 *     caller; "h_" pointers are host pointers owned by the caller.  Nothing the
 *     caller passes is freed or retained after a call returns, except that a
 *     search reads and writes its device buffers asynchronously on `stream`
 *     until the stream reaches that point.
 *   - `stream` is a CUDA runtime stream (cudaStream_t); NULL is the legacy
 *     default stream.  The header declares it as `struct CUstream_st *`, which
 *     is what cudaStream_t is, so that it needs no CUDA header.
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

/* Width of keys and values in bytes. */
typedef enum bt_width { BT_U32 = 4, BT_U64 = 8 } bt_width;

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

/* Shape of a built tree.  Level 0 is the root, level height-1 the leaves. */
typedef struct bt_info {
    uint32_t height;                       /* number of levels; 0 for an empty tree */
    uint32_t fanout;                       /* m: max children of an inner node */
    uint32_t key_bytes;                    /* 4 or 8 */
    uint32_t val_bytes;                    /* 4 or 8 */
    uint64_t n;                            /* keys stored */
    uint64_t level_nodes[BT_MAX_LEVELS];   /* nodes per level */
    uint64_t level_key_offset[BT_MAX_LEVELS]; /* byte offset of the level's key blocks */
    uint64_t leaf_val_offset;              /* byte offset of the leaf value blocks */
    uint64_t device_bytes;                 /* size of the device image */
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
 *   key_w, val_w   BT_U32 or BT_U64.
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
 * leaf's key count, so the all-ones key itself is legal.
 *
 * Errors: BT_ERR_ARG, BT_ERR_FANOUT, BT_ERR_UNSORTED, BT_ERR_DUPLICATE,
 * BT_ERR_NOMEM, BT_ERR_CUDA.  *out is set only on BT_OK.
 */
bt_status bt_build(const void *h_keys, const void *h_vals, uint64_t n, bt_width key_w,
                   bt_width val_w, uint32_t fanout, bt_stream stream, bt_tree **out);

/* Release a tree and its device memory (NULL is a no-op).  The caller must
 * make sure no search using it is still running. */
void bt_free(bt_tree *tree);

/* Copy the tree's shape into *out.  BT_ERR_ARG on null pointers. */
bt_status bt_tree_info(const bt_tree *tree, bt_info *out);

/* Copy the first `bytes` of the device image into host memory (for layout
 * checks); synchronous.  BT_ERR_ARG if bytes exceeds the image. */
bt_status bt_tree_copy_image(const bt_tree *tree, void *h_dst, uint64_t bytes);

/* Bytes of device workspace bt_search_batch needs for a batch of nq queries
 * (sort buffers and radix histograms).  Depends only on the tree's key width
 * and nq. */
uint64_t bt_search_workspace_bytes(const bt_tree *tree, uint64_t nq);

/* Options for bt_search_batch_ex. */
typedef struct bt_search_opts {
    /* How many leading bits of the normalised query key the batch is
     * radix-sorted on before the descent (Sec. IV-A sorts the batch so that
     * queries for one node are adjacent): -1 lets the library choose from nq
     * and the tree, 0 skips the sort, 1..64 forces that many bits (rounded up
     * to whole 8-bit radix passes, capped at the key width). */
    int32_t sort_bits;
    /* If non-NULL: device array of `height` counters to which the search
     * adds, per level, how many node key blocks it fetched -- the quantity
     * the paper's method keeps near the number of distinct nodes (Sec. IV-A).
     * Counting adds one atomic per warp and level. */
    unsigned long long *d_fetch_counts;
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
 * bt_sort_batch -- the first step of a search on its own: the on-device LSD
 * radix sort of the batch (Sec. IV-A: queries are sorted so that those
 * routed to one node are adjacent).  Writes the reordered queries and, for
 * each, its input position.  The sort key is the query's offset above the
 * tree's smallest key, clamped to the tree's key range (a monotone map, so
 * the order agrees with the key order); `sort_bits` leading bits of it are
 * used, rounded up to whole 8-bit passes (-1 = library choice, 0 = no
 * reordering: the queries are copied and the index is the identity).  The
 * sort is stable, so equal sort keys keep their input order.
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

/* Status of the last sort that ran in this workspace (bt_search_batch,
 * bt_search_batch_ex or bt_sort_batch with the same tree and nq): BT_OK, or
 * BT_ERR_TIMEOUT if a bounded wait of the sort's look-back gave up (the
 * results of that search are then invalid).  Synchronous: reads one word of
 * the workspace after the device has finished all work.  A search that did
 * not sort leaves the word as the previous sort left it. */
bt_status bt_workspace_status(const bt_tree *tree, const void *d_workspace, uint64_t nq);

/* Number of 8-bit radix passes bt_sort_batch / bt_search_batch would run
 * for this tree, batch size and sort_bits (0 = no sort).  -1 on a NULL tree. */
int32_t bt_sort_passes(const bt_tree *tree, uint64_t nq, int32_t sort_bits);

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
 * Scratch space (sort buffers, histograms, look-back words) is a 2 MiB
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
 * Errors: as bt_search_batch, plus BT_ERR_ARG for nq > BT_NOALLOC_MAX_QUERIES.
 */
#define BT_NOALLOC_MAX_QUERIES 65536
bt_status bt_search_batch_noalloc(const bt_tree *tree, const void *d_queries, uint64_t nq,
                                  void *d_out_vals, uint8_t *d_out_found, bt_stream stream);

/* Static text for a status code. */
const char *bt_status_str(bt_status status);

/* Thread-local detail of the last BT_ERR_CUDA on this thread ("" if none). */
const char *bt_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* BTREE_GB300_H */
