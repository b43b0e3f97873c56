/*
 * CPU oracle for batched B+ tree point search.  TEST INFRASTRUCTURE ONLY:
 * the GPU library never links, loads or calls this file; only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark use it.
 *
 * It is a plain, deliberately slow, pointer-based B+ tree written from the
 * paper's definitions (Tzschoppe et al., "Efficient Batch Search Algorithm
 * for B+ Tree Index Structures with Level-Wise Traversal on FPGAs"):
 *
 *   - Sec. III:  order m = maximum children of an inner node, k_max = m - 1
 *                keys per node, every non-root inner node at least half
 *                full, all data in the leaves, all leaves at one depth.
 *   - Sec. IV-E: a query is routed to the first slot whose key it is
 *                "less than or equal" to (priority encoder = lowest such
 *                slot); at the leaf an equal key is a match.
 *   - Sec. IV-D: the leaf result is the stored data, or -1 for a miss.
 *
 * The paper does not say how the tree was filled (its trees come from the
 * TLX library).  The reading used here, and by the GPU library's builder
 * independently, is an even bulk load:
 *   leaves  L = ceil(n / k_max), leaf i holds floor(n/L) keys plus one more
 *           if i < n mod L, in sorted order;
 *   parents P = ceil(C / m) over C child nodes, node j takes floor(C/P)
 *           children plus one more if j < C mod P, left to right;
 *   separator i of an inner node = the largest key in the subtree of its
 *           child i (Sec. IV-E's "<=" routing then finds the child whose
 *           range holds the query); the last child has no separator;
 *   stop when one node is left.  n <= k_max gives a root that is a leaf;
 *   n = 0 gives an empty tree in which every query misses.
 *
 * Keys and values are held as uint64_t; 32-bit keys and values are zero
 * extended, which preserves their order.  A miss returns all-ones of the
 * value width (the paper's -1) with found = 0.
 *
 * Queries are answered one at a time by walking from the root (no batching,
 * no sorting, no blocking): the obviously-correct statement of what the
 * level-wise batch method must return.
 *
 * Planted mistakes (compile-time, off by default) let the pin tests show
 * that each pin catches a plausible error:
 *   BTO_PLANT_ROUTE_LT     route on q < sep instead of q <= sep
 *   BTO_PLANT_SEP_MIN      separator = smallest key of the child
 *   BTO_PLANT_LAST_CHILD   fall through to the second-to-last child
 *   BTO_PLANT_LEAF_FLOOR   L = floor(n / k_max) leaves (over-full leaves)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define BTO_MAX_LEVELS 64

typedef struct bto_node {
    int is_leaf;
    int level;                 /* 0 = root */
    uint64_t index;            /* left-to-right position within its level */
    int nkeys;                 /* leaf: keys held; inner: separators (= children - 1) */
    uint64_t *keys;
    uint64_t *vals;            /* leaf only */
    struct bto_node **child;   /* inner only, nkeys + 1 entries */
    uint64_t subtree_max;      /* largest key below this node */
    uint64_t subtree_min;      /* smallest key below this node */
} bto_node;

typedef struct bto_tree {
    int m;
    int val_bits;
    uint64_t n;
    int height;                               /* number of levels */
    uint64_t level_nodes[BTO_MAX_LEVELS];     /* index 0 = root level */
    bto_node **level[BTO_MAX_LEVELS];
    uint64_t miss;
} bto_tree;

/* Size of part i when `total` items are split as evenly as possible into
 * `parts` consecutive parts, the larger parts first. */
static uint64_t even_part(uint64_t total, uint64_t parts, uint64_t i)
{
    return total / parts + (i < total % parts ? 1u : 0u);
}

static bto_node *new_node(int is_leaf, int nkeys)
{
    bto_node *x = (bto_node *)calloc(1, sizeof(bto_node));
    if (!x) return NULL;
    x->is_leaf = is_leaf;
    x->nkeys = nkeys;
    x->keys = (uint64_t *)calloc((size_t)(nkeys > 0 ? nkeys : 1), sizeof(uint64_t));
    if (is_leaf)
        x->vals = (uint64_t *)calloc((size_t)(nkeys > 0 ? nkeys : 1), sizeof(uint64_t));
    else
        x->child = (bto_node **)calloc((size_t)nkeys + 1, sizeof(bto_node *));
    return x;
}

void bto_free(bto_tree *t)
{
    if (!t) return;
    for (int l = 0; l < t->height; ++l) {
        for (uint64_t i = 0; i < t->level_nodes[l]; ++i) {
            bto_node *x = t->level[l][i];
            free(x->keys);
            free(x->vals);
            free(x->child);
            free(x);
        }
        free(t->level[l]);
    }
    free(t);
}

/* Bulk load from n strictly increasing keys with their values.
 * Returns NULL on bad arguments or allocation failure. */
bto_tree *bto_build(const uint64_t *keys, const uint64_t *vals, uint64_t n,
                    int m, int val_bits)
{
    if (m < 3 || (val_bits != 32 && val_bits != 64)) return NULL;
    bto_tree *t = (bto_tree *)calloc(1, sizeof(bto_tree));
    if (!t) return NULL;
    t->m = m;
    t->val_bits = val_bits;
    t->n = n;
    t->miss = (val_bits == 64) ? ~(uint64_t)0 : (uint64_t)0xFFFFFFFFu;
    if (n == 0) return t;

    const uint64_t kmax = (uint64_t)(m - 1);
    /* Levels are built bottom-up into `tmp`, then reversed. */
    bto_node **tmp[BTO_MAX_LEVELS];
    uint64_t tmp_count[BTO_MAX_LEVELS];
    int nlev = 0;

#ifdef BTO_PLANT_LEAF_FLOOR
    uint64_t L = n / kmax;
    if (L == 0) L = 1;
#else
    uint64_t L = (n + kmax - 1) / kmax;
#endif
    bto_node **leaves = (bto_node **)calloc((size_t)L, sizeof(bto_node *));
    uint64_t off = 0;
    for (uint64_t i = 0; i < L; ++i) {
        uint64_t s = even_part(n, L, i);
        bto_node *x = new_node(1, (int)s);
        for (uint64_t j = 0; j < s; ++j) {
            x->keys[j] = keys[off + j];
            x->vals[j] = vals[off + j];
        }
        x->subtree_min = keys[off];
        x->subtree_max = keys[off + s - 1];
        off += s;
        leaves[i] = x;
    }
    tmp[nlev] = leaves;
    tmp_count[nlev] = L;
    nlev++;

    uint64_t C = L;
    bto_node **below = leaves;
    while (C > 1) {
        uint64_t P = (C + (uint64_t)m - 1) / (uint64_t)m;
        bto_node **par = (bto_node **)calloc((size_t)P, sizeof(bto_node *));
        uint64_t c0 = 0;
        for (uint64_t j = 0; j < P; ++j) {
            uint64_t nc = even_part(C, P, j);
            bto_node *x = new_node(0, (int)nc - 1);
            for (uint64_t c = 0; c < nc; ++c) x->child[c] = below[c0 + c];
            for (uint64_t c = 0; c + 1 < nc; ++c) {
#ifdef BTO_PLANT_SEP_MIN
                x->keys[c] = below[c0 + c]->subtree_min;
#else
                x->keys[c] = below[c0 + c]->subtree_max;
#endif
            }
            x->subtree_min = below[c0]->subtree_min;
            x->subtree_max = below[c0 + nc - 1]->subtree_max;
            c0 += nc;
            par[j] = x;
        }
        tmp[nlev] = par;
        tmp_count[nlev] = P;
        nlev++;
        below = par;
        C = P;
    }

    t->height = nlev;
    for (int l = 0; l < nlev; ++l) {
        t->level[l] = tmp[nlev - 1 - l];
        t->level_nodes[l] = tmp_count[nlev - 1 - l];
        for (uint64_t i = 0; i < t->level_nodes[l]; ++i) {
            t->level[l][i]->level = l;
            t->level[l][i]->index = i;
        }
    }
    return t;
}

/* Walk one query from the root to its leaf (Sec. IV-E routing).
 * path[l] receives the index of the node visited at level l. */
static const bto_node *descend(const bto_tree *t, uint64_t q, uint64_t *path)
{
    const bto_node *x = t->level[0][0];
    int l = 0;
    while (!x->is_leaf) {
        if (path) path[l] = x->index;
        int i = 0;
#ifdef BTO_PLANT_ROUTE_LT
        while (i < x->nkeys && !(q < x->keys[i])) i++;
#else
        while (i < x->nkeys && !(q <= x->keys[i])) i++;
#endif
#ifdef BTO_PLANT_LAST_CHILD
        if (i == x->nkeys && i > 0) i--;
#endif
        x = x->child[i];
        l++;
    }
    if (path) path[l] = x->index;
    return x;
}

/* Leaf probe (Sec. IV-D): the slot holding q, or -1. */
static int leaf_slot(const bto_node *x, uint64_t q)
{
    for (int j = 0; j < x->nkeys; ++j)
        if (x->keys[j] == q) return j;
    return -1;
}

/* One query at a time.  Any of vals/found/leaf/slot may be NULL. */
void bto_search(const bto_tree *t, const uint64_t *q, uint64_t nq,
                uint64_t *vals, uint8_t *found, uint64_t *leaf, int32_t *slot)
{
    for (uint64_t i = 0; i < nq; ++i) {
        if (t->height == 0) {
            if (vals) vals[i] = t->miss;
            if (found) found[i] = 0;
            if (leaf) leaf[i] = ~(uint64_t)0;
            if (slot) slot[i] = -1;
            continue;
        }
        const bto_node *x = descend(t, q[i], NULL);
        int j = leaf_slot(x, q[i]);
        if (vals) vals[i] = (j >= 0) ? x->vals[j] : t->miss;
        if (found) found[i] = (j >= 0) ? 1 : 0;
        if (leaf) leaf[i] = x->index;
        if (slot) slot[i] = j;
    }
}

/* Root-to-leaf path of every query: path[i * height + l]. */
void bto_paths(const bto_tree *t, const uint64_t *q, uint64_t nq, uint64_t *path)
{
    if (t->height == 0) return;
    for (uint64_t i = 0; i < nq; ++i)
        descend(t, q[i], path + i * (uint64_t)t->height);
}

/* ---- multi-threaded baseline: the batch split evenly over T threads,
 *      as the paper's CPU comparison does (Sec. V-F). ---- */
typedef struct {
    const bto_tree *t;
    const uint64_t *q;
    uint64_t nq;
    uint64_t *vals;
    uint8_t *found;
} bto_job;

static void *bto_worker(void *arg)
{
    bto_job *j = (bto_job *)arg;
    bto_search(j->t, j->q, j->nq, j->vals, j->found, NULL, NULL);
    return NULL;
}

int bto_search_mt(const bto_tree *t, const uint64_t *q, uint64_t nq,
                  uint64_t *vals, uint8_t *found, int nthreads)
{
    if (nthreads <= 1) {
        bto_search(t, q, nq, vals, found, NULL, NULL);
        return 0;
    }
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    bto_job *jobs = (bto_job *)calloc((size_t)nthreads, sizeof(bto_job));
    if (!th || !jobs) { free(th); free(jobs); return -1; }
    uint64_t off = 0;
    int started = 0, rc = 0;
    for (int k = 0; k < nthreads; ++k) {
        uint64_t s = even_part(nq, (uint64_t)nthreads, (uint64_t)k);
        jobs[k].t = t;
        jobs[k].q = q + off;
        jobs[k].nq = s;
        jobs[k].vals = vals + off;
        jobs[k].found = found + off;
        off += s;
        if (pthread_create(&th[k], NULL, bto_worker, &jobs[k]) != 0) { rc = -1; break; }
        started++;
    }
    for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
    free(th);
    free(jobs);
    return rc;
}

/* ---- structure accessors for the invariant tests ---- */
int bto_height(const bto_tree *t) { return t->height; }

uint64_t bto_level_nodes(const bto_tree *t, int level)
{
    return (level >= 0 && level < t->height) ? t->level_nodes[level] : 0;
}

/* Copy node (level, index): returns the key count (separators for inner
 * nodes), or -1 if out of range.  keys/vals need room for m entries;
 * child_index (inner only) for m entries. */
int bto_node_dump(const bto_tree *t, int level, uint64_t index, int *is_leaf,
                  uint64_t *keys, uint64_t *vals, uint64_t *child_index)
{
    if (level < 0 || level >= t->height || index >= t->level_nodes[level]) return -1;
    const bto_node *x = t->level[level][index];
    *is_leaf = x->is_leaf;
    for (int j = 0; j < x->nkeys; ++j) {
        keys[j] = x->keys[j];
        if (x->is_leaf && vals) vals[j] = x->vals[j];
    }
    if (!x->is_leaf && child_index)
        for (int c = 0; c <= x->nkeys; ++c) child_index[c] = x->child[c]->index;
    return x->nkeys;
}

/* ---- distinct nodes touched per level by a batch, and the distinct
 *      32-byte value sectors read by its hits, for the algorithmic-byte
 *      count.  A hit in leaf i, slot j reads value bytes at
 *      (i * m + j) * val_bytes of a leaf-value array of m slots per leaf. ---- */
static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static uint64_t count_distinct(uint64_t *v, uint64_t n)
{
    if (n == 0) return 0;
    qsort(v, (size_t)n, sizeof(uint64_t), cmp_u64);
    uint64_t d = 1;
    for (uint64_t i = 1; i < n; ++i) d += (v[i] != v[i - 1]);
    return d;
}

int bto_touched(const bto_tree *t, const uint64_t *q, uint64_t nq,
                uint64_t *level_counts, uint64_t *value_sectors)
{
    *value_sectors = 0;
    if (t->height == 0 || nq == 0) {
        for (int l = 0; l < t->height; ++l) level_counts[l] = 0;
        return 0;
    }
    const int h = t->height;
    uint64_t *path = (uint64_t *)malloc((size_t)(nq * (uint64_t)h) * sizeof(uint64_t));
    uint64_t *col = (uint64_t *)malloc((size_t)nq * sizeof(uint64_t));
    if (!path || !col) { free(path); free(col); return -1; }
    bto_paths(t, q, nq, path);
    for (int l = 0; l < h; ++l) {
        for (uint64_t i = 0; i < nq; ++i) col[i] = path[i * (uint64_t)h + l];
        level_counts[l] = count_distinct(col, nq);
    }
    const uint64_t vbytes = (uint64_t)t->val_bits / 8u;
    uint64_t nh = 0;
    for (uint64_t i = 0; i < nq; ++i) {
        const bto_node *x = t->level[h - 1][path[i * (uint64_t)h + (h - 1)]];
        int j = leaf_slot(x, q[i]);
        if (j >= 0)
            col[nh++] = ((x->index * (uint64_t)t->m + (uint64_t)j) * vbytes) / 32u;
    }
    *value_sectors = count_distinct(col, nh);
    free(path);
    free(col);
    return 0;
}
