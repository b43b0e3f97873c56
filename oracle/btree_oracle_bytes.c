/*
 * CPU oracle for batched B+ tree point search on fixed-width BYTE-STRING
 * keys (the paper's 32-byte keys).  TEST INFRASTRUCTURE ONLY: the GPU
 * library never links, loads or calls this file; only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark use it.
 *
 * The tree is the same even bulk load as the integer-key oracle
 * (btree_oracle.c; Sec. III for the node capacities, Sec. IV-E for the
 * routing, Sec. IV-D for the result), restated for keys that are strings of
 * kb bytes.  Two keys compare as the paper's comparison module does
 * (Sec. IV-E): one comparator per byte position reports less, equal or
 * greater, and the first position (lowest address) that is not equal
 * decides -- plain lexicographic byte order, which is what memcmp computes.
 * A query is routed to the first separator it is less than or equal to; at
 * the leaf an equal key is a match, whose 8-byte data (or 4-byte, by
 * val_bits) is returned, else all-ones with found = 0.
 *
 * Queries are answered one at a time from the root, with no batching and no
 * sorting.
 *
 * Planted mistake (compile-time, off by default), for the pin tests:
 *   BTB_PLANT_LAST_BYTE_FIRST  compare from the last byte to the first
 *                              (a little-endian reading of the key)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define BTB_MAX_LEVELS 64

typedef struct btb_node {
    int is_leaf;
    uint64_t index;            /* left-to-right position within its level */
    int nkeys;                 /* leaf: keys held; inner: separators */
    unsigned char *keys;       /* nkeys * kb bytes */
    uint64_t *vals;            /* leaf only */
    struct btb_node **child;   /* inner only, nkeys + 1 entries */
    const unsigned char *subtree_max;  /* largest key below this node */
} btb_node;

typedef struct btb_tree {
    int m;
    int kb;
    int val_bits;
    uint64_t n;
    int height;
    uint64_t level_nodes[BTB_MAX_LEVELS];     /* index 0 = root level */
    btb_node **level[BTB_MAX_LEVELS];
    uint64_t miss;
} btb_tree;

/* <0, 0, >0 as a is less than, equal to or greater than b (Sec. IV-E). */
static int key_cmp(const unsigned char *a, const unsigned char *b, int kb)
{
#ifdef BTB_PLANT_LAST_BYTE_FIRST
    for (int i = kb - 1; i >= 0; --i)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
#else
    return memcmp(a, b, (size_t)kb);
#endif
}

static uint64_t even_part(uint64_t total, uint64_t parts, uint64_t i)
{
    return total / parts + (i < total % parts ? 1u : 0u);
}

static btb_node *new_node(int is_leaf, int nkeys, int kb)
{
    btb_node *x = (btb_node *)calloc(1, sizeof(btb_node));
    if (!x) return NULL;
    x->is_leaf = is_leaf;
    x->nkeys = nkeys;
    x->keys = (unsigned char *)calloc((size_t)(nkeys > 0 ? nkeys : 1), (size_t)kb);
    if (is_leaf)
        x->vals = (uint64_t *)calloc((size_t)(nkeys > 0 ? nkeys : 1), sizeof(uint64_t));
    else
        x->child = (btb_node **)calloc((size_t)nkeys + 1, sizeof(btb_node *));
    return x;
}

void btb_free(btb_tree *t)
{
    if (!t) return;
    for (int l = 0; l < t->height; ++l) {
        for (uint64_t i = 0; i < t->level_nodes[l]; ++i) {
            btb_node *x = t->level[l][i];
            free(x->keys);
            free(x->vals);
            free(x->child);
            free(x);
        }
        free(t->level[l]);
    }
    free(t);
}

/* Bulk load from n strictly increasing keys (n * kb bytes, key i at
 * keys + i * kb) with their values.  NULL on bad arguments. */
btb_tree *btb_build(const unsigned char *keys, const uint64_t *vals, uint64_t n, int kb, int m, int val_bits)
{
    if (m < 3 || kb < 1 || kb > 256 || (val_bits != 32 && val_bits != 64)) return NULL;
    btb_tree *t = (btb_tree *)calloc(1, sizeof(btb_tree));
    if (!t) return NULL;
    t->m = m;
    t->kb = kb;
    t->val_bits = val_bits;
    t->n = n;
    t->miss = (val_bits == 64) ? ~(uint64_t)0 : (uint64_t)0xFFFFFFFFu;
    if (n == 0) return t;

    const uint64_t kmax = (uint64_t)(m - 1);
    btb_node **tmp[BTB_MAX_LEVELS];
    uint64_t tmp_count[BTB_MAX_LEVELS];
    int nlev = 0;

    uint64_t L = (n + kmax - 1) / kmax;
    btb_node **leaves = (btb_node **)calloc((size_t)L, sizeof(btb_node *));
    uint64_t off = 0;
    for (uint64_t i = 0; i < L; ++i) {
        uint64_t s = even_part(n, L, i);
        btb_node *x = new_node(1, (int)s, kb);
        memcpy(x->keys, keys + off * (uint64_t)kb, (size_t)(s * (uint64_t)kb));
        for (uint64_t j = 0; j < s; ++j) x->vals[j] = vals[off + j];
        x->subtree_max = x->keys + (s - 1) * (uint64_t)kb;
        off += s;
        leaves[i] = x;
    }
    tmp[nlev] = leaves;
    tmp_count[nlev] = L;
    nlev++;

    uint64_t C = L;
    btb_node **below = leaves;
    while (C > 1) {
        uint64_t P = (C + (uint64_t)m - 1) / (uint64_t)m;
        btb_node **par = (btb_node **)calloc((size_t)P, sizeof(btb_node *));
        uint64_t c0 = 0;
        for (uint64_t j = 0; j < P; ++j) {
            uint64_t nc = even_part(C, P, j);
            btb_node *x = new_node(0, (int)nc - 1, kb);
            for (uint64_t c = 0; c < nc; ++c) x->child[c] = below[c0 + c];
            for (uint64_t c = 0; c + 1 < nc; ++c)
                memcpy(x->keys + c * (uint64_t)kb, below[c0 + c]->subtree_max, (size_t)kb);
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
        for (uint64_t i = 0; i < t->level_nodes[l]; ++i) t->level[l][i]->index = i;
    }
    return t;
}

/* Root to leaf for one query; path[l] = node index visited at level l. */
static const btb_node *descend(const btb_tree *t, const unsigned char *q, uint64_t *path)
{
    const btb_node *x = t->level[0][0];
    int l = 0;
    while (!x->is_leaf) {
        if (path) path[l] = x->index;
        int i = 0;
        while (i < x->nkeys && key_cmp(q, x->keys + (uint64_t)i * t->kb, t->kb) > 0) i++;
        x = x->child[i];
        l++;
    }
    if (path) path[l] = x->index;
    return x;
}

static int leaf_slot(const btb_tree *t, const btb_node *x, const unsigned char *q)
{
    for (int j = 0; j < x->nkeys; ++j)
        if (key_cmp(x->keys + (uint64_t)j * t->kb, q, t->kb) == 0) return j;
    return -1;
}

/* One query at a time; query i at q + i * kb.  Outputs may be NULL. */
void btb_search(const btb_tree *t, const unsigned char *q, uint64_t nq, uint64_t *vals, uint8_t *found,
                uint64_t *leaf, int32_t *slot)
{
    for (uint64_t i = 0; i < nq; ++i) {
        const unsigned char *qi = q + i * (uint64_t)t->kb;
        if (t->height == 0) {
            if (vals) vals[i] = t->miss;
            if (found) found[i] = 0;
            if (leaf) leaf[i] = ~(uint64_t)0;
            if (slot) slot[i] = -1;
            continue;
        }
        const btb_node *x = descend(t, qi, NULL);
        int j = leaf_slot(t, x, qi);
        if (vals) vals[i] = (j >= 0) ? x->vals[j] : t->miss;
        if (found) found[i] = (j >= 0) ? 1 : 0;
        if (leaf) leaf[i] = x->index;
        if (slot) slot[i] = j;
    }
}

void btb_paths(const btb_tree *t, const unsigned char *q, uint64_t nq, uint64_t *path)
{
    if (t->height == 0) return;
    for (uint64_t i = 0; i < nq; ++i) descend(t, q + i * (uint64_t)t->kb, path + i * (uint64_t)t->height);
}

typedef struct {
    const btb_tree *t;
    const unsigned char *q;
    uint64_t nq;
    uint64_t *vals;
    uint8_t *found;
} btb_job;

static void *btb_worker(void *arg)
{
    btb_job *j = (btb_job *)arg;
    btb_search(j->t, j->q, j->nq, j->vals, j->found, NULL, NULL);
    return NULL;
}

/* The batch split evenly over nthreads threads (Sec. V-F's CPU runs). */
int btb_search_mt(const btb_tree *t, const unsigned char *q, uint64_t nq, uint64_t *vals, uint8_t *found,
                  int nthreads)
{
    if (nthreads <= 1) {
        btb_search(t, q, nq, vals, found, NULL, NULL);
        return 0;
    }
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    btb_job *jobs = (btb_job *)calloc((size_t)nthreads, sizeof(btb_job));
    if (!th || !jobs) { free(th); free(jobs); return -1; }
    uint64_t off = 0;
    int started = 0, rc = 0;
    for (int k = 0; k < nthreads; ++k) {
        uint64_t s = even_part(nq, (uint64_t)nthreads, (uint64_t)k);
        jobs[k].t = t;
        jobs[k].q = q + off * (uint64_t)t->kb;
        jobs[k].nq = s;
        jobs[k].vals = vals + off;
        jobs[k].found = found + off;
        off += s;
        if (pthread_create(&th[k], NULL, btb_worker, &jobs[k]) != 0) { rc = -1; break; }
        started++;
    }
    for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
    free(th);
    free(jobs);
    return rc;
}

int btb_height(const btb_tree *t) { return t->height; }

uint64_t btb_level_nodes(const btb_tree *t, int level)
{
    return (level >= 0 && level < t->height) ? t->level_nodes[level] : 0;
}

/* Copy node (level, index): returns its key count, or -1 if out of range.
 * keys needs m * kb bytes, vals m entries, child_index m entries. */
int btb_node_dump(const btb_tree *t, int level, uint64_t index, int *is_leaf, unsigned char *keys,
                  uint64_t *vals, uint64_t *child_index)
{
    if (level < 0 || level >= t->height || index >= t->level_nodes[level]) return -1;
    const btb_node *x = t->level[level][index];
    *is_leaf = x->is_leaf;
    memcpy(keys, x->keys, (size_t)x->nkeys * (size_t)t->kb);
    if (x->is_leaf && vals)
        for (int j = 0; j < x->nkeys; ++j) vals[j] = x->vals[j];
    if (!x->is_leaf && child_index)
        for (int c = 0; c <= x->nkeys; ++c) child_index[c] = x->child[c]->index;
    return x->nkeys;
}
