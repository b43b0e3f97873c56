"""Pins for the CPU oracle: checks against things other than the oracle itself.

Each check returns a list of failure messages (empty = pinned), so the same
checks serve the oracle tests and the planted-mistake tests.

* ``lookup_vs_lower_bound``: a point lookup has a plain definition -- the
  value of the equal key found by binary search (std::lower_bound, here
  numpy.searchsorted) over the sorted key array, else a miss (Sec. IV-D's -1).
* ``invariants``: the B+ tree shape rules of Sec. III (k_max = m - 1, inner
  nodes at least half full, all leaves at one depth, data only in leaves),
  sorted nodes, separators equal to the largest key of the child's subtree
  (the reading of Sec. IV-E's "<=" routing), children contiguous left to
  right, node count within N_max = sum_{i<h} m^i.
* ``leaf_index_vs_leaf_max``: a query's leaf is the first leaf whose largest
  key is >= the query (or the last leaf) -- binary search over the leaf
  maxima, independent of the inner levels.
"""
from __future__ import annotations

import numpy as np


def reference_lookup(sorted_keys, vals, queries, val_bits: int = 64):
    k = np.asarray(sorted_keys).astype(np.uint64)
    v = np.asarray(vals).astype(np.uint64)
    q = np.asarray(queries).astype(np.uint64)
    pos = np.searchsorted(k, q, side="left")
    inb = pos < k.size
    hit = np.zeros(q.size, bool)
    hit[inb] = k[pos[inb]] == q[inb]
    out = np.full(q.size, (1 << val_bits) - 1, np.uint64)
    out[hit] = v[pos[hit]]
    return out, hit.astype(np.uint8)


def lookup_vs_lower_bound(tree, keys, vals, queries, val_bits=64):
    exp_v, exp_f = reference_lookup(keys, vals, queries, val_bits)
    got_v, got_f, _, _ = tree.search(queries)
    errs = []
    bad = np.nonzero((got_v != exp_v) | (got_f != exp_f))[0]
    if bad.size:
        i = int(bad[0])
        errs.append(f"lookup mismatch at {bad.size} queries, first q={int(np.asarray(queries)[i])}: "
                    f"got ({int(got_v[i])},{int(got_f[i])}) want ({int(exp_v[i])},{int(exp_f[i])})")
    return errs


def dump_tree(tree):
    """levels[l] = list of (is_leaf, keys, vals, children) for every node."""
    out = []
    for l, cnt in enumerate(tree.level_nodes()):
        out.append([tree.node(l, i) for i in range(cnt)])
    return out


def invariants(tree, keys, vals):
    errs = []
    m = tree.m
    kmax = m - 1
    n = len(keys)
    h = tree.height
    if n == 0:
        if h != 0:
            errs.append("empty key set must give an empty tree")
        return errs
    lv = dump_tree(tree)
    if len(lv[0]) != 1:
        errs.append("root level must hold exactly one node")
    # all leaves on the last level, inner nodes everywhere else
    for l, nodes in enumerate(lv):
        for i, (is_leaf, ks, vs, ch) in enumerate(nodes):
            if is_leaf != (l == h - 1):
                errs.append(f"node ({l},{i}) leaf flag wrong for its depth")
    # leaves: sorted, fill bounds, concatenation = all keys in order with values
    leaves = lv[-1]
    cat_k = np.concatenate([np.asarray(x[1], np.uint64) for x in leaves])
    cat_v = np.concatenate([np.asarray(x[2], np.uint64) for x in leaves])
    if cat_k.size != n or not np.array_equal(cat_k, np.asarray(keys).astype(np.uint64)):
        errs.append("leaves do not hold exactly the keys, in order")
    elif not np.array_equal(cat_v, np.asarray(vals).astype(np.uint64)):
        errs.append("leaf values do not match their keys")
    lo_leaf = -(-kmax // 2)
    for i, (_, ks, _, _) in enumerate(leaves):
        if len(ks) > kmax:
            errs.append(f"leaf {i} holds {len(ks)} > k_max keys")
        if h > 1 and len(ks) < lo_leaf:
            errs.append(f"leaf {i} holds {len(ks)} < ceil(k_max/2) keys")
        kl = [int(x) for x in ks]
        if any(kl[j] >= kl[j + 1] for j in range(len(kl) - 1)):
            errs.append(f"leaf {i} keys not strictly increasing")
    # inner levels: separators, children, fill
    sub_max = [None] * h
    sub_max[h - 1] = [int(x[1][-1]) for x in leaves]
    for l in range(h - 2, -1, -1):
        maxes = []
        expect_next = 0
        for i, (_, ks, _, ch) in enumerate(lv[l]):
            ch = [int(c) for c in ch]
            nc = len(ch)
            if nc > m:
                errs.append(f"node ({l},{i}) has {nc} > m children")
            if l > 0 and nc < -(-m // 2):
                errs.append(f"node ({l},{i}) has {nc} < ceil(m/2) children")
            if l == 0 and h > 1 and nc < 2:
                errs.append("inner root needs at least 2 children")
            if ch != list(range(expect_next, expect_next + nc)):
                errs.append(f"node ({l},{i}) children not contiguous left to right")
            expect_next += nc
            if len(ks) != nc - 1:
                errs.append(f"node ({l},{i}) separator count != children - 1")
            for j, s in enumerate(ks):
                if j + 1 < nc and int(s) != sub_max[l + 1][ch[j]]:
                    errs.append(f"node ({l},{i}) separator {j} != max key of child subtree")
            if any(int(ks[j]) >= int(ks[j + 1]) for j in range(len(ks) - 1)):
                errs.append(f"node ({l},{i}) separators not increasing")
            maxes.append(sub_max[l + 1][ch[-1]])
        if expect_next != len(lv[l + 1]):
            errs.append(f"level {l} children do not cover level {l + 1}")
        sub_max[l] = maxes
    nmax = sum(m ** i for i in range(h))
    total = sum(len(x) for x in lv)
    if total > nmax:
        errs.append(f"{total} nodes > N_max = {nmax}")
    if n > (m ** (h - 1)) * kmax:
        errs.append(f"n = {n} exceeds m^(h-1) * k_max for h = {h}")
    return errs


def leaf_index_vs_leaf_max(tree, queries):
    errs = []
    if tree.height == 0:
        return errs
    lv_leaf = tree.height - 1
    leaf_max = np.array([int(tree.node(lv_leaf, i)[1][-1]) for i in range(tree.level_nodes()[-1])],
                        dtype=np.uint64)
    q = np.asarray(queries).astype(np.uint64)
    want = np.minimum(np.searchsorted(leaf_max, q, side="left"), leaf_max.size - 1)
    _, _, got, _ = tree.search(queries)
    bad = np.nonzero(got != want)[0]
    if bad.size:
        errs.append(f"leaf index mismatch at {bad.size} queries")
    return errs


def probe_queries(keys, width_bits, g, extra=64):
    """Every key, key +- 1, both ends of the key space and random values."""
    top = (1 << width_bits) - 1
    k = np.asarray(keys).astype(np.uint64)
    parts = [k]
    if k.size:
        parts.append(k[k < np.uint64(top)] + np.uint64(1))
        parts.append(k[k > 0] - np.uint64(1))
    parts.append(np.array([0, 1, top - 1, top], np.uint64))
    parts.append(g.integers(0, 2**width_bits, size=extra, dtype=np.uint64))
    return np.concatenate(parts)
