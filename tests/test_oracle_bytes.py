"""Pins for the byte-string-key oracle (no GPU).

The oracle's answers are checked against things other than itself: a Python
dict (the plain definition of a point lookup), Python's bytes ordering with
bisect (the leaf a query must reach), the integer-key oracle on big-endian
encodings of integers (where lexicographic byte order equals integer order),
and structural invariants; a planted little-endian compare must fail them.
"""
from __future__ import annotations

import bisect

import numpy as np
import pytest

from oracle import OracleTree
from oracle import bytes_keys as OB
from paper_2604_21117_gb300 import workloads as W


def _leaf_rows(t):
    h = t.height
    return [t.node(h - 1, i) for i in range(t.level_nodes()[-1])]


def _pin_errors(t, keys, vals, queries):
    """Failure messages of the dict and lower-bound pins (empty = pinned)."""
    errs = []
    ev, ef = OB.dict_lookup(keys, vals, queries, t.val_bits)
    v, f, leaf, slot = t.search(queries)
    if not (np.array_equal(v, ev) and np.array_equal(f, ef)):
        errs.append("lookup differs from the dict")
    if t.height:
        leaf_max = [bytes(x[1][-1]) for x in _leaf_rows(t)]
        want = [min(bisect.bisect_left(leaf_max, bytes(q)), len(leaf_max) - 1) for q in queries]
        if not np.array_equal(leaf, np.array(want, np.uint64)):
            errs.append("leaf differs from the lower bound over leaf maxima")
    return errs


@pytest.mark.parametrize("n,m,prefix", [(0, 4, 0), (1, 4, 0), (2, 3, 0), (37, 3, 0), (200, 4, 2),
                                        (1000, 8, 0), (5000, 16, 8), (20000, 32, 24), (70000, 64, 0)])
def test_lookup_and_leaf_pins(n, m, prefix):
    keys = W.byte_keys(n, 32, seed=100 + n, prefix_bytes=prefix)
    vals = np.arange(n, dtype=np.uint64) * 7 + 3
    t = OB.OracleBytesTree(keys, vals, m)
    q = W.make_byte_queries(keys, 3000, 0.5, seed=200 + n)
    extra = [np.zeros((1, 32), np.uint8), np.full((1, 32), 255, np.uint8)]
    if n:
        # neighbours of stored keys: last byte +- 1 where it does not wrap
        k = keys[: min(n, 500)].copy()
        up = k[k[:, -1] < 255].copy()
        up[:, -1] += 1
        dn = k[k[:, -1] > 0].copy()
        dn[:, -1] -= 1
        extra += [k, up, dn]
    q = np.concatenate([q] + extra)
    assert _pin_errors(t, keys, vals, q) == []


@pytest.mark.parametrize("n,m", [(1, 3), (50, 3), (1234, 8), (40000, 32)])
def test_equals_integer_oracle_on_big_endian_encodings(n, m):
    """Keys that are 24 zero bytes followed by a big-endian uint64: byte order
    is integer order, so leaves, slots and every path must equal the
    integer-key oracle's."""
    ik = W.uniform_keys(n, 64, seed=300 + n)
    iv = W.rank_values(n, 64)
    bk = np.zeros((n, 32), np.uint8)
    bk[:, 24:] = ik.astype(">u8").view(np.uint8).reshape(n, 8)
    iq = W.make_queries(ik, 4000, 0.6, seed=301, width_bits=64)
    bq = np.zeros((iq.size, 32), np.uint8)
    bq[:, 24:] = iq.astype(">u8").view(np.uint8).reshape(iq.size, 8)
    a = OracleTree(ik, iv, m)
    b = OB.OracleBytesTree(bk, iv, m)
    assert a.level_nodes() == b.level_nodes()
    for x, y in zip(a.search(iq), b.search(bq)):
        assert np.array_equal(x, y)
    assert np.array_equal(a.paths(iq), b.paths(bq))


@pytest.mark.parametrize("n,m", [(1, 4), (31, 4), (999, 8), (30000, 16)])
def test_structure_invariants(n, m):
    keys = W.byte_keys(n, 32, seed=400 + n, prefix_bytes=3)
    vals = np.arange(n, dtype=np.uint64)
    t = OB.OracleBytesTree(keys, vals, m)
    h = t.height
    levels = [[t.node(l, i) for i in range(c)] for l, c in enumerate(t.level_nodes())]
    leaves = levels[-1]
    cat = np.concatenate([x[1] for x in leaves])
    assert np.array_equal(cat, keys)
    assert np.array_equal(np.concatenate([x[2] for x in leaves]), vals)
    sub_max = [bytes(x[1][-1]) for x in leaves]
    for l in range(h - 2, -1, -1):
        nxt = 0
        maxes = []
        for _, ks, _, ch in levels[l]:
            ch = [int(c) for c in ch]
            assert ch == list(range(nxt, nxt + len(ch)))
            nxt += len(ch)
            assert len(ch) <= m and (l == 0 or len(ch) >= -(-m // 2))
            assert [bytes(s) for s in ks] == [sub_max[c] for c in ch[:-1]]
            maxes.append(sub_max[ch[-1]])
        sub_max = maxes
    # level sizes depend on n and m only
    assert t.level_nodes() == OracleTree(np.arange(n, dtype=np.uint64), vals, m).level_nodes()


def test_empty_tree_misses_everything():
    t = OB.OracleBytesTree(np.zeros((0, 32), np.uint8), np.zeros(0, np.uint64), 16, val_bits=32)
    v, f, leaf, slot = t.search(np.zeros((3, 32), np.uint8))
    assert t.height == 0 and np.all(f == 0) and np.all(v == 2**32 - 1) and np.all(slot == -1)


def test_planted_little_endian_compare_is_caught():
    lib = OB.load_planted("BTB_PLANT_LAST_BYTE_FIRST")
    keys = W.byte_keys(3000, 32, seed=500)
    vals = np.arange(3000, dtype=np.uint64)
    t = OB.OracleBytesTree(keys, vals, 8, lib=lib)
    q = W.make_byte_queries(keys, 2000, 0.7, seed=501)
    assert _pin_errors(t, keys, vals, q) != []


def test_multithreaded_equals_single():
    keys = W.byte_keys(20000, 32, seed=600)
    vals = np.arange(20000, dtype=np.uint64)
    t = OB.OracleBytesTree(keys, vals, 16)
    q = W.make_byte_queries(keys, 10001, 0.5, seed=601)
    v1, f1, _, _ = t.search(q)
    v2, f2 = t.search_mt(q, 4)
    assert np.array_equal(v1, v2) and np.array_equal(f1, f2)


def test_byte_key_generators():
    k = W.byte_keys(5000, 32, seed=700, prefix_bytes=5)
    rows = [bytes(r) for r in k]
    assert rows == sorted(set(rows)) and len(rows) == 5000
    assert np.all(k[:, :5] == k[0, :5])
    q = W.make_byte_queries(k, 4000, 0.4, seed=701)
    hits = sum(bytes(r) in set(rows) for r in q)
    assert 0.35 < hits / 4000 < 0.45
