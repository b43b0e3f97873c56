"""Pins for the CPU oracle (no GPU).  See tests/pins.py for what each pin is."""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from oracle import OracleTree
from paper_2604_21117_gb300 import workloads as W
import pins

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _parse_tree_fixture(name):
    spec = {"nodes": [], "queries": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "m":
                spec["m"] = int(tok[1])
            elif tok[0] == "keys":
                spec["keys"] = [int(x) for x in tok[1:]]
            elif tok[0] == "levels":
                spec["levels"] = [int(x) for x in tok[1:]]
            elif tok[0] == "node":
                spec["nodes"].append((int(tok[1]), int(tok[2]), tok[3] == "leaf", [int(x) for x in tok[4:]]))
            elif tok[0] == "query":
                p = tok.index("path")
                res = None if tok[2] == "miss" else int(tok[2])
                spec["queries"].append((int(tok[1]), res, [int(x) for x in tok[p + 1:]]))
    return spec


@pytest.mark.parametrize("name", ["order3_ten_keys.txt", "order4_thirteen_keys.txt"])
def test_golden_hand_worked_trees(name):
    spec = _parse_tree_fixture(name)
    keys = np.array(spec["keys"], np.uint64)
    vals = np.arange(keys.size, dtype=np.uint64)
    t = OracleTree(keys, vals, spec["m"])
    assert t.level_nodes() == spec["levels"]
    for level, idx, is_leaf, ks in spec["nodes"]:
        got_leaf, got_keys, _, _ = t.node(level, idx)
        assert got_leaf == is_leaf, (level, idx)
        assert [int(x) for x in got_keys] == ks, (level, idx)
    q = np.array([x[0] for x in spec["queries"]], np.uint64)
    v, f, _, _ = t.search(q)
    paths = t.paths(q)
    for i, (_, res, path) in enumerate(spec["queries"]):
        if res is None:
            assert f[i] == 0 and v[i] == np.uint64(2**64 - 1), int(q[i])
        else:
            assert f[i] == 1 and int(v[i]) == res, int(q[i])
        assert [int(x) for x in paths[i]] == path, int(q[i])


def _level_size_cases():
    cases = []
    with open(os.path.join(GOLDEN, "level_sizes.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                tok = [int(x) for x in line.split()]
                cases.append((tok[0], tok[1], tok[2:]))
    return cases


@pytest.mark.parametrize("n,m,levels", _level_size_cases())
def test_golden_level_sizes(n, m, levels):
    if n > 2**24:
        pytest.skip("2e7-key oracle tree is covered by the bench-side level check")
    keys = np.arange(n, dtype=np.uint64) * np.uint64(3) + np.uint64(1)
    t = OracleTree(keys, keys, m)
    assert t.level_nodes() == levels
    t.close()


@pytest.mark.parametrize("m", [3, 4, 5, 8, 16, 32])
@pytest.mark.parametrize("h", [1, 2, 3])
def test_full_tree_closed_forms(m, h):
    """Sec. III: a full tree of h levels holds m^(h-1) * k_max keys in
    exactly N_max = sum_{i<h} m^i nodes; one more key adds a level."""
    n = m ** (h - 1) * (m - 1)
    if n > 2_000_000:
        pytest.skip("too large for a unit test")
    keys = np.arange(n, dtype=np.uint64) * np.uint64(2)
    t = OracleTree(keys, keys, m)
    assert t.height == h
    assert sum(t.level_nodes()) == sum(m ** i for i in range(h))
    keys1 = np.arange(n + 1, dtype=np.uint64) * np.uint64(2)
    t1 = OracleTree(keys1, keys1, m)
    assert t1.height == h + 1


def _boundary_sizes(m):
    k = m - 1
    return sorted({0, 1, 2, k, k + 1, m * k, m * k + 1, m * m * k, m * m * k + 1})


@pytest.mark.parametrize("width", [32, 64])
@pytest.mark.parametrize("m", [3, 4, 8, 16, 32, 64])
def test_lookup_matches_lower_bound_at_height_boundaries(width, m):
    g = W.rng(1000 + m + width)
    for n in _boundary_sizes(m):
        if n > 300_000:
            continue
        keys = W.uniform_keys(n, width, seed=7 * n + m) if n else np.empty(0, W.key_dtype(width))
        vals = W.rank_values(n, 64)
        t = OracleTree(keys, vals, m)
        q = pins.probe_queries(keys, width, g)
        assert not pins.lookup_vs_lower_bound(t, keys, vals, q), (m, n)
        assert not pins.invariants(t, keys, vals), (m, n, pins.invariants(t, keys, vals)[:3])
        assert not pins.leaf_index_vs_leaf_max(t, q), (m, n)


@pytest.mark.parametrize("m", [3, 4, 5, 6, 7, 8, 9, 16, 32, 64])
def test_brute_force_tiny_trees(m):
    """Trees of up to 64 keys against a linear scan of the key list."""
    g = W.rng(77 + m)
    for n in range(0, 65):
        keys = np.sort(g.choice(1000, size=n, replace=False)).astype(np.uint64) * np.uint64(2) + np.uint64(5)
        vals = g.integers(0, 2**64, size=n, dtype=np.uint64)
        t = OracleTree(keys, vals, m)
        qs = np.arange(0, 2010, dtype=np.uint64)
        v, f, _, _ = t.search(qs)
        kl = [int(x) for x in keys]
        for i, q in enumerate(qs):
            want = None
            for j, k in enumerate(kl):  # linear scan
                if k == int(q):
                    want = int(vals[j])
            if want is None:
                assert f[i] == 0 and int(v[i]) == 2**64 - 1
            else:
                assert f[i] == 1 and int(v[i]) == want


def test_u32_value_miss_is_all_ones_of_width():
    keys = np.array([5, 9, 12], np.uint32)
    vals = np.array([1, 2, 0xFFFFFFFF], np.uint32)
    t = OracleTree(keys, vals, 4, val_bits=32)
    v, f, _, _ = t.search(np.array([5, 6, 12], np.uint32))
    assert list(map(int, v)) == [1, 0xFFFFFFFF, 0xFFFFFFFF]
    assert list(map(int, f)) == [1, 0, 1]  # a stored all-ones value stays distinguishable


def test_extreme_keys_zero_and_max():
    top = 2**64 - 1
    keys = np.array([0, 1, top - 1, top], np.uint64)
    vals = np.array([10, 11, 12, 13], np.uint64)
    for m in (3, 4, 8):
        t = OracleTree(keys, vals, m)
        v, f, _, _ = t.search(np.array([0, top, top - 1, 2, top - 2], np.uint64))
        assert list(map(int, f)) == [1, 1, 1, 0, 0]
        assert list(map(int, v[:3])) == [10, 13, 12]


def test_paths_are_parent_child_chains():
    keys = W.uniform_keys(5000, 64, seed=3)
    t = OracleTree(keys, keys, 8)
    q = W.make_queries(keys, 500, 0.5, seed=4, width_bits=64)
    P = t.paths(q)
    dump = pins.dump_tree(t)
    for row in P:
        for l in range(t.height - 1):
            ch = dump[l][int(row[l])][3]
            assert int(row[l + 1]) in set(int(c) for c in ch)


def test_touched_counts_match_set_counting():
    keys = W.uniform_keys(20000, 64, seed=11)
    vals = W.rank_values(keys.size, 64)
    m = 16
    t = OracleTree(keys, vals, m)
    q = W.make_queries(keys, 3000, 0.9, seed=12, width_bits=64)
    counts, sectors = t.touched(q)
    P = t.paths(q)
    assert counts == [len(set(int(x) for x in P[:, l])) for l in range(t.height)]
    # value sectors: leaf i, slot j -> byte (i*m + j)*8 -> sector //32, from searchsorted ranks
    _, f, leaf, slot = t.search(q)
    # slot of a hit independently: rank in sorted keys minus the leaf's first rank
    rank = np.searchsorted(keys, q)
    starts = np.array([0] + list(np.cumsum([len(t.node(t.height - 1, i)[1])
                                            for i in range(t.level_nodes()[-1])]))[:-1])
    hits = f.astype(bool)
    js = rank[hits] - starts[leaf[hits].astype(np.int64)]
    assert np.array_equal(js, slot[hits])
    sec = set(((leaf[hits].astype(np.int64) * m + js) * 8) // 32)
    assert sectors == len(sec)


def test_multithreaded_equals_single_threaded():
    keys = W.uniform_keys(50000, 64, seed=21)
    vals = W.rank_values(keys.size, 64)
    t = OracleTree(keys, vals, 16)
    q = W.make_queries(keys, 10007, 0.5, seed=22, width_bits=64)
    v1, f1, _, _ = t.search(q)
    for th in (2, 3, 8):
        v2, f2 = t.search_mt(q, th)
        assert np.array_equal(v1, v2) and np.array_equal(f1, f2)


def _pin_suite(lib):
    """A compact run of every pin; returns all failure messages."""
    errs = []
    for name in ("order3_ten_keys.txt", "order4_thirteen_keys.txt"):
        spec = _parse_tree_fixture(name)
        keys = np.array(spec["keys"], np.uint64)
        vals = np.arange(keys.size, dtype=np.uint64)
        t = OracleTree(keys, vals, spec["m"], lib=lib)
        if t.level_nodes() != spec["levels"]:
            errs.append(f"{name}: level sizes")
        q = np.array([x[0] for x in spec["queries"]], np.uint64)
        v, f, _, _ = t.search(q)
        for i, (_, res, _) in enumerate(spec["queries"]):
            if (res is None) != (f[i] == 0) or (res is not None and int(v[i]) != res):
                errs.append(f"{name}: query {int(q[i])}")
    g = W.rng(5)
    for m in (3, 8, 32):
        for n in (m * (m - 1) + 1, 3000):
            keys = W.uniform_keys(n, 64, seed=n + m)
            vals = W.rank_values(n, 64)
            t = OracleTree(keys, vals, m, lib=lib)
            q = pins.probe_queries(keys, 64, g)
            errs += pins.lookup_vs_lower_bound(t, keys, vals, q)
            errs += pins.invariants(t, keys, vals)
            errs += pins.leaf_index_vs_leaf_max(t, q)
    return errs


def test_pin_suite_passes_on_the_oracle():
    assert _pin_suite(oracle.load()) == []


@pytest.mark.parametrize("plant", ["BTO_PLANT_ROUTE_LT", "BTO_PLANT_SEP_MIN",
                                   "BTO_PLANT_LAST_CHILD", "BTO_PLANT_LEAF_FLOOR"])
def test_each_planted_mistake_is_caught(plant):
    lib = oracle.load_planted(plant)
    assert _pin_suite(lib), f"{plant} went unnoticed by every pin"
