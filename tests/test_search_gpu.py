"""GPU parity: the CUDA search through the C ABI against the CPU oracle,
bit-exact on values and found flags (all outputs are integers)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2604_21117_gb300 import workloads as W
from oracle import OracleTree
import pins
import sortcheck

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_21117_gb300 import build_lib
    build_lib.build()
    from paper_2604_21117_gb300 import btree
    return btree


def _to_dev(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu_search(tree, q: np.ndarray, sort_bits=-1):
    v, f = tree.search(_to_dev(q), sort_bits=sort_bits)
    return v.cpu().numpy(), f.cpu().numpy()


def _check(tree, oracle, q, sort_bits=-1, val_bits=64):
    gv, gf = _gpu_search(tree, q, sort_bits)
    ov, of, _, _ = oracle.search(q)
    assert gf.dtype == np.uint8
    bad = np.nonzero((gv.astype(np.uint64) != ov) | (gf != of))[0]
    assert bad.size == 0, (f"{bad.size} mismatches; first q={int(q[bad[0]])} gpu=({int(gv[bad[0]])},"
                           f"{int(gf[bad[0]])}) oracle=({int(ov[bad[0]])},{int(of[bad[0]])})")


def test_small_config_u32_fanout16(bt):
    """4096 distinct uint32 keys, rank values, m = 16; 256 lookups, exactly
    half hits; bit-exact against the oracle and against lower_bound."""
    keys = W.uniform_keys(4096, 32, seed=W.SEED_BASE + 1)
    vals = W.rank_values(keys.size, 32)
    q = W.make_queries(keys, 256, 0.5, seed=W.SEED_BASE + 2, width_bits=32, exact_hits=True)
    tree = bt.BTree(keys, vals, 16)
    assert tree.level_nodes == [1, 2, 18, 274]
    o = OracleTree(keys, vals, 16, val_bits=32)
    for sb in (-1, 0, 8, 16, 32):
        _check(tree, o, q, sb, 32)
    gv, gf = _gpu_search(tree, q)
    ev, ef = pins.reference_lookup(keys, vals, q, 32)
    assert np.array_equal(gv.astype(np.uint64), ev) and np.array_equal(gf, ef)
    assert int(gf.sum()) == 128


@pytest.mark.parametrize("m", [8, 16, 32, 64])
@pytest.mark.parametrize("kw,vw", [(32, 32), (32, 64), (64, 32), (64, 64)])
def test_widths_and_fanouts_sorted_and_unsorted(bt, m, kw, vw):
    n = 60_000 + m
    keys = W.uniform_keys(n, kw, seed=100 + m + kw)
    vals = W.rank_values(n, vw)
    tree = bt.BTree(keys, vals, m)
    o = OracleTree(keys, vals, m, val_bits=vw)
    q = W.make_queries(keys, 20_011, 0.7, seed=200 + m, width_bits=kw)  # ragged: not a multiple of 32
    for sb in (0, 8, 16, kw):
        _check(tree, o, q, sb, vw)


@pytest.mark.parametrize("m", [8, 16, 32, 64])
def test_height_boundaries_and_probe_queries(bt, m):
    g = W.rng(300 + m)
    k = m - 1
    for n in (1, 2, k, k + 1, m * k, m * k + 1, m * m * k, m * m * k + 1):
        keys = W.uniform_keys(n, 64, seed=400 + n)
        vals = g.integers(0, 2**64, size=n, dtype=np.uint64)
        tree = bt.BTree(keys, vals, m)
        o = OracleTree(keys, vals, m)
        assert tree.level_nodes == o.level_nodes()
        q = pins.probe_queries(keys, 64, g)
        for sb in (0, 16):
            _check(tree, o, q, sb)


def test_extreme_keys_and_all_ones_value(bt):
    top = 2**64 - 1
    keys = np.array([0, 1, 2**63, top - 1, top], np.uint64)
    vals = np.array([top, 0, 5, 6, 7], np.uint64)
    tree = bt.BTree(keys, vals, 8)
    o = OracleTree(keys, vals, 8)
    q = np.array([0, top, top - 1, 2, 2**63, 2**63 - 1, 1, top, 0], np.uint64)
    for sb in (0, 8, 64):
        _check(tree, o, q, sb)
    gv, gf = _gpu_search(tree, q)
    assert int(gv[0]) == top and int(gf[0]) == 1  # stored all-ones is a hit


def test_empty_tree_and_single_key(bt):
    tree = bt.BTree(np.empty(0, np.uint64), np.empty(0, np.uint64), 32)
    q = np.array([0, 5, 2**64 - 1], np.uint64)
    gv, gf = _gpu_search(tree, q)
    assert np.all(gf == 0) and np.all(gv == np.uint64(2**64 - 1))
    tree1 = bt.BTree(np.array([42], np.uint32), np.array([7], np.uint32), 16)
    gv, gf = _gpu_search(tree1, np.array([41, 42, 43], np.uint32))
    assert list(gf) == [0, 1, 0] and list(map(int, gv)) == [0xFFFFFFFF, 7, 0xFFFFFFFF]


@pytest.mark.parametrize("nq", [1, 31, 32, 33, 4095, 4096, 4097, 16383, 16384, 70001])
def test_ragged_batch_sizes(bt, nq):
    keys = W.uniform_keys(30_000, 64, seed=5)
    vals = W.rank_values(keys.size, 64)
    tree = bt.BTree(keys, vals, 16)
    o = OracleTree(keys, vals, 16)
    q = W.make_queries(keys, nq, 0.9, seed=nq, width_bits=64)
    for sb in (-1, 0, 16):
        _check(tree, o, q, sb)


def test_duplicate_and_skewed_queries(bt):
    keys = W.uniform_keys(100_000, 64, seed=9)
    vals = W.rank_values(keys.size, 64)
    tree = bt.BTree(keys, vals, 32)
    o = OracleTree(keys, vals, 32)
    q = W.make_queries(keys, 50_000, 0.9, seed=10, width_bits=64, zipf_s=1.1)
    for sb in (-1, 0, 16, 64):
        _check(tree, o, q, sb)
    same = np.full(10_000, keys[777], np.uint64)
    _check(tree, o, same, 16)
    _check(tree, o, same, 0)


def test_lognormal_keys(bt):
    keys = W.lognormal_mixture_keys(200_000, seed=11)
    vals = W.rank_values(keys.size, 64)
    tree = bt.BTree(keys, vals, 32)
    o = OracleTree(keys, vals, 32)
    q = W.make_queries(keys, 40_000, 0.9, seed=12, width_bits=64)
    for sb in (-1, 0, 16, 64):
        _check(tree, o, q, sb)


def test_device_layout_matches_oracle_nodes(bt):
    """The device image, copied back, holds per level m key slots per node,
    each level 256-byte aligned, padding all-ones, leaf values per slot --
    node for node equal to the oracle's pointer tree."""
    n, m = 5000, 16
    keys = W.uniform_keys(n, 64, seed=13)
    vals = W.rank_values(n, 64)
    tree = bt.BTree(keys, vals, m)
    o = OracleTree(keys, vals, m)
    info = bt.bt_tree_info(tree.handle)
    img = bt.bt_tree_copy_image(tree.handle, int(info.device_bytes))
    for l in range(tree.height):
        off = int(info.level_key_offset[l])
        assert off % 256 == 0
        blocks = img[off: off + tree.level_nodes[l] * m * 8].view(np.uint64).reshape(-1, m)
        for i in range(tree.level_nodes[l]):
            is_leaf, ks, vs, _ = o.node(l, i)
            assert np.array_equal(blocks[i, :ks.size], ks)
            assert np.all(blocks[i, ks.size:] == np.uint64(2**64 - 1))
            if is_leaf:
                voff = int(info.leaf_val_offset)
                assert voff % 256 == 0
                vb = img[voff: voff + tree.level_nodes[l] * m * 8].view(np.uint64).reshape(-1, m)
                assert np.array_equal(vb[i, :vs.size], vs)


@pytest.mark.parametrize("sb", [64, 16, 0])
def test_fetch_counts_equal_distinct_nodes_per_warp(bt, sb):
    """Every warp of 32 consecutive queries of the (sorted) batch fetches
    each distinct node it needs exactly once per level (Sec. IV-A)."""
    import torch
    keys = W.uniform_keys(200_000, 64, seed=14)
    vals = W.rank_values(keys.size, 64)
    m = 16
    tree = bt.BTree(keys, vals, m)
    o = OracleTree(keys, vals, m)
    q = W.make_queries(keys, 30_000, 0.9, seed=15, width_bits=64, zipf_s=1.1)
    cnt = torch.zeros(tree.height, dtype=torch.int64, device="cuda")
    sq, si, hsq, _ = _sorted(bt, tree, q, sb)
    v, f = tree.alloc_outputs(q.size)
    bt.bt_descend_sorted(tree.handle, sq, si, q.size, v, f, cnt)
    got = [int(x) for x in cnt.cpu().numpy()]
    ov, of, _, _ = o.search(q)
    assert np.array_equal(v.cpu().numpy(), ov) and np.array_equal(f.cpu().numpy(), of)
    paths = o.paths(hsq)
    want = []
    for l in range(tree.height):
        col = paths[:, l]
        want.append(sum(len(set(col[i:i + 32].tolist())) for i in range(0, col.size, 32)))
    assert got == want
    dist, _ = o.touched(q)
    assert all(g >= d for g, d in zip(got, dist))


def test_host_buffer_entry_point(bt):
    keys = W.uniform_keys(50_000, 64, seed=16)
    vals = W.rank_values(keys.size, 64)
    tree = bt.BTree(keys, vals, 32)
    o = OracleTree(keys, vals, 32)
    q = W.make_queries(keys, 33_333, 0.9, seed=17, width_bits=64)
    hv, hf = tree.search_host(q)
    ov, of, _, _ = o.search(q)
    assert np.array_equal(hv, ov) and np.array_equal(hf, of)


@pytest.mark.slow
@pytest.mark.parametrize("zipf", [None, 1.1])
def test_full_size_2p24_keys_fanout32(bt, zipf):
    """2^24 distinct uniform uint64 keys, m = 32, uint64 rank values; batches
    1..2^20 at 90% hits, every result checked against the oracle."""
    n = 1 << 24
    keys = W.uniform_keys(n, 64, seed=W.SEED_BASE + 2)
    vals = W.rank_values(n, 64)
    tree = bt.BTree(keys, vals, 32)
    assert tree.level_nodes == [1, 17, 529, 16913, 541201]
    assert bt.bt_sort_bits(tree.handle, 786431, -1) == 0 and bt.bt_sort_bits(tree.handle, 786432, -1) > 9
    o = OracleTree(keys, vals, 32)
    for b in (1, 16, 64, 256, 1024, 1 << 20):
        q = W.make_queries(keys, b, 0.9, seed=W.SEED_BASE + 1000 + b, width_bits=64, zipf_s=zipf)
        # the tree's image exceeds the L2: the automatic choice partitions 2^20 queries only
        assert (bt.bt_sort_bits(tree.handle, b, -1) > 9) == (b == 1 << 20)
        _check(tree, o, q, -1)
        if b == 1 << 20:
            _check(tree, o, q, 0)


def _sorted(bt, tree, q, sb):
    import torch
    dq = _to_dev(q)
    sq = torch.empty_like(dq)
    si = torch.empty(q.size, dtype=torch.int32, device="cuda")
    ws, nb = tree.alloc_workspace(q.size)
    bt.bt_sort_batch(tree.handle, dq, q.size, sb, sq, si, ws, nb)
    return sq, si, sq.cpu().numpy(), si.cpu().numpy().view(np.uint32)


def _splitters(bt, tree):
    info = bt.bt_tree_info(tree.handle)
    img = bt.bt_tree_copy_image(tree.handle, int(info.device_bytes))
    kb = int(info.key_bytes)
    dt = np.uint64 if kb == 8 else np.uint32
    o = int(info.split_offset)
    sp = img[o: o + int(info.nsplit) * kb].view(dt).astype(np.uint64)
    return sp, int(info.nsplit)


def _check_sort_contract(bt, tree, keys, q, hsq, hsi, sb):
    """A permutation with its keys, in the documented order: by coarse
    bucket, and inside coarse buckets of at most the tile size by the bucket
    number f -- exactly by splitter segment (the count of the tree's
    splitters below the key), inside a segment out of order only between keys
    less than one interpolation bucket apart."""
    nq = q.size
    assert np.array_equal(np.sort(hsi), np.arange(nq, dtype=np.uint32))
    assert np.array_equal(hsq, q[hsi])
    sp, nsplit = _splitters(bt, tree)
    bits = bt.bt_sort_bits(tree.handle, nq, sb)
    if bits == 0:
        assert np.array_equal(hsi, np.arange(nq, dtype=np.uint32))
        return
    if sb > 0:
        assert bits == min(sb, 21)
    if sb < 0:  # automatic: only for large batches on trees larger than a quarter of the L2
        assert nq >= 786432 and bits > 9
    k = hsq.astype(np.uint64)
    c = np.searchsorted(sp, k, side="left")
    lo = np.concatenate([[int(keys[0])], sp.astype(object)]) if nsplit else np.array([int(keys[0])], object)
    hi = np.concatenate([sp.astype(object), [int(keys[-1])]]) if nsplit else np.array([int(keys[-1])], object)
    lo_f = np.array([float(x) for x in lo])
    width = np.array([float(int(h) - int(l) + 1) for l, h in zip(lo, hi)])
    # keys beyond the key range share the end buckets
    run = np.clip(k, np.uint64(keys[0]), np.uint64(keys[-1])).astype(np.float64)
    sortcheck.check_order(c, bits, nsplit, sortcheck.tile_for(int(keys.dtype.itemsize)),
                          pos=run - lo_f[c], width=width[c])


@pytest.mark.parametrize("kw", [32, 64])
@pytest.mark.parametrize("sb", [-1, 0, 8, 16, 64])
def test_split_sort_then_descend(bt, kw, sb):
    """bt_sort_batch yields a permutation with the documented order, and
    bt_descend_sorted on it gives the oracle's results."""
    keys = W.uniform_keys(80_000, kw, seed=18)
    vals = W.rank_values(keys.size, 64)
    tree = bt.BTree(keys, vals, 32)
    o = OracleTree(keys, vals, 32)
    q = W.make_queries(keys, 50_001, 0.9, seed=19, width_bits=kw, zipf_s=1.1)
    sq, si, hsq, hsi = _sorted(bt, tree, q, sb)
    _check_sort_contract(bt, tree, keys, q, hsq, hsi, sb)
    v, fo = tree.alloc_outputs(q.size)
    bt.bt_descend_sorted(tree.handle, sq, si, q.size, v, fo)
    ov, of, _, _ = o.search(q)
    assert np.array_equal(v.cpu().numpy().astype(np.uint64), ov)
    assert np.array_equal(fo.cpu().numpy(), of)


@pytest.mark.parametrize("dist", ["uniform", "zipf", "lognormal", "same"])
@pytest.mark.parametrize("nq", [1, 4095, 16383, 16384, 100_000, 1 << 20])
def test_sort_contract_sizes_and_skew(bt, dist, nq):
    """The partition on skewed input (a hot key's bucket holds most of the
    batch), skewed keys (splitter segments follow the key distribution) and
    sizes from 1 to 2^20; the tree is small (5 MB), so the automatic choice
    is no partition at every size."""
    keys = W.lognormal_mixture_keys(300_000, seed=20) if dist == "lognormal" else W.uniform_keys(300_000, 64, seed=20)
    tree = bt.BTree(keys, W.rank_values(keys.size, 64), 32)
    if dist == "same":
        q = np.full(nq, keys[1234], np.uint64)
    else:
        q = W.make_queries(keys, nq, 0.9, seed=nq + 1, width_bits=64, zipf_s=1.1 if dist == "zipf" else None)
    for sb in (-1, 4, 16, 64):
        _, _, hsq, hsi = _sorted(bt, tree, q, sb)
        _check_sort_contract(bt, tree, keys, q, hsq, hsi, sb)
