"""32-byte keys (the paper's key format) on the GPU, bit-exact against the
byte-key oracle: every fanout and value width, with and without the batch
partition, both node staging modes, shared key prefixes, the all-zero and
all-ones keys, ragged batch sizes, host-buffer and no-alloc entry points."""
from __future__ import annotations

import bisect

import numpy as np
import pytest

import sortcheck

from oracle.bytes_keys import OracleBytesTree
from paper_2604_21117_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_21117_gb300 import btree
    return btree


def _dev(q):
    import torch
    return torch.from_numpy(np.ascontiguousarray(q)).cuda()


def _check(bt, tree, o, q, sb=-1):
    v, f = tree.search(_dev(q), sort_bits=sb)
    ov, of, _, _ = o.search(q)
    got_v = v.cpu().numpy().astype(np.uint64)
    assert np.array_equal(f.cpu().numpy(), of), sb
    assert np.array_equal(got_v, ov), sb


def _edge_keys(keys):
    """Stored keys plus the all-zero and all-ones keys, re-sorted."""
    extra = np.stack([np.zeros(32, np.uint8), np.full(32, 255, np.uint8)])
    k = np.concatenate([keys, extra])
    order = np.lexsort(k.T[::-1])
    k = k[order]
    keep = np.ones(k.shape[0], bool)
    keep[1:] = np.any(k[1:] != k[:-1], axis=1)
    return np.ascontiguousarray(k[keep])


@pytest.mark.parametrize("m", [8, 16, 32, 64])
@pytest.mark.parametrize("vbits", [32, 64])
def test_parity_every_fanout_and_value_width(bt, m, vbits):
    keys = _edge_keys(W.byte_keys(60_000, 32, seed=900 + m))
    vals = W.rank_values(keys.shape[0], vbits)
    tree = bt.BTree(keys, vals, m)
    assert tree.key_bytes == 32
    o = OracleBytesTree(keys, vals, m, val_bits=vbits)
    q = W.make_byte_queries(keys, 40_003, 0.7, seed=901)
    q = np.concatenate([q, keys[:1], keys[-1:], np.full((3, 32), 255, np.uint8), np.zeros((2, 32), np.uint8)])
    for sb in (-1, 0, 8, 16):
        _check(bt, tree, o, q, sb)


@pytest.mark.parametrize("prefix", [0, 8, 13, 24, 30])
def test_shared_prefixes(bt, prefix):
    """Keys that share their first `prefix` bytes: the partition interpolates
    on the bytes after the shared ones."""
    keys = W.byte_keys(100_000 if prefix < 30 else 10_000, 32, seed=910 + prefix, prefix_bytes=prefix)
    vals = W.rank_values(keys.shape[0], 64)
    tree = bt.BTree(keys, vals, 16)
    o = OracleBytesTree(keys, vals, 16)
    q = W.make_byte_queries(keys, 70_001, 0.5, seed=911)
    _check(bt, tree, o, q, -1)
    _check(bt, tree, o, q, 16)


@pytest.mark.parametrize("n", [1, 2, 15, 16, 17, 1000])
@pytest.mark.parametrize("nq", [1, 31, 33, 20_000])
def test_small_trees_and_ragged_batches(bt, n, nq):
    keys = W.byte_keys(n, 32, seed=920 + n)
    vals = W.rank_values(n, 32)
    tree = bt.BTree(keys, vals, 16)
    o = OracleBytesTree(keys, vals, 16, val_bits=32)
    q = W.make_byte_queries(keys, nq, 0.5, seed=921 + nq)
    for sb in (-1, 0, 12):
        _check(bt, tree, o, q, sb)


def test_empty_tree_misses(bt):
    tree = bt.BTree(np.zeros((0, 32), np.uint8), np.zeros(0, np.uint64), 32)
    v, f = tree.search(_dev(np.zeros((5, 32), np.uint8)))
    assert np.all(f.cpu().numpy() == 0) and np.all(v.cpu().numpy() == np.uint64(2**64 - 1))


@pytest.mark.parametrize("m", [8, 16, 32, 64])
def test_bulk_staging(bt, m):
    keys = W.byte_keys(50_000, 32, seed=930 + m)
    vals = W.rank_values(keys.shape[0], 64)
    tree = bt.BTree(keys, vals, m)
    bt.bt_tree_set_staging(tree.handle, bt.BT_STAGE_BULK)
    o = OracleBytesTree(keys, vals, m)
    q = W.make_byte_queries(keys, 30_001, 0.6, seed=931)
    _check(bt, tree, o, q, -1)
    _check(bt, tree, o, q, 0)
    _check(bt, tree, o, q, 16)
    bt.bt_check_timeouts()


@pytest.mark.parametrize("warps,pin,lq", [(4, 0, 1), (16, 49152, 1), (8, 16384, 2)])
def test_launch_settings(bt, warps, pin, lq):
    keys = W.byte_keys(80_000, 32, seed=940)
    vals = W.rank_values(keys.shape[0], 64)
    tree = bt.BTree(keys, vals, 16)
    bt.bt_tree_set_launch(tree.handle, warps, pin)
    bt.bt_tree_set_lane_queries(tree.handle, lq)
    o = OracleBytesTree(keys, vals, 16)
    q = W.make_byte_queries(keys, 25_000, 0.6, seed=941)
    _check(bt, tree, o, q)
    _check(bt, tree, o, q, 16)


def test_device_layout_is_big_endian_words(bt):
    n, m = 3000, 8
    keys = W.byte_keys(n, 32, seed=950)
    vals = W.rank_values(n, 64)
    tree = bt.BTree(keys, vals, m)
    o = OracleBytesTree(keys, vals, m)
    info = bt.bt_tree_info(tree.handle)
    assert int(info.key_bytes) == 32
    img = bt.bt_tree_copy_image(tree.handle, int(info.device_bytes))
    for l in range(tree.height):
        off = int(info.level_key_offset[l])
        words = img[off: off + tree.level_nodes[l] * m * 32].view(np.uint64).reshape(-1, m, 4)
        for i in range(tree.level_nodes[l]):
            _, ks, _, _ = o.node(l, i)
            want = ks.reshape(-1, 4, 8).view(">u8").reshape(-1, 4).astype(np.uint64)
            assert np.array_equal(words[i, :ks.shape[0]], want)
            assert np.all(words[i, ks.shape[0]:] == np.uint64(2**64 - 1))


def test_partition_orders_by_splitter_segment(bt):
    """The partitioned batch is a permutation in the documented order: by
    coarse bucket, and inside coarse buckets of at most 2048 queries by the
    number of splitters below each query (lexicographic byte order)."""
    import torch
    keys = W.byte_keys(200_000, 32, seed=960, prefix_bytes=3)
    vals = W.rank_values(keys.shape[0], 64)
    tree = bt.BTree(keys, vals, 32)
    q = W.make_byte_queries(keys, 100_000, 0.8, seed=961)
    dq = _dev(q)
    sq = torch.empty_like(dq)
    si = torch.empty(q.shape[0], dtype=torch.int32, device="cuda")
    ws, nb = tree.alloc_workspace(q.shape[0])
    bt.bt_sort_batch(tree.handle, dq, q.shape[0], 16, sq, si, ws, nb)
    hsq, hsi = sq.cpu().numpy(), si.cpu().numpy().view(np.uint32)
    assert np.array_equal(np.sort(hsi), np.arange(q.shape[0], dtype=np.uint32))
    assert np.array_equal(hsq, q[hsi])
    info = bt.bt_tree_info(tree.handle)
    img = bt.bt_tree_copy_image(tree.handle, int(info.device_bytes))
    o = int(info.split_offset)
    ns = int(info.nsplit)
    sp_words = img[o: o + ns * 32].view(np.uint64).reshape(ns, 4)
    sp = [sp_words[j].astype(">u8").tobytes() for j in range(ns)]
    c = np.array([bisect.bisect_left(sp, bytes(r)) for r in hsq])
    sortcheck.check_order(c, bt.bt_sort_bits(tree.handle, q.shape[0], 16), ns, sortcheck.tile_for(32))
    v, f = tree.alloc_outputs(q.shape[0])
    bt.bt_descend_sorted(tree.handle, sq, si, q.shape[0], v, f)
    ov, of, _, _ = OracleBytesTree(keys, vals, 32).search(q)
    assert np.array_equal(v.cpu().numpy(), ov) and np.array_equal(f.cpu().numpy(), of)


def test_host_buffers_and_noalloc(bt):
    import torch
    keys = W.byte_keys(30_000, 32, seed=970)
    vals = W.rank_values(keys.shape[0], 64)
    tree = bt.BTree(keys, vals, 16)
    o = OracleBytesTree(keys, vals, 16)
    q = W.make_byte_queries(keys, 20_001, 0.6, seed=971)
    ov, of, _, _ = o.search(q)
    hv, hf = tree.search_host(q)
    assert np.array_equal(hv, ov) and np.array_equal(hf, of)
    v, f = tree.alloc_outputs(q.shape[0])
    bt.bt_search_batch_noalloc(tree.handle, _dev(q), q.shape[0], v, f)
    torch.cuda.synchronize()
    assert np.array_equal(v.cpu().numpy(), ov) and np.array_equal(f.cpu().numpy(), of)


def test_unsupported_uses_are_refused(bt):
    keys = W.byte_keys(1000, 32, seed=980)
    tree = bt.BTree(keys, W.rank_values(1000, 64), 16)
    with pytest.raises(bt.BTreeError):
        bt.bt_model_train(tree.handle, bt.BT_MODEL_PL, segments=16)
    with pytest.raises(bt.BTreeError):
        bt.bt_forest_create([tree])


@pytest.mark.slow
def test_paper_tree_full_batch(bt):
    """The paper's own tree (2^20 distinct 32-byte keys, 8-byte values,
    fanout 16) and a batch of 2^20 queries at 90% hits: the automatic choice
    partitions it (the tree's image is larger than a quarter of the L2 and
    the batch above the 32-byte keys' threshold), and
    every result, through both node layouts, equals the byte-key oracle."""
    import torch
    n = nq = 1 << 20
    keys = W.byte_keys(n, 32, seed=W.SEED_BASE + 8)
    vals = W.rank_values(n, 64)
    tree = bt.BTree(keys, vals, 16)
    o = OracleBytesTree(keys, vals, 16)
    q = W.make_byte_queries(keys, nq, 0.9, seed=W.SEED_BASE + 9 + nq)
    assert bt.bt_sort_bits(tree.handle, nq, -1) == 20
    # 32-byte keys are partitioned automatically from 393216 queries
    assert bt.bt_sort_bits(tree.handle, 393215, -1) == 0 and bt.bt_sort_bits(tree.handle, 393216, -1) > 9
    _check(bt, tree, o, q, -1)
    bt.bt_paper_layout_build(tree.handle)
    v, f = tree.alloc_outputs(nq)
    ws, nb = tree.alloc_workspace(nq)
    bt.bt_paper_search_batch(tree.handle, _dev(q), nq, v, f, ws, nb)
    ov, of, _, _ = o.search(q)
    assert np.array_equal(v.cpu().numpy(), ov) and np.array_equal(f.cpu().numpy(), of)
    torch.cuda.synchronize()
    o.close()
    tree.close()


def test_misaligned_arrays_are_refused(bt):
    """32-byte keys move as 16-byte pieces: a key array that is not 16-byte
    aligned is refused on the host (BT_ERR_ARG) before anything is launched,
    by the search, the sort and the descent; so is a misaligned value array."""
    import torch
    keys = W.byte_keys(5000, 32, seed=990)
    tree = bt.BTree(keys, W.rank_values(keys.shape[0], 64), 16)
    nq = 1000
    buf = torch.zeros((nq + 1) * 32, dtype=torch.uint8, device="cuda")
    base = buf.data_ptr()
    assert base % 256 == 0
    v, f = tree.alloc_outputs(nq)
    ws, nb = tree.alloc_workspace(nq)
    si = torch.empty(nq, dtype=torch.int32, device="cuda")
    # every misaligned pointer still has room for the whole array after it
    obuf = torch.zeros((nq + 1) * 32, dtype=torch.uint8, device="cuda")
    vbuf = torch.zeros(nq + 1, dtype=torch.uint64, device="cuda")
    ibuf = torch.zeros(nq + 1, dtype=torch.int32, device="cuda")
    for call in (
        lambda: bt.bt_search_batch(tree.handle, base + 8, nq, v, f, ws, nb),
        lambda: bt.bt_search_batch(tree.handle, base, nq, vbuf.data_ptr() + 4, f, ws, nb),
        lambda: bt.bt_sort_batch(tree.handle, base + 8, nq, 16, obuf, si, ws, nb),
        lambda: bt.bt_sort_batch(tree.handle, base, nq, 16, obuf.data_ptr() + 8, si, ws, nb),
        lambda: bt.bt_descend_sorted(tree.handle, base + 8, si, nq, v, f),
        lambda: bt.bt_descend_sorted(tree.handle, base, ibuf.data_ptr() + 2, nq, v, f),
    ):
        with pytest.raises(bt.BTreeError) as e:
            call()
        assert e.value.code == "BT_ERR_ARG"
    # the aligned calls on the same buffers go through
    bt.bt_search_batch(tree.handle, base, nq, v, f, ws, nb)
    torch.cuda.synchronize()
    tree.close()
