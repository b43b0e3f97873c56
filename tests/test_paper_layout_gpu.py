"""The paper's node layout (Eq. 1: header, keys, child addresses or data in
one node, BFS order) searched on the GPU: bit-exact against the oracles for
every key width and fanout, on the batch as given and on the batch
partitioned by bt_sort_batch."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import OracleTree
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


def _run(bt, tree, q, nq):
    import torch
    dq = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    v, f = tree.alloc_outputs(nq)
    ws, nb = tree.alloc_workspace(nq)
    bt.bt_paper_search_batch(tree.handle, dq, nq, v, f, ws, nb)
    pv, pf = v.cpu().numpy(), f.cpu().numpy()
    v2, f2 = tree.alloc_outputs(nq)
    bt.bt_paper_descend_sorted(tree.handle, dq, None, nq, v2, f2)  # unsorted order
    assert np.array_equal(v2.cpu().numpy(), pv) and np.array_equal(f2.cpu().numpy(), pf)
    sq = torch.empty_like(dq)
    si = torch.empty(nq, dtype=torch.int32, device="cuda")
    bt.bt_sort_batch(tree.handle, dq, nq, 16, sq, si, ws, nb)
    v3, f3 = tree.alloc_outputs(nq)
    bt.bt_paper_descend_sorted(tree.handle, sq, si, nq, v3, f3)  # partitioned, results in input order
    assert np.array_equal(v3.cpu().numpy(), pv) and np.array_equal(f3.cpu().numpy(), pf)
    return pv, pf


@pytest.mark.parametrize("m", [8, 16, 32, 64])
@pytest.mark.parametrize("kw,vw", [(32, 32), (64, 64), (64, 32)])
def test_integer_keys(bt, m, kw, vw):
    keys = W.uniform_keys(150_000, kw, seed=1000 + m)
    vals = W.rank_values(keys.size, vw)
    tree = bt.BTree(keys, vals, m)
    bt.bt_paper_layout_build(tree.handle)
    o = OracleTree(keys, vals, m, val_bits=vw)
    q = W.make_queries(keys, 50_003, 0.8, seed=1001, width_bits=kw, zipf_s=1.05)
    pv, pf = _run(bt, tree, q, q.size)
    ov, of, _, _ = o.search(q)
    assert np.array_equal(pv.astype(np.uint64), ov) and np.array_equal(pf, of)


@pytest.mark.parametrize("m", [8, 16, 32, 64])
def test_32_byte_keys(bt, m):
    keys = W.byte_keys(80_000, 32, seed=1010 + m, prefix_bytes=2)
    vals = W.rank_values(keys.shape[0], 64)
    tree = bt.BTree(keys, vals, m)
    bt.bt_paper_layout_build(tree.handle)
    o = OracleBytesTree(keys, vals, m)
    q = W.make_byte_queries(keys, 30_001, 0.7, seed=1011)
    pv, pf = _run(bt, tree, q, q.shape[0])
    ov, of, _, _ = o.search(q)
    assert np.array_equal(pv, ov) and np.array_equal(pf, of)


@pytest.mark.parametrize("n", [1, 7, 8, 64, 65, 4096])
def test_small_trees(bt, n):
    keys = W.uniform_keys(n, 32, seed=1020 + n)
    vals = W.rank_values(n, 32)
    tree = bt.BTree(keys, vals, 8)
    bt.bt_paper_layout_build(tree.handle)
    o = OracleTree(keys, vals, 8, val_bits=32)
    q = W.make_queries(keys, 1000, 0.5, seed=1021, width_bits=32)
    pv, pf = _run(bt, tree, q, q.size)
    ov, of, _, _ = o.search(q)
    assert np.array_equal(pv.astype(np.uint64), ov) and np.array_equal(pf, of)


def test_search_without_the_layout_is_refused(bt):
    keys = W.uniform_keys(1000, 64, seed=1030)
    tree = bt.BTree(keys, W.rank_values(1000, 64), 16)
    q = W.make_queries(keys, 100, 0.5, seed=1031, width_bits=64)
    with pytest.raises(bt.BTreeError):
        _run(bt, tree, q, q.size)
