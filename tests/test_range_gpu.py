"""Range-partitioned trees on one GPU (bt_range_*): P subtrees over
contiguous key ranges, queries routed to their part and results back in
input order -- bit-exact against the oracle over the whole key set."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import OracleTree
from paper_2604_21117_gb300 import workloads as W

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


def _range_search(bt, r, q, val_bits=64):
    import torch
    nq = q.size
    dq = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    dt = torch.uint64 if val_bits == 64 else torch.uint32  # the tree's value width
    v = torch.zeros(max(nq, 1), dtype=dt, device="cuda")
    f = torch.full((max(nq, 1),), 9, dtype=torch.uint8, device="cuda")
    nb = bt.bt_range_workspace_bytes(r, nq)
    ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
    bt.bt_range_search(r, dq, nq, v, f, ws, nb)
    torch.cuda.synchronize()
    return v.cpu().numpy()[:nq].astype(np.uint64), f.cpu().numpy()[:nq]


@pytest.mark.parametrize("parts", [1, 2, 4, 7])
@pytest.mark.parametrize("kw,m", [(64, 32), (32, 16)])
def test_range_search_matches_oracle(bt, parts, kw, m):
    keys = W.uniform_keys(300_000, kw, seed=700 + parts + kw)
    vals = W.rank_values(keys.size, 64)
    r = bt.bt_range_build(keys, vals, m, parts)
    o = OracleTree(keys, vals, m)
    nparts, split, nkeys = bt.bt_range_info(r)
    assert nparts == parts and int(nkeys.sum()) == keys.size
    bounds = np.cumsum(nkeys)
    assert np.array_equal(split, keys[bounds[:-1] - 1].astype(np.uint64))  # each part's largest key
    for nq, zipf in ((1, None), (1000, None), (40_007, 1.1), (100_003, None)):
        q = W.make_queries(keys, nq, 0.8, seed=710 + nq, width_bits=kw, zipf_s=zipf)
        q[:2] = [0, np.iinfo(q.dtype).max][: min(2, nq)] if nq >= 2 else q[:2]
        gv, gf = _range_search(bt, r, q)
        ov, of, _, _ = o.search(q)
        assert np.array_equal(gv, ov) and np.array_equal(gf, of), (nq, zipf)
    bt.bt_range_free(r)


def test_range_all_queries_in_one_part_and_parts_of_one_key(bt):
    keys = W.uniform_keys(64, 64, seed=720)
    vals = W.rank_values(keys.size, 64)
    r = bt.bt_range_build(keys, vals, 8, 64)  # 64 parts of one key each
    o = OracleTree(keys, vals, 8)
    q = np.concatenate([keys, keys + np.uint64(1), np.full(5000, keys[10], np.uint64)])
    gv, gf = _range_search(bt, r, q)
    ov, of, _, _ = o.search(q)
    assert np.array_equal(gv, ov) and np.array_equal(gf, of)
    bt.bt_range_free(r)


def test_range_build_checks(bt):
    keys = W.uniform_keys(100, 64, seed=721)
    vals = W.rank_values(keys.size, 64)
    for parts in (0, 65, 101):
        with pytest.raises(bt.BTreeError):
            bt.bt_range_build(keys, vals, 16, parts)
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_range_build(keys[::-1].copy(), vals, 16, 2)
    assert e.value.code in ("BT_ERR_UNSORTED",)


def test_range_search_refuses_misaligned_arrays(bt):
    """A query or value array that is not aligned to its element size is
    refused on the host (BT_ERR_ARG), before any launch."""
    import torch
    keys = W.uniform_keys(10_000, 64, seed=730)
    r = bt.bt_range_build(keys, W.rank_values(keys.size, 64), 16, 4)
    nq = 1000
    qbuf = torch.zeros((nq + 1) * 8, dtype=torch.uint8, device="cuda")
    vbuf = torch.zeros((nq + 1) * 8, dtype=torch.uint8, device="cuda")
    f = torch.zeros(nq, dtype=torch.uint8, device="cuda")
    nb = bt.bt_range_workspace_bytes(r, nq)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    for q, v in ((qbuf.data_ptr() + 4, vbuf.data_ptr()), (qbuf.data_ptr(), vbuf.data_ptr() + 4)):
        with pytest.raises(bt.BTreeError) as e:
            bt.bt_range_search(r, q, nq, v, f, ws, nb)
        assert e.value.code == "BT_ERR_ARG"
    bt.bt_range_search(r, qbuf.data_ptr(), nq, vbuf.data_ptr(), f, ws, nb)
    torch.cuda.synchronize()
    bt.bt_range_free(r)
