"""The no-allocation entry point (bt_search_batch_noalloc), for callers that
cannot allocate device memory, against the workspace entry point.

It lives in a file of its own that pytest collects last, so a run that stops
at the first failure has run every other test first."""
from __future__ import annotations

import numpy as np
import pytest

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


def test_noalloc_matches_workspace_entry_point_on_two_calls(bt):
    import torch
    keys = W.uniform_keys(300_000, 64, seed=31)
    vals = W.rank_values(keys.size, 64)
    tree = bt.BTree(keys, vals, 32)
    # the largest batch then a ragged one: the second call runs on scratch
    # that still holds the first call's contents
    for nq, seed in ((bt.BT_NOALLOC_MAX_QUERIES, 32), (40_001, 33)):
        q = torch.from_numpy(W.make_queries(keys, nq, 0.9, seed=seed, width_bits=64, zipf_s=1.1)).cuda()
        v_ref, f_ref = tree.alloc_outputs(nq)
        ws, nb = tree.alloc_workspace(nq)
        bt.bt_search_batch(tree.handle, q, nq, v_ref, f_ref, ws, nb)
        v, f = tree.alloc_outputs(nq)
        v.fill_(0)
        f.fill_(7)
        bt.bt_search_batch_noalloc(tree.handle, q, nq, v, f)
        torch.cuda.synchronize()
        assert np.array_equal(v.cpu().numpy(), v_ref.cpu().numpy())
        assert np.array_equal(f.cpu().numpy(), f_ref.cpu().numpy())
    tree.close()


def test_noalloc_32_byte_keys_at_its_limit_against_the_oracle(bt):
    """The largest no-allocation batch of the paper's 32-byte keys (the
    workspace it asks for, sized for a partition's pairs, keys and
    positions, fits the scratch), every result against the byte-key
    oracle."""
    import torch
    from oracle.bytes_keys import OracleBytesTree
    keys = W.byte_keys(200_000, 32, seed=35)
    vals = W.rank_values(keys.shape[0], 64)
    tree = bt.BTree(keys, vals, 16)
    o = OracleBytesTree(keys, vals, 16)
    nq = bt.BT_NOALLOC_MAX_QUERIES
    qh = W.make_byte_queries(keys, nq, 0.9, seed=36)
    v, f = tree.alloc_outputs(nq)
    bt.bt_search_batch_noalloc(tree.handle, torch.from_numpy(qh).cuda(), nq, v, f)
    torch.cuda.synchronize()
    ov, of, _, _ = o.search(qh)
    assert np.array_equal(v.cpu().numpy(), ov) and np.array_equal(f.cpu().numpy(), of)
    o.close()
    tree.close()


def test_noalloc_rejects_batches_above_its_limit(bt):
    import torch
    keys = W.uniform_keys(1000, 64, seed=34)
    tree = bt.BTree(keys, W.rank_values(keys.size, 64), 16)
    nq = bt.BT_NOALLOC_MAX_QUERIES + 1
    q = torch.zeros(nq, dtype=torch.uint64, device="cuda")
    v, f = tree.alloc_outputs(nq)
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_search_batch_noalloc(tree.handle, q, nq, v, f)
    assert e.value.code == "BT_ERR_ARG"
    tree.close()
