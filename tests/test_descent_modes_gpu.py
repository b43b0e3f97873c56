"""The descent's selectable designs give the oracle's results, bit-exact:
the pipelined descent (leaf blocks staged by bulk copies overlapped with
the next chunk) with inner levels read through L1 or staged in shared
memory, leaf ranks by binary search or by warp ballot + popc, with and
without the L2 persistence window; the synchronous descents; and the
bounded wait of the bulk-copy staging, made to give up on purpose."""
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _same(tree, o, q, sort_bits=-1):
    v, f = tree.search(_dev(q), sort_bits=sort_bits)
    ov, of, _, _ = o.search(q)
    gv = v.cpu().numpy().astype(np.uint64)
    gf = f.cpu().numpy()
    bad = np.nonzero((gv != ov) | (gf != of))[0]
    assert bad.size == 0, f"{bad.size} mismatches, first at {int(bad[0])}"


@pytest.mark.parametrize("inner,ballot", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("m", [8, 16, 32, 64])
@pytest.mark.parametrize("kw,vw", [(32, 32), (64, 64), (64, 32)])
def test_pipelined_options(bt, inner, ballot, m, kw, vw):
    """Every fanout and width; sorted (12 bits) and unsorted batches (the
    automatic choice on this small tree, and forced); a ragged size,
    so the last chunk has tail lanes."""
    keys = W.uniform_keys(90_000 + m, kw, seed=500 + m + kw)
    vals = W.rank_values(keys.size, vw)
    tree = bt.BTree(keys, vals, m)
    bt.bt_tree_set_staging(tree.handle, bt.BT_STAGE_PIPELINED)
    bt.bt_tree_set_descent(tree.handle, inner, ballot)
    o = OracleTree(keys, vals, m, val_bits=vw)
    q = W.make_queries(keys, 40_011, 0.8, seed=600 + m, width_bits=kw, zipf_s=1.1)
    for sb in (-1, 0, 12):
        _same(tree, o, q, sb)
    bt.bt_check_timeouts()


@pytest.mark.parametrize("staging", [0, 1, 2])
@pytest.mark.parametrize("nq", [1, 31, 33, 1000, 16_384, 100_003])
def test_staging_modes_and_sizes(bt, staging, nq):
    keys = W.uniform_keys(400_000, 64, seed=610)
    vals = W.rank_values(keys.size, 64)
    tree = bt.BTree(keys, vals, 32)
    bt.bt_tree_set_staging(tree.handle, staging)
    o = OracleTree(keys, vals, 32)
    q = W.make_queries(keys, nq, 0.9, seed=611 + nq, width_bits=64)
    _same(tree, o, q)
    if nq >= 1000:
        _same(tree, o, q, 16)
    bt.bt_check_timeouts()


@pytest.mark.parametrize("warps,pin", [(4, 0), (8, 16384), (16, 49152)])
def test_pipelined_launch_settings(bt, warps, pin):
    keys = W.uniform_keys(700_000, 64, seed=620)
    vals = W.rank_values(keys.size, 64)
    tree = bt.BTree(keys, vals, 16)
    bt.bt_tree_set_launch(tree.handle, warps, pin)
    o = OracleTree(keys, vals, 16)
    _same(tree, o, W.make_queries(keys, 70_001, 0.9, seed=621, width_bits=64))


@pytest.mark.parametrize("m", [16, 32])
def test_l2_window_keeps_results(bt, m):
    keys = W.uniform_keys(2_000_000, 64, seed=630 + m)
    vals = W.rank_values(keys.size, 64)
    tree = bt.BTree(keys, vals, m)
    o = OracleTree(keys, vals, m)
    q = W.make_queries(keys, 200_000, 0.9, seed=631, width_bits=64)
    bt.bt_tree_set_l2_window(tree.handle, 64 << 20)
    _same(tree, o, q)
    bt.bt_tree_set_l2_window(tree.handle, 0)
    _same(tree, o, q)


@pytest.mark.parametrize("staging", [1, 2])
def test_bounded_wait_gives_up_and_is_reported(bt, staging):
    """With the first wait's poll limit at 0 every bulk-copy wait gives up at
    once: the warp counts it, waits (full limit) for its copies, and stops.
    bt_check_timeouts reports it; with the limit restored the next search is
    bit-exact and nothing more is reported."""
    import torch
    keys = W.uniform_keys(300_000, 64, seed=640)
    vals = W.rank_values(keys.size, 64)
    tree = bt.BTree(keys, vals, 32)
    bt.bt_tree_set_staging(tree.handle, staging)
    o = OracleTree(keys, vals, 32)
    q = W.make_queries(keys, 50_000, 0.9, seed=641, width_bits=64)
    bt.bt_check_timeouts()  # clear anything earlier
    try:
        bt.bt_debug_set_wait_polls(0)
        tree.search(_dev(q))
        torch.cuda.synchronize()
    finally:
        bt.bt_debug_set_wait_polls(bt.BT_DEFAULT_WAIT_POLLS)
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_check_timeouts()
    assert e.value.code == "BT_ERR_TIMEOUT"
    _same(tree, o, q)
    bt.bt_check_timeouts()  # nothing new


@pytest.mark.parametrize("caps", [(3, 1), (2, 1), (1, 1)])
def test_two_streams_with_corun_caps(bt, caps):
    """Steps alternating between two streams, each with its own workspace and
    outputs, with the descent and partition capped so that they run side by
    side: every step's results equal the oracle's."""
    import torch
    n, m, B = 300_000, 32, 70_001
    keys = W.uniform_keys(n, 64, seed=131)
    vals = W.rank_values(n, 64)
    tree = bt.BTree(keys, vals, m)
    o = OracleTree(keys, vals, m)
    bt.bt_tree_set_corun(tree.handle, *caps)
    qs = [W.make_queries(keys, B, 0.9, seed=132 + i, width_bits=64) for i in range(4)]
    want = [o.search(q)[:2] for q in qs]
    nb = tree.workspace_bytes(B)
    bufs = [(torch.empty(nb, dtype=torch.uint8, device="cuda"), torch.empty(B, dtype=torch.uint64, device="cuda"),
             torch.empty(B, dtype=torch.uint8, device="cuda")) for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    dq = [torch.from_numpy(q).cuda() for q in qs]
    torch.cuda.synchronize()
    got = []
    for i in range(8):
        ws, v, f = bufs[i % 2]
        bt.bt_search_batch(tree.handle, dq[i % 4], B, v, f, ws, nb, streams[i % 2])
        if i >= 6:  # the last two steps, one on each stream
            streams[i % 2].synchronize()
            got.append((i % 4, v.cpu().numpy().copy(), f.cpu().numpy().copy()))
    torch.cuda.synchronize()
    bt.bt_check_timeouts()
    for qi, v, f in got:
        assert np.array_equal(v, want[qi][0]) and np.array_equal(f, want[qi][1])
    bt.bt_tree_set_corun(tree.handle, 0, 0)
    tree.close()


@pytest.mark.parametrize("kind", ["bytes32", "learned"])
def test_two_streams_with_corun_caps_other_paths(bt, kind):
    """The same two-stream pattern over 32-byte keys and over the learned
    search: results equal the oracle's."""
    import torch
    B = 50_003
    if kind == "bytes32":
        from oracle.bytes_keys import OracleBytesTree
        keys = W.byte_keys(100_000, 32, seed=141)
        vals = W.rank_values(keys.shape[0], 64)
        tree = bt.BTree(keys, vals, 16)
        o = OracleBytesTree(keys, vals, 16)
        qs = [W.make_byte_queries(keys, B, 0.9, seed=142 + i) for i in range(2)]
        mdl = None
    else:
        keys = W.lognormal_mixture_keys(300_000, seed=143)
        vals = W.rank_values(keys.size, 64)
        tree = bt.BTree(keys, vals, 32)
        o = OracleTree(keys, vals, 32)
        qs = [W.make_queries(keys, B, 0.9, seed=144 + i, width_bits=64) for i in range(2)]
        mdl = bt.bt_model_train(tree.handle, bt.BT_MODEL_PL, segments=256)
    bt.bt_tree_set_corun(tree.handle, 0, 1)
    want = [o.search(q)[:2] for q in qs]
    nb = tree.workspace_bytes(B)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for i in range(2):
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        v, f = tree.alloc_outputs(B)
        dq = torch.from_numpy(qs[i]).cuda()
        torch.cuda.synchronize()
        outs.append((ws, v, f, dq))
    for rep in range(3):
        for i in range(2):
            ws, v, f, dq = outs[i]
            if mdl is None:
                bt.bt_search_batch(tree.handle, dq, B, v, f, ws, nb, streams[i])
            else:
                bt.bt_learned_search_batch(tree.handle, mdl, dq, B, v, f, ws, nb, streams[i])
    torch.cuda.synchronize()
    bt.bt_check_timeouts()
    for i in range(2):
        _, v, f, _ = outs[i]
        assert np.array_equal(v.cpu().numpy().astype(np.uint64), want[i][0])
        assert np.array_equal(f.cpu().numpy(), want[i][1])
    if mdl is not None:
        bt.bt_model_free(mdl)
    o.close()
    tree.close()
