"""GPU tests of multi-tree batching (one launch over a work list of batches
addressed to several trees), launch tuning and the autotuner: every result
bit-exact against the oracle of the batch's tree."""
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


def _forest_case(bt, sizes, fanouts, nbatches, seed, kw=64, vw=64):
    import torch
    trees, oracles, keysets = [], [], []
    for i, (n, m) in enumerate(zip(sizes, fanouts)):
        keys = W.uniform_keys(n, kw, seed=seed + i) if n else np.empty(0, W.key_dtype(kw))
        vals = W.rank_values(n, vw)
        trees.append(bt.BTree(keys, vals, m))
        oracles.append(OracleTree(keys, vals, m, val_bits=vw))
        keysets.append(keys)
    g = W.rng(seed)
    counts = W.log_uniform_batch_sizes(nbatches, seed=seed + 100)
    counts[::17] = 0  # some empty batches
    tids = g.integers(0, len(trees), size=nbatches)
    desc = np.zeros(nbatches, bt.BATCH_DESC_DTYPE)
    qs, off = [], 0
    for b in range(nbatches):
        c = int(counts[b])
        q = W.make_queries(keysets[tids[b]], c, 0.8, seed=seed + 1000 + b, width_bits=kw, zipf_s=0.9) if c else \
            np.empty(0, W.key_dtype(kw))
        qs.append(q)
        desc[b] = (tids[b], c, off)
        off += c
    allq = np.concatenate(qs) if off else np.empty(0, W.key_dtype(kw))
    return trees, oracles, desc, qs, allq, torch.from_numpy(desc.view(np.uint8)).cuda()


def _check_forest(bt, oracles, desc, qs, v, f):
    vv, ff = v.cpu().numpy().astype(np.uint64), f.cpu().numpy()
    for b in range(desc.size):
        c, off = int(desc[b]["count"]), int(desc[b]["offset"])
        if c == 0:
            continue
        ov, of, _, _ = oracles[int(desc[b]["tree"])].search(qs[b])
        assert np.array_equal(vv[off:off + c], ov), b
        assert np.array_equal(ff[off:off + c], of), b


@pytest.mark.parametrize("warps", [0, 4, 16])
def test_forest_matches_oracles(bt, warps):
    import torch
    trees, oracles, desc, qs, allq, d_desc = _forest_case(
        bt, [1000, 100_000, 300_000, 7, 0], [8, 16, 64, 32, 32], 500, seed=61)
    forest = bt.bt_forest_create(trees)
    nb = desc.size
    v = torch.empty(allq.size, dtype=torch.uint64, device="cuda")
    f = torch.empty(allq.size, dtype=torch.uint8, device="cuda")
    wsb = bt.bt_forest_workspace_bytes(nb)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    bt.bt_forest_search(forest, d_desc, nb, torch.from_numpy(allq).cuda(), v, f, ws, wsb, warps)
    _check_forest(bt, oracles, desc, qs, v, f)
    bt.bt_forest_free(forest)


def test_forest_search_replays_from_a_cuda_graph(bt):
    import torch
    trees, oracles, desc, qs, allq, d_desc = _forest_case(bt, [5000, 200_000], [16, 32], 300, seed=62)
    forest = bt.bt_forest_create(trees)
    nb = desc.size
    dq = torch.from_numpy(allq).cuda()
    v = torch.empty(allq.size, dtype=torch.uint64, device="cuda")
    f = torch.empty(allq.size, dtype=torch.uint8, device="cuda")
    wsb = bt.bt_forest_workspace_bytes(nb)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bt.bt_forest_search(forest, d_desc, nb, dq, v, f, ws, wsb, 8, s)  # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bt.bt_forest_search(forest, d_desc, nb, dq, v, f, ws, wsb, 8, torch.cuda.current_stream())
    for _ in range(2):
        v.fill_(0)
        f.fill_(9)
        g.replay()
        torch.cuda.synchronize()
        _check_forest(bt, oracles, desc, qs, v, f)
    bt.bt_forest_free(forest)


@pytest.mark.parametrize("warps,pin,staging,lq", [(4, 0, 0, 1), (16, 0, 0, 1), (4, 49152, 0, 1), (16, 49152, 0, 1),
                                                  (8, 16384, 0, 1), (4, 0, 1, 1), (16, 49152, 1, 1), (8, 16384, 1, 1),
                                                  (8, 16384, 0, 2), (4, 0, 0, 2), (16, 49152, 0, 2),
                                                  (4, 0, 2, 1), (16, 49152, 2, 1), (8, 16384, 2, 1)])
def test_launch_settings_do_not_change_results(bt, warps, pin, staging, lq):
    keys = W.uniform_keys(500_000, 64, seed=63)
    vals = W.rank_values(keys.size, 64)
    tree = bt.BTree(keys, vals, 16)
    o = OracleTree(keys, vals, 16)
    bt.bt_tree_set_launch(tree.handle, warps, pin)
    bt.bt_tree_set_staging(tree.handle, staging)
    bt.bt_tree_set_lane_queries(tree.handle, lq)
    q = W.make_queries(keys, 70_001, 0.9, seed=64, width_bits=64)
    import torch
    v, f = tree.search(torch.from_numpy(q).cuda())
    bt.bt_check_timeouts()
    ov, of, _, _ = o.search(q)
    assert np.array_equal(v.cpu().numpy(), ov) and np.array_equal(f.cpu().numpy(), of)


@pytest.mark.parametrize("fanout,key_bits", [(8, 32), (8, 64), (32, 32), (64, 64), (64, 32)])
def test_bulk_staging_every_block_size(bt, fanout, key_bits):
    """Bulk copies of every node-block size (8 slots of 4 bytes up to 64 of 8)."""
    import torch
    keys = W.uniform_keys(300_000, key_bits, seed=68 + fanout)
    vals = W.rank_values(keys.size, 32)
    tree = bt.BTree(keys, vals, fanout)
    bt.bt_tree_set_staging(tree.handle, bt.BT_STAGE_BULK)
    o = OracleTree(keys, vals, fanout, val_bits=32)
    q = W.make_queries(keys, 40_003, 0.7, seed=69, width_bits=key_bits)
    for sb in (-1, 0):
        v, f = tree.search(torch.from_numpy(q).cuda(), sort_bits=sb)
        bt.bt_check_timeouts()
        ov, of, _, _ = o.search(q)
        assert np.array_equal(v.cpu().numpy(), ov) and np.array_equal(f.cpu().numpy(), of)


def test_autotune_returns_a_correct_tree(bt):
    import torch
    keys = W.uniform_keys(200_000, 64, seed=65)
    vals = W.rank_values(keys.size, 64)
    sample = W.make_queries(keys, 1024, 0.8, seed=66, width_bits=64, zipf_s=0.9)
    h, best = bt.bt_autotune(keys, vals, torch.from_numpy(sample).cuda(), sample.size)
    tree = bt.BTree(None, None, handle=h)
    assert best.fanout in (8, 16, 32, 64) and best.warps_per_block in (4, 8, 16)
    assert best.pin_bytes in (0, 16384, 49152) and best.staging in (0, 1, 2) and best.lane_queries in (1, 2)
    assert best.inner_staged in (0, 1)
    assert best.us_per_batch > 0
    assert tree.fanout == best.fanout
    # 1024 queries are under one chunk per SM: the pipelined designs keep the default blocks
    if best.staging == bt.BT_STAGE_PIPELINED:
        assert best.warps_per_block == 8
    o = OracleTree(keys, vals, best.fanout)
    q = W.make_queries(keys, 30_000, 0.8, seed=67, width_bits=64)
    v, f = tree.search(torch.from_numpy(q).cuda())
    ov, of, _, _ = o.search(q)
    assert np.array_equal(v.cpu().numpy(), ov) and np.array_equal(f.cpu().numpy(), of)


@pytest.mark.parametrize("m,kw,vw", [(8, 32, 32), (16, 64, 64), (32, 64, 32), (64, 32, 64)])
@pytest.mark.parametrize("nq", [1, 33, 63, 64, 65, 20_011])
def test_two_queries_per_lane(bt, m, kw, vw, nq):
    """64-query chunks: every fanout and width, ragged sizes, sorted and
    unsorted order, narrow and wide node ranges per warp."""
    import torch
    keys = W.uniform_keys(200_000, kw, seed=71 + m)
    vals = W.rank_values(keys.size, vw)
    tree = bt.BTree(keys, vals, m)
    bt.bt_tree_set_lane_queries(tree.handle, 2)
    o = OracleTree(keys, vals, m, val_bits=vw)
    q = W.make_queries(keys, nq, 0.8, seed=72 + nq, width_bits=kw, zipf_s=1.1)
    ov, of, _, _ = o.search(q)
    for sb in (-1, 0, 6):
        v, f = tree.search(torch.from_numpy(q).cuda(), sort_bits=sb)
        assert np.array_equal(v.cpu().numpy().astype(np.uint64), ov) and np.array_equal(f.cpu().numpy(), of), sb


def _forest_outputs(bt, forest, desc, allq, d_desc, warps=0, vw=64):
    import torch
    nb = desc.size
    v = torch.zeros(max(1, allq.size), dtype=torch.uint64 if vw == 64 else torch.uint32, device="cuda")
    f = torch.full((max(1, allq.size),), 9, dtype=torch.uint8, device="cuda")
    wsb = bt.bt_forest_workspace_bytes(nb)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    bt.bt_forest_search(forest, d_desc, nb, torch.from_numpy(allq).cuda(), v, f, ws, wsb, warps, nq=allq.size)
    return v, f


@pytest.mark.parametrize("warps,pin,lq,staging", [(8, 32768, 0, 0), (4, 0, 1, 1), (16, 98304, 2, 1), (8, 16384, 1, 2),
                                                  (4, 98304, 2, 2), (12, 49152, 0, 2), (1, 0, 2, 0)])
def test_forest_settings_do_not_change_results(bt, warps, pin, lq, staging):
    """Each tree keeps its own tuned design (two queries per lane, staged
    levels, pinned levels) unless the forest overrides it; every combination
    gives the oracle's results."""
    trees, oracles, desc, qs, allq, d_desc = _forest_case(
        bt, [3000, 150_000, 400_000, 1, 0], [16, 32, 64, 8, 32], 400, seed=91)
    bt.bt_tree_set_lane_queries(trees[0].handle, 2)
    bt.bt_tree_set_staging(trees[1].handle, bt.BT_STAGE_CP_ASYNC)
    bt.bt_tree_set_launch(trees[2].handle, 8, 49152)
    bt.bt_tree_set_launch(trees[0].handle, 8, 16384)
    forest = bt.bt_forest_create(trees)
    bt.bt_forest_set_launch(forest, warps, pin, lq, staging)
    got = bt.bt_forest_get_launch(forest)
    assert (got.warps_per_block, got.pin_budget, got.lane_queries, got.staging) == (warps, pin, lq, staging)
    assert got.pin_applied <= pin
    v, f = _forest_outputs(bt, forest, desc, allq, d_desc)
    _check_forest(bt, oracles, desc, qs, v, f)
    assert bt.bt_forest_bad_batches() == 0
    bt.bt_forest_free(forest)


def test_forest_pins_tuned_levels_within_its_budget(bt):
    trees, oracles, desc, qs, allq, d_desc = _forest_case(bt, [300_000, 300_000, 300_000], [8, 16, 32], 60, seed=92)
    for t in trees:
        bt.bt_tree_set_launch(t.handle, 8, 49152)
    forest = bt.bt_forest_create(trees)
    for budget in (98304, 49152, 16384, 0):
        bt.bt_forest_set_launch(forest, 8, budget, 0, 0)
        got = bt.bt_forest_get_launch(forest)
        assert got.pin_applied <= budget
        if budget == 98304:
            assert got.pin_applied > 16384  # the three trees' tuned pins, trimmed to fit
        v, f = _forest_outputs(bt, forest, desc, allq, d_desc)
        _check_forest(bt, oracles, desc, qs, v, f)
    bt.bt_forest_free(forest)


@pytest.mark.parametrize("lq", [0, 2])
def test_learned_forest_matches_oracles(bt, lq):
    """Trees with a PL model, an MLP model and none in one forest: lanes whose
    window proves their leaf skip the inner levels, the others walk them."""
    import torch  # noqa: F401
    trees, oracles, desc, qs, allq, d_desc = _forest_case(bt, [50_000, 400_000, 2000], [32, 16, 8], 300, seed=93)
    models = [bt.bt_model_train(trees[0].handle, bt.BT_MODEL_PL, segments=64),
              bt.bt_model_train(trees[1].handle, bt.BT_MODEL_MLP, h_init=W.mlp_init_params(W.SEED_BASE + 5),
                                steps=200, batch=4096, lr=2e-3, seed=94),
              None]
    forest = bt.bt_forest_create_learned(trees, models)
    bt.bt_forest_set_launch(forest, 8, 16384, lq, 2)  # staging is ignored for trees with a model
    v, f = _forest_outputs(bt, forest, desc, allq, d_desc)
    _check_forest(bt, oracles, desc, qs, v, f)
    bt.bt_forest_free(forest)
    # a forest of PL models only
    pl = [bt.bt_model_train(trees[i].handle, bt.BT_MODEL_PL, segments=256) for i in range(3)]
    forest = bt.bt_forest_create_learned(trees, pl)
    v, f = _forest_outputs(bt, forest, desc, allq, d_desc)
    _check_forest(bt, oracles, desc, qs, v, f)
    bt.bt_forest_free(forest)
    for m in models[:2] + pl:
        bt.bt_model_free(m)


def test_learned_forest_rejects_a_model_of_another_tree(bt):
    trees, _, _, _, _, _ = _forest_case(bt, [50_000, 400_000], [32, 16], 4, seed=95)
    m = bt.bt_model_train(trees[0].handle, bt.BT_MODEL_PL, segments=64)
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_forest_create_learned(trees, [None, m])
    assert e.value.code == "BT_ERR_ARG"
    bt.bt_model_free(m)


def test_forest_autotune_keeps_the_fastest_correct_settings(bt):
    import torch
    trees, oracles, desc, qs, allq, d_desc = _forest_case(bt, [1000, 100_000, 500_000], [8, 32, 16], 800, seed=96)
    forest = bt.bt_forest_create(trees)
    nb = desc.size
    dq = torch.from_numpy(allq).cuda()
    v = torch.empty(allq.size, dtype=torch.uint64, device="cuda")
    f = torch.empty(allq.size, dtype=torch.uint8, device="cuda")
    wsb = bt.bt_forest_workspace_bytes(nb)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    best = bt.bt_forest_autotune(forest, d_desc, nb, dq, v, f, ws, wsb)
    assert best.warps_per_block in (4, 8, 16) and best.pin_budget in (0, 16384, 49152, 98304)
    assert best.lane_queries in (0, 1, 2) and best.staging in (0, 1, 2) and best.us > 0
    got = bt.bt_forest_get_launch(forest)
    assert (got.warps_per_block, got.pin_budget, got.lane_queries, got.staging) == \
        (best.warps_per_block, best.pin_budget, best.lane_queries, best.staging)
    v.zero_()
    f.fill_(9)
    bt.bt_forest_search(forest, d_desc, nb, dq, v, f, ws, wsb)
    _check_forest(bt, oracles, desc, qs, v, f)
    bt.bt_forest_free(forest)


def test_bad_work_list_entries_are_skipped_and_counted(bt):
    """Entries naming a tree outside the forest or queries beyond the arrays
    write nothing and are counted; the others are served."""
    import torch
    trees, oracles, desc, qs, allq, _ = _forest_case(bt, [5000, 50_000], [16, 32], 40, seed=97)
    forest = bt.bt_forest_create(trees)
    bt.bt_forest_bad_batches()  # clear
    bad = desc.copy()
    bad[3]["tree"] = 7                     # no such tree
    bad[5]["offset"] = allq.size + 1000    # beyond the arrays
    bad[6]["count"] = allq.size + 1        # runs past the end
    v, f = _forest_outputs(bt, forest, bad, allq, torch.from_numpy(bad.view(np.uint8)).cuda())
    assert bt.bt_forest_bad_batches() == 3
    ff = f.cpu().numpy()
    for b in (3, 5, 6):  # their own result ranges stay untouched
        c, off = int(desc[b]["count"]), int(desc[b]["offset"])
        assert (ff[off:off + c] == 9).all(), b
    good = np.ones(desc.size, bool)
    good[[3, 5, 6]] = False
    keep = desc.copy()
    keep["count"][~good] = 0
    _check_forest(bt, oracles, keep, qs, v, f)
    bt.bt_forest_free(forest)


@pytest.mark.parametrize("kw,vw", [(32, 32), (32, 64), (64, 32)])
@pytest.mark.parametrize("learned", [False, True])
def test_forest_every_key_and_value_width(bt, kw, vw, learned):
    """The four kernel instantiations (key x value width), plain and learned,
    at two queries per lane and at one."""
    trees, oracles, desc, qs, allq, d_desc = _forest_case(bt, [3000, 200_000, 40], [16, 32, 8], 300, seed=98,
                                                          kw=kw, vw=vw)
    models = [bt.bt_model_train(t.handle, bt.BT_MODEL_PL, segments=64) for t in trees] if learned else None
    forest = bt.bt_forest_create_learned(trees, models) if learned else bt.bt_forest_create(trees)
    for lq in (1, 2):
        bt.bt_forest_set_launch(forest, 8, 16384, lq, 0)
        v, f = _forest_outputs(bt, forest, desc, allq, d_desc, vw=vw)
        _check_forest(bt, oracles, desc, qs, v, f)
    bt.bt_forest_free(forest)
    for m in models or ():
        bt.bt_model_free(m)


def test_misaligned_arrays_are_refused(bt):
    """A work list, query array or value array that is not aligned to its
    element size is refused on the host (BT_ERR_ARG), before any launch."""
    import torch
    trees, _, desc, _, allq, d_desc = _forest_case(bt, [5000], [16], 20, seed=3100)
    forest = bt.bt_forest_create(trees)
    n = allq.size
    # byte buffers; every misaligned pointer still has room for the whole
    # array after it
    qbuf = torch.zeros((n + 1) * 8, dtype=torch.uint8, device="cuda")
    qbuf[:n * 8].copy_(torch.from_numpy(allq.view(np.uint8)))
    vbuf = torch.zeros((n + 1) * 8, dtype=torch.uint8, device="cuda")
    dbuf = torch.zeros(d_desc.numel() + 16, dtype=torch.uint8, device="cuda")
    dbuf[:d_desc.numel()].copy_(d_desc)
    f = torch.zeros(n, dtype=torch.uint8, device="cuda")
    wsb = bt.bt_forest_workspace_bytes(desc.size)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    dp, qp, vp = dbuf.data_ptr(), qbuf.data_ptr(), vbuf.data_ptr()
    for dd, q, v in ((dp, qp + 4, vp), (dp, qp, vp + 4), (dp + 4, qp, vp)):
        with pytest.raises(bt.BTreeError) as e:
            bt.bt_forest_search(forest, dd, desc.size, q, v, f, ws, wsb, nq=n)
        assert e.value.code == "BT_ERR_ARG"
    bt.bt_forest_search(forest, dp, desc.size, qp, vp, f, ws, wsb, nq=n)
    torch.cuda.synchronize()
    bt.bt_forest_free(forest)
    for t in trees:
        t.close()
