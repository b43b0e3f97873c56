"""GPU tests of the learned leaf predictor against its oracle, and bit-exact
search results with the model against the plain tree's oracle."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import OracleTree
from oracle import learned as LO
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


@pytest.mark.parametrize("dist", ["uniform", "lognormal"])
def test_pl_fit_matches_oracle_and_error_bound_is_exact(bt, dist):
    n, m, S = 300_000, 32, 256
    keys = W.uniform_keys(n, 64, seed=41) if dist == "uniform" else W.lognormal_mixture_keys(n, seed=41)
    vals = W.rank_values(n, 64)
    tree = bt.BTree(keys, vals, m)
    o = OracleTree(keys, vals, m)
    _, _, leaf, _ = o.search(keys)
    mdl = bt.bt_model_train(tree.handle, bt.BT_MODEL_PL, segments=S)
    b, inv_w, slope, icpt = bt.bt_model_copy_params(mdl)
    ob, oinv, oslope, oicpt = LO.pl_fit(keys, leaf, S)
    assert np.array_equal(b, ob) and np.array_equal(inv_w, oinv)
    assert np.allclose(slope, oslope, rtol=1e-5, atol=1e-3) and np.allclose(icpt, oicpt, rtol=1e-5, atol=1e-2)
    # the error bound the GPU computed equals the oracle's, using the GPU's parameters
    L = tree.level_nodes[-1]
    hat = LO.pl_predict(b, inv_w, slope, icpt, keys, L)
    info = bt.bt_model_get_info(mdl)
    assert info.max_err == LO.max_error(hat, leaf)
    assert np.array_equal(bt.bt_model_copy_err_bounds(mdl).astype(np.int64), LO.range_errors(hat, leaf, L))
    bt.bt_model_free(mdl)


def test_mlp_gradient_matches_oracle(bt):
    import torch
    g = W.rng(42)
    p = W.mlp_init_params(43)
    x = g.random(3000).astype(np.float32)
    t = g.random(3000).astype(np.float32)
    dg = torch.empty(bt.BT_MLP_PARAMS, dtype=torch.float32, device="cuda")
    dl = torch.empty(1, dtype=torch.float32, device="cuda")
    bt.bt_mlp_grad(_dev(p), _dev(x), _dev(t), x.size, dg, dl)
    torch.cuda.synchronize()
    want = LO.mlp_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    got = dg.cpu().numpy().astype(np.float64)
    scale = np.abs(want).max()
    assert np.allclose(got, want, rtol=2e-3, atol=2e-5 * scale)
    assert abs(float(dl.item()) - LO.mlp_loss(p, x, t)) < 1e-4 * max(1.0, LO.mlp_loss(p, x, t))


def test_mlp_training_lowers_the_loss(bt):
    keys = W.uniform_keys(100_000, 64, seed=44)
    tree = bt.BTree(keys, W.rank_values(keys.size, 64), 32)
    p0 = W.mlp_init_params(45)
    _, _, leaf, _ = OracleTree(keys, keys, 32).search(keys)
    L = tree.level_nodes[-1]
    x = LO.mlp_x(keys, *LO.mlp_stage1(keys))
    loss0 = LO.mlp_loss(p0, x, leaf / (L - 1))
    mdl = bt.bt_model_train(tree.handle, bt.BT_MODEL_MLP, h_init=p0, steps=300, batch=4096, lr=3e-3, seed=46)
    p1 = bt.bt_model_copy_params(mdl)
    loss1 = LO.mlp_loss(p1, x, leaf / (L - 1))
    assert loss1 < 0.2 * loss0
    info = bt.bt_model_get_info(mdl)
    assert info.max_err < L and np.isfinite(info.final_loss)
    bt.bt_model_free(mdl)


def test_mlp_rank_input_bounds_lognormal_keys(bt):
    """On keys from the lognormal mixture the MLP, fed the first stage's rank
    coordinate, learns the leaf to a small fraction of the leaves (an input
    scaled over the key range could not: the CDF rises within the first
    millionth of that range)."""
    keys = W.lognormal_mixture_keys(1 << 20, seed=49)
    tree = bt.BTree(keys, W.rank_values(keys.size, 64), 32)
    L = tree.level_nodes[-1]
    mdl = bt.bt_model_train(tree.handle, bt.BT_MODEL_MLP, h_init=W.mlp_init_params(50), steps=1000, batch=16384,
                            lr=2e-3, seed=51)
    info = bt.bt_model_get_info(mdl)
    assert info.max_err < L // 8, (info.max_err, L)
    o = OracleTree(keys, W.rank_values(keys.size, 64), 32)
    _learned_check(bt, tree, o, mdl, W.make_queries(keys, 50_000, 0.9, seed=52, width_bits=64))
    bt.bt_model_free(mdl)
    tree.close()


def _learned_check(bt, tree, o, mdl, q, stats=None):
    import torch
    nq = q.size
    v, f = tree.alloc_outputs(nq)
    ws, nb = tree.alloc_workspace(nq)
    bt.bt_learned_search_batch(tree.handle, mdl, _dev(q), nq, v, f, ws, nb)
    ov, of, _, _ = o.search(q)
    assert np.array_equal(v.cpu().numpy().astype(np.uint64), ov)
    assert np.array_equal(f.cpu().numpy(), of)
    if stats is not None:
        # the model path on the sorted batch, counting served / fallen-back warps
        dq = _dev(q)
        sq = torch.empty_like(dq)
        si = torch.empty(nq, dtype=torch.int32, device="cuda")
        bt.bt_sort_batch(tree.handle, dq, nq, 16, sq, si, ws, nb)
        v2, f2 = tree.alloc_outputs(nq)
        bt.bt_learned_descend_sorted(tree.handle, mdl, sq, si, nq, v2, f2, stats)
        assert np.array_equal(v2.cpu().numpy().astype(np.uint64), ov)
        assert np.array_equal(f2.cpu().numpy(), of)


@pytest.mark.parametrize("kind", ["pl", "mlp"])
@pytest.mark.parametrize("dist", ["uniform", "lognormal"])
def test_learned_search_is_bit_exact(bt, kind, dist):
    import torch
    n, m = 400_000, 32
    keys = W.uniform_keys(n, 64, seed=47) if dist == "uniform" else W.lognormal_mixture_keys(n, seed=47)
    vals = W.rank_values(n, 64)
    tree = bt.BTree(keys, vals, m)
    o = OracleTree(keys, vals, m)
    if kind == "pl":
        mdl = bt.bt_model_train(tree.handle, bt.BT_MODEL_PL, segments=256)
    else:
        mdl = bt.bt_model_train(tree.handle, bt.BT_MODEL_MLP, h_init=W.mlp_init_params(48), steps=200,
                                batch=8192, lr=3e-3, seed=49)
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    for nq, zipf in ((1, None), (33, None), (1024, None), (100_003, None), (50_000, 1.1)):
        q = W.make_queries(keys, nq, 0.9, seed=nq + 50, width_bits=64, zipf_s=zipf)
        _learned_check(bt, tree, o, mdl, q, stats)
    top = np.uint64(2**64 - 1)
    edge = np.array([0, keys[0], keys[0] - np.uint64(1), keys[-1], keys[-1] + np.uint64(1), top], np.uint64)
    _learned_check(bt, tree, o, mdl, edge)
    served, fell = (int(x) for x in stats.cpu().numpy())
    assert served + fell > 0
    if kind == "pl" and dist == "uniform":
        assert served > fell  # the model window serves most warps on uniform keys
    bt.bt_model_free(mdl)


@pytest.mark.parametrize("m", [8, 16, 64])
@pytest.mark.parametrize("n", [1, 5, 200, 5000])
def test_learned_small_trees_and_u32(bt, m, n):
    keys = W.uniform_keys(n, 32, seed=n + m)
    vals = W.rank_values(n, 32)
    tree = bt.BTree(keys, vals, m)
    o = OracleTree(keys, vals, m, val_bits=32)
    for kind in (bt.BT_MODEL_PL, bt.BT_MODEL_MLP):
        if kind == bt.BT_MODEL_PL:
            mdl = bt.bt_model_train(tree.handle, kind, segments=64)
        else:
            mdl = bt.bt_model_train(tree.handle, kind, h_init=W.mlp_init_params(n), steps=20, batch=256,
                                    lr=1e-2, seed=1)
        q = pins_queries(keys)
        _learned_check(bt, tree, o, mdl, q)
        bt.bt_model_free(mdl)


def pins_queries(keys):
    import pins
    return pins.probe_queries(keys, 32, W.rng(7), extra=300).astype(np.uint32)


def test_training_is_what_narrows_the_window(bt):
    """What the trained network gains over the untrained one on the same
    tree: the error window that bounds the leaf search shrinks by far, and
    the window (not the inner levels) then serves nearly every query."""
    import torch
    n, m = 400_000, 32
    keys = W.lognormal_mixture_keys(n, seed=57)
    vals = W.rank_values(n, 64)
    tree = bt.BTree(keys, vals, m)
    o = OracleTree(keys, vals, m)
    L = int(tree.level_nodes[-1])
    one = bt.bt_model_train(tree.handle, bt.BT_MODEL_MLP, h_init=W.mlp_init_params(58), steps=1, batch=16384,
                            lr=2e-3, seed=59)
    trained = bt.bt_model_train(tree.handle, bt.BT_MODEL_MLP, h_init=W.mlp_init_params(58), steps=1000,
                                batch=16384, lr=2e-3, seed=59)
    e1, e2 = bt.bt_model_get_info(one).max_err, bt.bt_model_get_info(trained).max_err
    r1 = bt.bt_model_copy_err_bounds(one).astype(np.float64)
    r2 = bt.bt_model_copy_err_bounds(trained).astype(np.float64)
    assert e2 * 8 < e1 and e2 < L // 8, (e1, e2, L)
    assert r2.mean() * 8 < r1.mean()  # the windows actually searched, per range of prediction
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    _learned_check(bt, tree, o, trained, W.make_queries(keys, 1 << 17, 0.9, seed=60, width_bits=64), stats)
    served, walked = (int(x) for x in stats.cpu().numpy())
    assert served >= 0.95 * (served + walked)
    bt.bt_model_free(one)
    bt.bt_model_free(trained)
    tree.close()
