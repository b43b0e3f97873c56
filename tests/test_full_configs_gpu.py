"""The batching, learned and serving workloads at their full configured sizes,
every result compared with the CPU oracle (the paper checks every batch
against a CPU search, Sec. V-A):

- batching: one CUDA-graph replay of a persistent launch over 10,000 batches
  (sizes log-uniform in 1..1024, Zipf(0.9) queries, 80% hits) addressed to
  four trees of 10^3, 10^5, 10^6 and 2*10^7 uint64 keys whose fanouts and
  launch settings the autotuner chose, with the forest's launch shape from
  the forest autotuner (tuned on the first 1000 batches);
- learned: 2^24 uint64 keys from the three-lognormal mixture, fanout 32, the
  256-segment piecewise-linear model and the 1-32-32-1 MLP, batches of 1024
  and 2^20 at 90% hits;
- serving: a Poisson trace of requests of 1..64 lookups over two resident
  trees of 10^6 and 2*10^7 uint64 keys, plain and learned.

The inputs are the ones the benchmark builds (same recipes and seeds)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import OracleTree
from paper_2604_21117_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def bt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_21117_gb300 import build_lib
    build_lib.build()
    from paper_2604_21117_gb300 import btree
    return btree


def _equal(got_v, got_f, ov, of):
    gv = np.asarray(got_v).astype(np.uint64)
    bad = np.nonzero((gv != ov) | (np.asarray(got_f) != of))[0]
    assert bad.size == 0, f"{bad.size} mismatches, first at {int(bad[0])}"


def test_batching_config_full_size(bt):
    import torch
    sizes = [1000, 100_000, 1_000_000, 20_000_000]
    nbatches = 10_000
    trees, keysets, oracles = [], [], []
    for i, n in enumerate(sizes):
        keys = W.uniform_keys(n, 64, seed=W.SEED_BASE + 20 + i)
        vals = W.rank_values(n, 64)
        sample = W.make_queries(keys, 1024, 0.8, seed=W.SEED_BASE + 30 + i, width_bits=64, zipf_s=0.9)
        h, best = bt.bt_autotune(keys, vals, torch.from_numpy(sample).cuda(), sample.size)
        trees.append(bt.BTree(None, None, handle=h))
        keysets.append(keys)
        oracles.append(OracleTree(keys, vals, int(best.fanout)))
    g = W.rng(W.SEED_BASE + 40)
    counts = W.log_uniform_batch_sizes(nbatches, seed=W.SEED_BASE + 41)
    tids = g.integers(0, len(trees), size=nbatches)
    pools = {ti: W.make_queries(keysets[ti], int(counts[tids == ti].sum()), 0.8, seed=W.SEED_BASE + 50 + ti,
                                width_bits=64, zipf_s=0.9) for ti in range(len(trees))}
    used = {ti: 0 for ti in pools}
    desc = np.zeros(nbatches, bt.BATCH_DESC_DTYPE)
    parts, off = [], 0
    for b in range(nbatches):
        c, ti = int(counts[b]), int(tids[b])
        parts.append(pools[ti][used[ti]:used[ti] + c])
        used[ti] += c
        desc[b] = (ti, c, off)
        off += c
    allq = np.concatenate(parts)
    dq = torch.from_numpy(allq).cuda()
    d_desc = torch.from_numpy(desc.view(np.uint8)).cuda()
    forest = bt.bt_forest_create(trees)
    v = torch.zeros(off, dtype=torch.uint64, device="cuda")
    f = torch.full((off,), 9, dtype=torch.uint8, device="cuda")
    wsb = bt.bt_forest_workspace_bytes(nbatches)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    # the forest's launch shape chosen by its autotuner, as the benchmark does
    bt.bt_forest_autotune(forest, d_desc[: 16 * 1000], 1000, dq, v, f, ws, wsb)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        bt.bt_forest_search(forest, d_desc, nbatches, dq, v, f, ws, wsb, 0, s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bt.bt_forest_search(forest, d_desc, nbatches, dq, v, f, ws, wsb, 0, torch.cuda.current_stream())
    v.zero_()
    f.fill_(9)
    graph.replay()
    torch.cuda.synchronize()
    assert bt.bt_forest_bad_batches() == 0
    vv, ff = v.cpu().numpy(), f.cpu().numpy()
    # every query, tree by tree, against that tree's oracle
    for ti in range(len(trees)):
        sel = np.concatenate([np.arange(int(desc[b]["offset"]), int(desc[b]["offset"]) + int(desc[b]["count"]))
                              for b in range(nbatches) if int(desc[b]["tree"]) == ti])
        ov, of, _, _ = oracles[ti].search(allq[sel])
        _equal(vv[sel], ff[sel], ov, of)
    bt.bt_forest_free(forest)
    for t in trees:
        t.close()
    for o in oracles:
        o.close()


@pytest.fixture(scope="module")
def lognormal_tree(bt):
    n = 1 << 24
    keys = W.lognormal_mixture_keys(n, seed=W.SEED_BASE + 4)
    vals = W.rank_values(n, 64)
    tree = bt.BTree(keys, vals, 32)
    o = OracleTree(keys, vals, 32)
    yield keys, tree, o
    tree.close()
    o.close()


@pytest.mark.parametrize("kind", ["pl256", "mlp"])
def test_learned_config_full_size(bt, lognormal_tree, kind):
    import torch
    keys, tree, o = lognormal_tree
    if kind == "pl256":
        mdl = bt.bt_model_train(tree.handle, bt.BT_MODEL_PL, segments=256)
    else:
        mdl = bt.bt_model_train(tree.handle, bt.BT_MODEL_MLP, h_init=W.mlp_init_params(W.SEED_BASE + 5),
                                steps=2000, batch=16384, lr=2e-3, seed=W.SEED_BASE + 6)
    for B in (1024, 1 << 20):
        q = W.make_queries(keys, B, 0.9, seed=W.SEED_BASE + 7 + B, width_bits=64)
        dq = torch.from_numpy(q).cuda()
        ws, nb = tree.alloc_workspace(B)
        v, f = tree.alloc_outputs(B)
        v.fill_(0)
        f.fill_(9)
        bt.bt_learned_search_batch(tree.handle, mdl, dq, B, v, f, ws, nb)
        torch.cuda.synchronize()
        ov, of, _, _ = o.search(q)
        _equal(v.cpu().numpy(), f.cpu().numpy(), ov, of)
    bt.bt_model_free(mdl)


@pytest.mark.parametrize("learned", [False, True])
def test_serving_config_full_size(bt, learned):
    sizes = [1_000_000, 20_000_000]
    trees, keysets, oracles, models = [], [], [], []
    for i, n in enumerate(sizes):
        keys = W.uniform_keys(n, 64, seed=W.SEED_BASE + 60 + i)
        vals = W.rank_values(n, 64)
        trees.append(bt.BTree(keys, vals, 32))
        keysets.append(keys)
        oracles.append(OracleTree(keys, vals, 32))
        if learned:
            models.append(bt.bt_model_train(trees[-1].handle, bt.BT_MODEL_PL, segments=256))
    rate, seconds = 5e6, 0.05
    nreq = int(rate / 8.0 * seconds)
    seed = W.SEED_BASE + 75
    cnt = W.geometric_request_sizes(nreq, seed=seed).astype(np.uint32)
    tid = W.rng(seed).integers(0, 2, size=nreq).astype(np.uint32)
    pools = [W.make_queries(keysets[i], int(cnt[tid == i].sum()), 0.8, seed=seed + 1 + i, width_bits=64)
             for i in range(2)]
    base = [0, pools[0].size]
    allk = np.concatenate(pools)
    koff = np.empty(nreq, np.uint64)
    cur = [0, 0]
    for r in range(nreq):
        i = int(tid[r])
        koff[r] = base[i] + cur[i]
        cur[i] += int(cnt[r])
    t_arr = W.poisson_arrivals(rate / 8.0, nreq, seed=seed + 3)
    srv = bt.bt_server_create(trees, models if learned else None, slots=8, max_batch=8192, deadline_us=50.0,
                              mem_cap_bytes=16 << 20)
    vals = np.zeros(allk.size, np.uint64)
    found = np.full(allk.size, 9, np.uint8)
    bt.bt_server_run_trace(srv, t_arr, tid, cnt, koff, allk, vals, found)
    st = bt.bt_server_get_stats(srv)
    bt.bt_server_destroy(srv)
    assert st.completed == nreq and st.lookups == allk.size
    for i in range(2):
        lo, hi = base[i], base[i] + pools[i].size
        ov, of, _, _ = oracles[i].search(allk[lo:hi])
        _equal(vals[lo:hi], found[lo:hi], ov, of)
    for m in models:
        bt.bt_model_free(m)
    for t in trees:
        t.close()
    for o in oracles:
        o.close()
