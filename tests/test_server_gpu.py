"""GPU tests of the serving loop: every request's results equal the oracle's,
the same whether the request is served alone or in a mix with many others,
with plain and learned searches, under a memory cap and back-pressure."""
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


@pytest.fixture(scope="module")
def two_trees(bt):
    out = []
    for i, (n, m) in enumerate(((20_000, 16), (300_000, 32))):
        keys = W.uniform_keys(n, 64, seed=71 + i)
        vals = W.rank_values(n, 64)
        out.append((keys, vals, bt.BTree(keys, vals, m), OracleTree(keys, vals, m)))
    return out


def _trace(trees, nreq, seed, rate):
    sizes = W.geometric_request_sizes(nreq, seed=seed)
    tids = W.rng(seed).integers(0, len(trees), size=nreq)
    keys, offs, off = [], [], 0
    for r in range(nreq):
        k = W.make_queries(trees[tids[r]][0], int(sizes[r]), 0.8, seed=seed * 7919 + r, width_bits=64)
        keys.append(k)
        offs.append(off)
        off += k.size
    t = W.poisson_arrivals(rate, nreq, seed=seed + 1)
    return np.concatenate(keys), np.array(offs, np.uint64), sizes.astype(np.uint32), tids.astype(np.uint32), t


@pytest.mark.parametrize("learned", [False, True, "mixed"])
def test_each_request_alone_equals_in_the_mix(bt, two_trees, learned):
    models = None
    if learned == "mixed":  # an MLP on one tree, the plain descent on the other
        models = [bt.bt_model_train(two_trees[0][2].handle, bt.BT_MODEL_MLP, h_init=W.mlp_init_params(W.SEED_BASE + 5),
                                    steps=200, batch=4096, lr=2e-3, seed=84), None]
    elif learned:
        models = [bt.bt_model_train(t[2].handle, bt.BT_MODEL_PL, segments=64) for t in two_trees]
    srv = bt.bt_server_create([t[2] for t in two_trees], models, slots=4, max_batch=2048, deadline_us=50.0)
    keys, offs, sizes, tids, t = _trace(two_trees, 3000, seed=81, rate=2e5)
    vals = np.zeros(keys.size, np.uint64)
    found = np.full(keys.size, 9, np.uint8)
    bt.bt_server_run_trace(srv, t, tids, sizes, offs, keys, vals, found)
    st = bt.bt_server_get_stats(srv)
    assert st.completed == 3000 and st.lookups == keys.size and st.batches < 3000
    # in the mix == oracle
    for r in range(0, 3000, 7):
        o, c, tr = int(offs[r]), int(sizes[r]), int(tids[r])
        ov, of, _, _ = two_trees[tr][3].search(keys[o:o + c])
        assert np.array_equal(vals[o:o + c], ov) and np.array_equal(found[o:o + c], of)
    # alone == in the mix, through the submit / poll interface
    done = bt.bt_server_poll(srv, 1 << 16)  # the trace's tickets
    assert len(done) == 3000 and len(set(done)) == 3000
    for r in range(0, 3000, 211):
        o, c, tr = int(offs[r]), int(sizes[r]), int(tids[r])
        q = keys[o:o + c].copy()
        v1 = np.zeros(c, np.uint64)
        f1 = np.zeros(c, np.uint8)
        ticket = bt.bt_server_submit(srv, tr, q, v1, f1)
        bt.bt_server_drain(srv, 10.0)
        assert bt.bt_server_poll(srv, 1 << 16) == [ticket]
        assert np.array_equal(v1, vals[o:o + c]) and np.array_equal(f1, found[o:o + c])
    bt.bt_server_destroy(srv)
    if models:
        for m in models:
            if m:
                bt.bt_model_free(m)


def test_memory_cap_and_back_pressure(bt, two_trees):
    # a cap of one small batch in flight, and a pending cap that refuses submissions
    srv = bt.bt_server_create([t[2] for t in two_trees], None, slots=4, max_batch=512, deadline_us=20.0,
                              mem_cap_bytes=512 * 17, pending_cap_bytes=64 * 17)
    keys, offs, sizes, tids, t = _trace(two_trees, 1500, seed=82, rate=1e6)
    vals = np.zeros(keys.size, np.uint64)
    found = np.zeros(keys.size, np.uint8)
    bt.bt_server_run_trace(srv, t, tids, sizes, offs, keys, vals, found)
    st = bt.bt_server_get_stats(srv)
    assert st.completed == 1500
    for r in range(0, 1500, 11):
        o, c, tr = int(offs[r]), int(sizes[r]), int(tids[r])
        ov, of, _, _ = two_trees[tr][3].search(keys[o:o + c])
        assert np.array_equal(vals[o:o + c], ov) and np.array_equal(found[o:o + c], of)
    # direct submissions beyond the pending cap are refused, not queued
    big = keys[: 200].copy()
    v = np.zeros(big.size, np.uint64)
    f = np.zeros(big.size, np.uint8)
    with pytest.raises(bt.BTreeError) as e:
        bt.bt_server_submit(srv, 0, big, v, f)
    assert e.value.code == "BT_ERR_ARG"  # larger than the pending cap: never admissible
    bt.bt_server_destroy(srv)


def test_one_batch_serves_both_trees(bt, two_trees):
    """A burst of requests to both trees, all waiting when the deadline
    passes, is served by one multi-tree batch."""
    srv = bt.bt_server_create([t[2] for t in two_trees], None, slots=2, max_batch=4096, deadline_us=20000.0)
    keys, offs, sizes, tids, _ = _trace(two_trees, 60, seed=85, rate=1e6)
    assert set(tids.tolist()) == {0, 1}
    vals = np.zeros(keys.size, np.uint64)
    found = np.zeros(keys.size, np.uint8)
    for r in range(60):
        o, c = int(offs[r]), int(sizes[r])
        bt.bt_server_submit(srv, int(tids[r]), keys[o:o + c], vals[o:o + c], found[o:o + c])
    bt.bt_server_drain(srv, 10.0)
    st = bt.bt_server_get_stats(srv)
    assert st.completed == 60 and st.batches == 1
    for r in range(60):
        o, c, tr = int(offs[r]), int(sizes[r]), int(tids[r])
        ov, of, _, _ = two_trees[tr][3].search(keys[o:o + c])
        assert np.array_equal(vals[o:o + c], ov) and np.array_equal(found[o:o + c], of)
    bt.bt_server_destroy(srv)


def test_batches_overlap_on_the_device(bt, two_trees):
    srv = bt.bt_server_create([t[2] for t in two_trees], None, slots=8, max_batch=256, deadline_us=5.0)
    keys, offs, sizes, tids, t = _trace(two_trees, 4000, seed=83, rate=5e6)
    vals = np.zeros(keys.size, np.uint64)
    found = np.zeros(keys.size, np.uint8)
    bt.bt_server_run_trace(srv, t, tids, sizes, offs, keys, vals, found)
    st = bt.bt_server_get_stats(srv)
    assert st.completed == 4000 and st.max_inflight >= 2
    bt.bt_server_destroy(srv)


def test_many_trees_and_32_bit_keys(bt):
    """40 trees of 32-bit keys and values: a batch's work list (up to two
    entries per tree) no longer fits the kernel's shared-memory copy and is
    read from host-mapped memory; every request equals its tree's oracle."""
    trees = []
    for i in range(40):
        n = 50 + 997 * i
        keys = W.uniform_keys(n, 32, seed=300 + i)
        vals = W.rank_values(n, 32)
        trees.append((keys, vals, bt.BTree(keys, vals, 16), OracleTree(keys, vals, 16, val_bits=32)))
    srv = bt.bt_server_create([t[2] for t in trees], None, slots=4, max_batch=4096, deadline_us=2000.0)
    g = W.rng(87)
    nreq = 2000
    tids = g.integers(0, 40, size=nreq)
    sizes = W.geometric_request_sizes(nreq, seed=88)
    reqs = []
    for r in range(nreq):
        q = W.make_queries(trees[tids[r]][0], int(sizes[r]), 0.8, seed=400 + r, width_bits=32)
        v = np.zeros(q.size, np.uint32)
        f = np.full(q.size, 9, np.uint8)
        bt.bt_server_submit(srv, int(tids[r]), q, v, f)
        reqs.append((int(tids[r]), q, v, f))
    bt.bt_server_drain(srv, 30.0)
    st = bt.bt_server_get_stats(srv)
    assert st.completed == nreq
    for tr, q, v, f in reqs:
        ov, of, _, _ = trees[tr][3].search(q)
        assert np.array_equal(v.astype(np.uint64), ov) and np.array_equal(f, of)
    bt.bt_server_destroy(srv)


def test_rings_wrap_many_times(bt, two_trees):
    """A ring of 3 * max_batch lookups per tree and one slot: thousands of
    requests wrap the rings again and again (requests never straddle the end:
    the space before it is skipped), and a tree's stretch in a batch splits
    into two work-list entries where it wraps; every request equals the
    oracle."""
    srv = bt.bt_server_create([t[2] for t in two_trees], None, slots=1, max_batch=64, deadline_us=1.0)
    keys, offs, sizes, tids, t = _trace(two_trees, 3000, seed=89, rate=2e6)
    vals = np.zeros(keys.size, np.uint64)
    found = np.full(keys.size, 9, np.uint8)
    bt.bt_server_run_trace(srv, t, tids, sizes, offs, keys, vals, found)
    st = bt.bt_server_get_stats(srv)
    assert st.completed == 3000 and st.lookups == keys.size and st.batches >= keys.size // 64
    for r in range(3000):
        o, c, tr = int(offs[r]), int(sizes[r]), int(tids[r])
        ov, of, _, _ = two_trees[tr][3].search(keys[o:o + c])
        assert np.array_equal(vals[o:o + c], ov) and np.array_equal(found[o:o + c], of), r
    bt.bt_server_destroy(srv)
