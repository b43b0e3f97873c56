"""Host-side logic of bench.py (no GPU): the algorithmic byte count against
the oracle, the IQM statistic (Eq. 2), and the max-over-ranks reduction of
the replicas-only multi-GPU timing on two gloo ranks."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import bench
from oracle import OracleTree
from paper_2604_21117_gb300 import workloads as W


@pytest.mark.parametrize("m,n,nq,zipf", [(16, 20_000, 3000, None), (32, 100_000, 20_000, 1.1),
                                         (8, 5_000, 777, None), (64, 300_000, 50_000, None)])
def test_touched_counts_match_oracle(m, n, nq, zipf):
    keys = W.uniform_keys(n, 64, seed=n)
    vals = W.rank_values(n, 64)
    o = OracleTree(keys, vals, m)
    q = W.make_queries(keys, nq, 0.9, seed=nq, width_bits=64, zipf_s=zipf)
    counts, sectors = bench.touched(keys, o.level_nodes(), m, q)
    oc, osec = o.touched(q)
    assert counts == oc and sectors == osec


@pytest.mark.parametrize("m,n,prefix", [(16, 5000, 0), (8, 30000, 4), (32, 100000, 24)])
def test_rank_touched_matches_byte_oracle(m, n, prefix):
    """Routing by lower-bound rank gives the byte-key oracle's distinct nodes
    per level and the distinct value sectors of its hits (leaf, slot)."""
    from oracle.bytes_keys import OracleBytesTree
    keys = W.byte_keys(n, 32, seed=60 + n, prefix_bytes=prefix)
    vals = np.arange(n, dtype=np.uint64)
    o = OracleBytesTree(keys, vals, m)
    q = W.make_byte_queries(keys, 4000, 0.7, seed=61)
    kv = keys.view("V32").ravel()
    rank = np.searchsorted(kv, q.view("V32").ravel())
    hit = rank < n
    hit[hit] = kv[rank[hit]] == q.view("V32").ravel()[hit]
    counts, sect = bench.rank_touched(n, o.level_nodes(), m, rank, hit, 8)
    paths = o.paths(q)
    assert counts == [int(np.unique(paths[:, l]).size) for l in range(paths.shape[1])]
    _, found, leaf, slot = o.search(q)
    assert np.array_equal(found.astype(bool), hit)
    h = found == 1
    assert sect == np.unique(((leaf[h] * m + slot[h].astype(np.uint64)) * 8) // 32).size


def test_iqm_eq2_hand_values():
    # n = 8: drop the lowest and highest two, mean of the middle four
    assert bench.iqm([8, 1, 7, 2, 6, 3, 5, 4]) == 4.5
    assert bench.iqm([10, 10, 10, 10]) == 10.0
    # n = 12: middle six of 1..12 are 4..9
    assert bench.iqm(list(range(1, 13))) == 6.5
    # outliers in the outer quartiles do not move it
    assert bench.iqm([1, 2, 3, 4, 5, 6, 7, 1000]) == 4.5


def test_algorithmic_bytes_formula():
    # two levels, 3 + 10 distinct nodes of 32 slots x 8 B, 7 value sectors,
    # batch of 100 (8 B query + 4 B index in, 8 B value + 1 B flag out)
    assert bench.descend_algorithmic_bytes([3, 10], 7, 32, 8, 8, 100) == 13 * 256 + 7 * 32 + 100 * 21


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    bench.dist_init(world, "gloo")
    t = bench.reduce_max(1.5 + rank, world)
    bench.barrier(world)
    out[rank] = t
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, start_method="spawn")
    assert dict(out) == {0: 2.5, 1: 2.5}


@pytest.mark.parametrize("nq,world", [(0, 2), (1, 2), (7, 2), (10, 3), (1 << 20, 8), (1000003, 4)])
def test_even_slices_cover_the_batch_once(nq, world):
    from paper_2604_21117_gb300.replicas import even_slice
    slices = [even_slice(nq, world, r) for r in range(world)]
    assert sum(c for _, c in slices) == nq
    assert max(c for _, c in slices) - min(c for _, c in slices) <= 1
    pos = 0
    for s, c in slices:  # contiguous, in rank order
        assert s == pos
        pos += c


def _split_rank_main(rank, world, port, nq, out):
    """Each rank searches its even slice of one batch with the CPU oracle and
    the results are gathered back in input order."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    from paper_2604_21117_gb300.replicas import even_slice, gather_in_input_order
    bench.dist_init(world, "gloo")
    keys = W.uniform_keys(50_000, 64, seed=90)
    vals = W.rank_values(keys.size, 64)
    q = W.make_queries(keys, nq, 0.8, seed=91, width_bits=64)
    s, c = even_slice(nq, world, rank)
    o = OracleTree(keys, vals, 16)
    v, f, _, _ = o.search(q[s:s + c])
    o.close()
    gv = gather_in_input_order(torch.from_numpy(v.view(np.int64).copy()), nq, world, rank)
    gf = gather_in_input_order(torch.from_numpy(f.astype(np.int64)), nq, world, rank)
    out[rank] = (gv.numpy().view(np.uint64).tobytes(), gf.numpy().astype(np.uint8).tobytes())
    dist.destroy_process_group()


@pytest.mark.parametrize("nq", [1, 5_001])
def test_batch_split_over_two_gloo_ranks(nq):
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_split_rank_main, args=(2, _free_port(), nq, out), nprocs=2, start_method="spawn")
    keys = W.uniform_keys(50_000, 64, seed=90)
    vals = W.rank_values(keys.size, 64)
    q = W.make_queries(keys, nq, 0.8, seed=91, width_bits=64)
    ev, ef = pins_lookup(keys, vals, q)
    for r in range(2):
        gv = np.frombuffer(out[r][0], np.uint64)
        gf = np.frombuffer(out[r][1], np.uint8)
        assert np.array_equal(gv, ev) and np.array_equal(gf, ef)


def pins_lookup(keys, vals, q):
    """The plain definition of a lookup (lower_bound on the sorted keys)."""
    pos = np.searchsorted(keys, q)
    hit = (pos < keys.size) & (keys[np.minimum(pos, keys.size - 1)] == q)
    v = np.full(q.size, np.uint64(2**64 - 1))
    v[hit] = vals[pos[hit]]
    return v, hit.astype(np.uint8)


def _range_rank_main(rank, world, port, out):
    """Rank r holds part r of the key set (a CPU oracle over its key range);
    each rank routes its own batch to the parts' ranks and gets its results
    back in input order."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_2604_21117_gb300 import range_split as RS
    bench.dist_init(world, "gloo")
    keys = W.uniform_keys(40_000, 64, seed=95)
    vals = W.rank_values(keys.size, 64)
    lo, hi = RS.part_bounds(keys.size, world, rank)
    part = OracleTree(keys[lo:hi], vals[lo:hi], 16)
    split = RS.splitters(keys, world)
    # every query lands in one part; misses below the first and above the last key too
    q = W.make_queries(keys, 3000 + 777 * rank, 0.7, seed=96 + rank, width_bits=64, zipf_s=1.1)
    q[:3] = [0, 2**64 - 1, keys[lo]]
    v, f = RS.exchange_search(q, split, lambda k: part.search(k)[:2], world)
    part.close()
    out[rank] = (q.tobytes(), v.tobytes(), f.tobytes())
    dist.destroy_process_group()


def test_range_split_exchange_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_range_rank_main, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    keys = W.uniform_keys(40_000, 64, seed=95)
    vals = W.rank_values(keys.size, 64)
    for r in range(2):
        q = np.frombuffer(out[r][0], np.uint64)
        ev, ef = pins_lookup(keys, vals, q)
        assert np.array_equal(np.frombuffer(out[r][1], np.uint64), ev)
        assert np.array_equal(np.frombuffer(out[r][2], np.uint8), ef)


def test_range_split_routes_by_part_ranges():
    from paper_2604_21117_gb300 import range_split as RS
    keys = W.uniform_keys(1000, 64, seed=97)
    for parts in (1, 2, 3, 7):
        split = RS.splitters(keys, parts)
        assert split.size == parts - 1
        dest = RS.route(keys, split)
        for p in range(parts):
            lo, hi = RS.part_bounds(keys.size, parts, p)
            assert np.all(dest[lo:hi] == p)  # every stored key routes to the part that holds it
        assert RS.route(np.array([0, 2**64 - 1], np.uint64), split).tolist() == [0, parts - 1]


def test_profile_cases_usage_without_a_case():
    from paper_2604_21117_gb300 import profile_cases
    assert profile_cases.main([]) == 2
    assert profile_cases.main(["nothing"]) == 2
