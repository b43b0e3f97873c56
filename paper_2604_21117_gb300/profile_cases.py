"""Small, self-contained workloads for profiling single kernels with ncu.

    python -m paper_2604_21117_gb300.profile_cases forest [warps pin_budget lane_queries staging]
    python -m paper_2604_21117_gb300.profile_cases keys32 [sorted|full]
    python -m paper_2604_21117_gb300.profile_cases crossover
    python -m paper_2604_21117_gb300.profile_cases shapes

forest: the multi-tree batching workload -- trees of 10^3, 10^5, 10^6 and
2*10^7 uniform uint64 keys at fanout 32, a work list of 10,000 batches whose
sizes are log-uniform in 1..1024, Zipf(0.9) queries with 80% hits -- searched
five times by bt_forest_search at the given forest launch settings (default:
4 warps per block, no pinned levels, two queries per lane, every level read
through L1).

keys32: the paper's own tree (2^20 distinct 32-byte keys, 8-byte values,
fanout 16) and a batch of 2^20 uniform queries at 90% hits: six descents of
the batch partitioned on 20 bits (sorted) or six whole searches (full).

crossover: whole searches (bt_search_batch_ex) with no partition and with
a partition on log2 B bits, batches B of 2^16 to 2^20 queries at 90% hits,
over three trees that the L2 could hold -- 2^20 32-byte keys at fanout 16,
and 10^6 and 4 * 10^6 uint64 keys at fanout 32 -- each with the L2 left warm
and with a 256 MB write before every call; medians of 40 calls.

shapes: the descent of 2^20 queries partitioned on 20 bits over 2^24 uniform
uint64 keys at fanout 32 (four batches in turn), at 4, 8 and 16 warps per
block and 1 to 8 resident blocks per SM (bt_tree_set_corun; "max" = as many
as fit); medians of 60 launches.

Each prints its CUDA-event times; the inputs come from workloads.py with
fixed seeds.
"""
from __future__ import annotations

import sys

import numpy as np


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def forest(warps: int = 4, pin_budget: int = 0, lane_queries: int = 2, staging: int = 1) -> None:
    import torch
    from . import build_lib
    build_lib.build()
    from . import btree as bt
    from . import workloads as W
    sizes = [1000, 100_000, 1_000_000, 20_000_000]
    trees, keysets = [], []
    for i, n in enumerate(sizes):
        keys = W.uniform_keys(n, 64, seed=W.SEED_BASE + 20 + i)
        trees.append(bt.BTree(keys, W.rank_values(n, 64), 32))
        keysets.append(keys)
    nbatches = 10_000
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
    f = bt.bt_forest_create(trees)
    bt.bt_forest_set_launch(f, warps, pin_budget, lane_queries, staging)
    v = torch.empty(allq.size, dtype=torch.uint64, device="cuda")
    found = torch.empty(allq.size, dtype=torch.uint8, device="cuda")
    wsb = bt.bt_forest_workspace_bytes(nbatches)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    for it in range(5):
        e0, e1 = _events()
        e0.record(s)
        bt.bt_forest_search(f, d_desc, nbatches, dq, v, found, ws, wsb)
        e1.record(s)
        torch.cuda.synchronize()
        print(f"forest launch {it}: {1000 * e0.elapsed_time(e1):.1f} us, {allq.size} queries")
    bt.bt_forest_free(f)
    for t in trees:
        t.close()


def keys32(mode: str = "sorted") -> None:
    import torch
    from . import build_lib
    build_lib.build()
    from . import btree as bt
    from . import workloads as W
    n, m, B = 1 << 20, 16, 1 << 20
    keys = W.byte_keys(n, 32, seed=W.SEED_BASE + 8)
    tree = bt.BTree(keys, W.rank_values(n, 64), m)
    q = torch.from_numpy(W.make_byte_queries(keys, B, 0.9, seed=W.SEED_BASE + 9 + B)).cuda()
    nb = tree.workspace_bytes(B)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    v, f = tree.alloc_outputs(B)
    s = torch.cuda.current_stream()
    sq = torch.empty_like(q)
    si = torch.empty(B, dtype=torch.int32, device="cuda")
    bt.bt_sort_batch(tree.handle, q, B, 20, sq, si, ws, nb, s)
    for it in range(6):
        e0, e1 = _events()
        e0.record(s)
        if mode == "sorted":
            bt.bt_descend_sorted(tree.handle, sq, si, B, v, f, None, s)
        else:
            bt.bt_search_batch(tree.handle, q, B, v, f, ws, nb, s)
        e1.record(s)
        torch.cuda.synchronize()
        print(f"32-byte keys, {mode} {it}: {1000 * e0.elapsed_time(e1):.1f} us")
    tree.close()


def crossover(steps: int = 40) -> None:
    import statistics
    import torch
    from . import build_lib
    build_lib.build()
    from . import btree as bt
    from . import workloads as W
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()

    def median_us(fn, flushing):
        for _ in range(3):
            fn()
        ev = []
        for i in range(steps):
            if flushing:
                flush.fill_(i & 255)
            e0, e1 = _events()
            e0.record(s)
            fn()
            e1.record(s)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        return statistics.median(1000 * a.elapsed_time(b) for a, b in ev)

    kb = W.byte_keys(1 << 20, 32, seed=W.SEED_BASE + 8)
    k6 = W.uniform_keys(1_000_000, 64, seed=W.SEED_BASE + 3)
    k7 = W.uniform_keys(4_000_000, 64, seed=W.SEED_BASE + 4)
    cases = [
        ("2^20 32-byte keys, m=16", bt.BTree(kb, W.rank_values(kb.shape[0], 64), 16),
         lambda B: W.make_byte_queries(kb, B, 0.9, seed=W.SEED_BASE + 9 + B)),
        ("10^6 uint64 keys, m=32", bt.BTree(k6, W.rank_values(k6.size, 64), 32),
         lambda B: W.make_queries(k6, B, 0.9, seed=B + 5, width_bits=64)),
        ("4*10^6 uint64 keys, m=32", bt.BTree(k7, W.rank_values(k7.size, 64), 32),
         lambda B: W.make_queries(k7, B, 0.9, seed=B + 6, width_bits=64)),
    ]
    for name, tree, make in cases:
        mb = int(bt.bt_tree_info(tree.handle).device_bytes) / 1e6
        for B in (1 << 16, 1 << 18, 1 << 19, 1 << 20):
            q = torch.from_numpy(make(B)).cuda()
            nb = tree.workspace_bytes(B)
            ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
            v, f = tree.alloc_outputs(B)
            cols = []
            for flushing in (False, True):
                for sb in (0, B.bit_length() - 1):
                    fn = lambda sb=sb: bt.bt_search_batch_ex(tree.handle, q, B, v, f, ws, nb, sb, None, s)
                    cols.append(f"{'flushed' if flushing else 'warm'} bits={sb}: {median_us(fn, flushing):.1f} us")
            print(f"{name} ({mb:.0f} MB), {B} queries: " + " | ".join(cols), flush=True)
        tree.close()


def shapes(steps: int = 60) -> None:
    import statistics
    import torch
    from . import build_lib
    build_lib.build()
    from . import btree as bt
    from . import workloads as W
    n, B = 1 << 24, 1 << 20
    keys = W.uniform_keys(n, 64, seed=W.SEED_BASE + 2)
    tree = bt.BTree(keys, W.rank_values(n, 64), 32)
    nb = tree.workspace_bytes(B)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    v, f = tree.alloc_outputs(B)
    s = torch.cuda.current_stream()
    batches = []
    for i in range(4):
        q = torch.from_numpy(W.make_queries(keys, B, 0.9, seed=W.SEED_BASE + 2 + 1000 * (i + 1), width_bits=64)).cuda()
        sq = torch.empty_like(q)
        si = torch.empty(B, dtype=torch.int32, device="cuda")
        bt.bt_sort_batch(tree.handle, q, B, 20, sq, si, ws, nb, s)
        batches.append((sq, si))
    for warps in (4, 8, 16):
        for bps in (0, 1, 2, 3, 4, 6, 8):
            if warps * bps > 64 or (bps and warps * bps < 8):
                continue
            bt.bt_tree_set_launch(tree.handle, warps, 16384)
            bt.bt_tree_set_corun(tree.handle, bps, 0)
            for i in range(4):
                bt.bt_descend_sorted(tree.handle, *batches[i], B, v, f, None, s)
            ev = []
            for i in range(steps):
                e0, e1 = _events()
                e0.record(s)
                bt.bt_descend_sorted(tree.handle, *batches[i % 4], B, v, f, None, s)
                e1.record(s)
                ev.append((e0, e1))
            torch.cuda.synchronize()
            us = statistics.median(1000 * a.elapsed_time(b) for a, b in ev)
            print(f"{warps} warps per block, {bps or 'max'} blocks per SM: descent {us:.1f} us", flush=True)
    tree.close()


def main(argv=None) -> int:
    argv = sys.argv[1:] if argv is None else argv
    if not argv or argv[0] not in ("forest", "keys32", "crossover", "shapes"):
        print(__doc__)
        return 2
    if argv[0] == "forest":
        forest(*(int(x) for x in argv[1:5]))
    elif argv[0] == "keys32":
        keys32(*argv[1:2])
    elif argv[0] == "crossover":
        crossover()
    else:
        shapes()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
