"""Range-partitioned trees across GPUs: the host side of the exchange.

Every rank holds one part of the key set (a contiguous key range, the part
bt_range_build would give it) as its own tree.  A rank's batch is routed:
every query goes to the rank whose range holds it (the first part whose
splitter -- its largest key -- is >= the query; the last part beyond all
splitters); one all-to-all moves the queries, each rank searches what it
received with its own tree, and a second all-to-all moves the results back,
where they are put at their input positions.  The paper's kernel instances
share one batch (Sec. IV-G); this is that sharing with the tree split by key
range instead of copied.

The collectives are torch.distributed all_to_all_single calls (NCCL on GPUs,
gloo on CPUs); the search itself is a callable, the GPU search on a GPU rank.
"""
from __future__ import annotations

import numpy as np


def part_bounds(n: int, parts: int, p: int) -> tuple[int, int]:
    """Ranks [lo, hi) of the keys of part p (as bt_range_build splits them)."""
    if not 0 <= p < parts or n < parts:
        raise ValueError("need 0 <= p < parts <= n")
    return p * n // parts, (p + 1) * n // parts


def splitters(keys: np.ndarray, parts: int) -> np.ndarray:
    """The largest key of every part but the last."""
    return np.array([keys[part_bounds(keys.size, parts, p)[1] - 1] for p in range(parts - 1)], dtype=keys.dtype)


def route(q: np.ndarray, split: np.ndarray) -> np.ndarray:
    """Destination part of every query: the number of splitters below it."""
    return np.searchsorted(split, q, side="left").astype(np.int64)


def exchange_search(q: np.ndarray, split: np.ndarray, search, world: int, group=None):
    """Route this rank's queries to their parts' ranks, search what arrives
    with `search(keys) -> (values uint64, found uint8)`, route the results
    back; returns (values, found) in this rank's input order."""
    import torch
    import torch.distributed as dist
    dest = route(q, split)
    order = np.argsort(dest, kind="stable")  # queries grouped by destination rank
    send_counts = np.bincount(dest, minlength=world).astype(np.int64)
    # 1. how many queries each rank sends to each rank
    sc = torch.from_numpy(send_counts)
    rc = torch.empty_like(sc)
    dist.all_to_all_single(rc, sc, group=group)
    recv_counts = rc.numpy().astype(np.int64)
    # 2. the queries (as int64 bit patterns)
    sq = torch.from_numpy(q[order].astype(np.uint64).view(np.int64))
    rq = torch.empty(int(recv_counts.sum()), dtype=torch.int64)
    dist.all_to_all_single(rq, sq, output_split_sizes=recv_counts.tolist(), input_split_sizes=send_counts.tolist(),
                           group=group)
    # 3. this rank's part searches what it received
    v, f = search(rq.numpy().view(np.uint64).astype(q.dtype))
    # 4. the results go back the way the queries came
    packed = torch.from_numpy(np.stack([np.asarray(v, np.uint64).view(np.int64),
                                        np.asarray(f, np.uint8).astype(np.int64)], axis=1).reshape(-1))
    back = torch.empty(2 * q.size, dtype=torch.int64)
    dist.all_to_all_single(back, packed, output_split_sizes=(2 * send_counts).tolist(),
                           input_split_sizes=(2 * recv_counts).tolist(), group=group)
    res = back.numpy().reshape(-1, 2)
    vals = np.empty(q.size, np.uint64)
    found = np.empty(q.size, np.uint8)
    vals[order] = res[:, 0].view(np.uint64)
    found[order] = res[:, 1].astype(np.uint8)
    return vals, found
