"""Replicas on several GPUs: one batch split evenly over the ranks.

The paper's kernel instances each hold the whole tree and each takes an
equal share of the batch (Sec. IV-G); across GPUs that is one process per
GPU, every rank with the whole tree resident, and a global batch cut into
contiguous, near-equal slices -- rank r searches slice r on its own GPU with
the single-GPU path, and the results come back in input order by placing
each rank's slice at its offset.  Searches need no exchange of data (every
query's result depends only on the tree); the only collective is the
gathering of the results, done here with torch.distributed (NCCL on GPUs,
gloo on CPUs).
"""
from __future__ import annotations


def even_slice(nq: int, world: int, rank: int) -> tuple[int, int]:
    """(start, count) of rank's slice of nq queries: the first nq % world
    ranks get one query more, so slice sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    base, rem = divmod(nq, world)
    start = rank * base + min(rank, rem)
    return start, base + (1 if rank < rem else 0)


def gather_in_input_order(local, nq: int, world: int, rank: int, group=None):
    """All ranks' result slices (a 1-D tensor per rank, rank's even slice of
    nq entries) assembled into one tensor of nq entries in input order, on
    every rank.  Slices are padded to the largest slice for the collective."""
    import torch
    import torch.distributed as dist
    start, count = even_slice(nq, world, rank)
    if local.numel() != count:
        raise ValueError("local results must hold this rank's slice")
    if world == 1:
        return local.clone()
    width = even_slice(nq, world, 0)[1]  # the largest slice
    pad = torch.zeros(width, dtype=local.dtype, device=local.device)
    pad[:count] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    out = torch.empty(nq, dtype=local.dtype, device=local.device)
    for r in range(world):
        s, c = even_slice(nq, world, r)
        out[s:s + c] = parts[r][:c]
    return out
