"""The documented order of the on-device batch partition (bt_sort_batch),
checked from the outside: whether an output order satisfies the contract
for the bits the library reports (bt_sort_bits).

Contract (bt_sort_batch in the C header): f(q) is a bucket number
on `bits` bits, f = (c << r) | s with c the number of the tree's splitters
below q and s the q's interpolated position in its splitter segment on r
bits (or c >> cshift when bits is below c's bits); coarse(q) = f >> lb.  The
output is ordered by coarse bucket; inside every coarse bucket of at most
`tile` queries it is ordered by f.
"""
from __future__ import annotations

import numpy as np

LOCAL_BITS = 9


def tile_for(key_bytes: int) -> int:
    """Largest coarse bucket the local sort orders."""
    return 1024


def part_plan(bits: int, nsplit: int):
    """(r, cshift, lb) for a partition on `bits` bits."""
    cbits = int(nsplit).bit_length()
    return max(bits - cbits, 0), max(cbits - bits, 0), min(LOCAL_BITS, bits - 1)


def _runs(a: np.ndarray):
    """(start, end) of the runs of equal values of a."""
    if a.size == 0:
        return []
    starts = np.flatnonzero(np.diff(a, prepend=a[0] - 1))
    ends = np.append(starts[1:], a.size)
    return list(zip(starts.tolist(), ends.tolist()))


def _back_order(pos: np.ndarray) -> float:
    """How far below the running maximum any element falls (0 if sorted)."""
    if pos.size == 0:
        return 0.0
    return float((np.maximum.accumulate(pos) - pos).max())


def check_order(c: np.ndarray, bits: int, nsplit: int, tile: int, pos=None, width=None) -> None:
    """c: exact splitter count below each output key, in output order.
    pos / width (optional, float arrays in output order): the key's offset
    inside its splitter segment and the segment's width, for the
    interpolation part of the order (checked to one interpolation bucket,
    with room for fp32 rounding)."""
    assert bits > 0
    r, cshift, lb = part_plan(bits, nsplit)
    c = c.astype(np.int64)

    def within_segments(lo: int, hi: int, sub_bits: int):
        if pos is None:
            return
        for s0, e0 in _runs(c[lo:hi]):
            s0 += lo
            e0 += lo
            bw = float(width[s0]) / (1 << sub_bits)
            assert _back_order(pos[s0:e0]) <= bw * 1.01 + 2, (int(c[s0]), bw)

    if r == 0:
        f = c >> cshift
        coarse = f >> lb
        assert np.all(np.diff(coarse) >= 0)
        for s0, e0 in _runs(coarse):
            if e0 - s0 <= tile:
                assert np.all(np.diff(f[s0:e0]) >= 0)
    elif r <= lb:
        coarse = c >> (lb - r)
        assert np.all(np.diff(coarse) >= 0)
        for s0, e0 in _runs(coarse):
            if e0 - s0 <= tile:
                assert np.all(np.diff(c[s0:e0]) >= 0)
                within_segments(s0, e0, r)
    else:
        # coarse buckets split splitter segments: c is ordered, and inside a
        # segment the order holds to one coarse interpolation bucket
        assert np.all(np.diff(c) >= 0)
        within_segments(0, c.size, r - lb)
