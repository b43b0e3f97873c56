"""Seeded synthetic inputs shared by the GPU path's tests, the benchmark and
the oracle's tests.

This module holds none of the search method's arithmetic: it only draws keys,
values, query mixes, batch sizes and arrival times.  The paper evaluates on
randomly generated tree entries and search keys (Sec. I, Sec. V-A), so seeded
synthetic data of the same shape stands in for its workloads.

Recipes (every draw is a numpy PCG64 stream from an explicit seed):

* keys, uniform: distinct integers drawn uniformly from [0, 2^w), w = 32/64,
  drawn with replacement, de-duplicated, topped up, then a uniform subset of
  exactly n is kept and sorted.
* keys, lognormal mixture: x from one of three lognormals (equal weights,
  mu = (0, 1, 2), sigma = (1.0, 2.0, 0.5)), key = floor(x * 2^40), distinct,
  exactly n kept.
* values: the key's rank (0..n-1) in the value width.
* queries: each query is a hit with probability p (or exactly round(p*B)
  hits, shuffled, when ``exact_hits``); a hit is a tree key chosen uniformly,
  or by Zipf(s) rank where rank r maps to key index perm[r-1] for a seeded
  random permutation (hot keys spread over the tree); a miss is uniform over
  [0, 2^w) with keys of the tree rejected.
* batch sizes: floor(exp(U(0, ln 1024))) clamped to [1, 1024].
* requests: Poisson arrivals at rate lambda, sizes geometric with mean 8
  truncated to [1, 64] by resampling.
"""
from __future__ import annotations

import functools

import numpy as np

SEED_BASE = 0xB7EE0000


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def key_dtype(width_bits: int):
    if width_bits == 32:
        return np.uint32
    if width_bits == 64:
        return np.uint64
    raise ValueError("key width must be 32 or 64 bits")


def _draw_uniform(g: np.random.Generator, size: int, width_bits: int) -> np.ndarray:
    if width_bits == 64:
        return g.integers(0, 2**64, size=size, dtype=np.uint64, endpoint=False)
    return g.integers(0, 2**32, size=size, dtype=np.uint64, endpoint=False)


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    """np.unique(a) for a 1-D array, by sorting (the same result, without
    numpy's hash-based path, which is slow for tens of millions of keys)."""
    a = np.sort(a)
    if a.size < 2:
        return a
    keep = np.empty(a.size, bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def _in_sorted(values: np.ndarray, sorted_keys: np.ndarray) -> np.ndarray:
    """np.isin(values, sorted_keys) for an ascending key array, by binary search."""
    if sorted_keys.size == 0:
        return np.zeros(values.size, bool)
    pos = np.searchsorted(sorted_keys, values)
    return sorted_keys[np.minimum(pos, sorted_keys.size - 1)] == values


def _exactly_n(pool: np.ndarray, n: int, g: np.random.Generator) -> np.ndarray:
    if pool.size > n:
        keep = g.choice(pool.size, size=n, replace=False)
        pool = np.sort(pool[keep])
    return pool


def uniform_keys(n: int, width_bits: int, seed: int) -> np.ndarray:
    """n distinct keys, uniform over [0, 2^width), sorted ascending."""
    if width_bits == 32 and n > 2**32:
        raise ValueError("too many distinct 32-bit keys")
    g = rng(seed)
    pool = np.empty(0, np.uint64)
    while pool.size < n:
        need = n - pool.size
        pool = _sorted_unique(np.concatenate([pool, _draw_uniform(g, need + need // 16 + 16, width_bits)]))
    return _exactly_n(pool, n, g).astype(key_dtype(width_bits))


def lognormal_mixture_keys(n: int, seed: int, mus=(0.0, 1.0, 2.0), sigmas=(1.0, 2.0, 0.5),
                           scale: float = 2.0**40) -> np.ndarray:
    """n distinct uint64 keys floor(x * scale), x from an equal-weight lognormal mixture."""
    g = rng(seed)
    mus = np.asarray(mus, np.float64)
    sigmas = np.asarray(sigmas, np.float64)
    pool = np.empty(0, np.uint64)
    limit = np.float64(2.0**64 - 2.0**12)
    while pool.size < n:
        need = n - pool.size
        size = need + need // 8 + 16
        comp = g.integers(0, mus.size, size=size)
        x = g.lognormal(mean=mus[comp], sigma=sigmas[comp])
        k = np.floor(np.minimum(x * scale, limit)).astype(np.uint64)
        pool = _sorted_unique(np.concatenate([pool, k]))
    return _exactly_n(pool, n, g)


def rank_values(n: int, width_bits: int) -> np.ndarray:
    """Value of key i = its rank i, in the value width."""
    return np.arange(n, dtype=key_dtype(width_bits))


@functools.lru_cache(maxsize=4)
def _zipf_cdf(n: int, s: float) -> np.ndarray:
    w = np.arange(1, n + 1, dtype=np.float64) ** (-float(s))
    c = np.cumsum(w)
    c /= c[-1]
    return c


def zipf_ranks(n: int, s: float, size: int, g: np.random.Generator) -> np.ndarray:
    """Ranks in 1..n with P(r) proportional to r^-s (exact discrete inverse CDF)."""
    cdf = _zipf_cdf(int(n), float(s))
    u = g.random(size)
    r = np.searchsorted(cdf, u, side="right") + 1
    return np.minimum(r, n).astype(np.int64)


def make_queries(keys: np.ndarray, nq: int, hit_frac: float, seed: int, width_bits: int,
                 zipf_s: float | None = None, exact_hits: bool = False) -> np.ndarray:
    """A batch of nq point queries against the sorted key array `keys`."""
    g = rng(seed)
    dt = key_dtype(width_bits)
    n = int(keys.size)
    if nq == 0:
        return np.empty(0, dt)
    if n == 0:
        hit_frac = 0.0
    if exact_hits:
        nh = int(round(nq * hit_frac))
        is_hit = np.zeros(nq, bool)
        is_hit[:nh] = True
        g.shuffle(is_hit)
    else:
        is_hit = g.random(nq) < hit_frac
    nh = int(is_hit.sum())
    out = np.empty(nq, np.uint64)
    if nh:
        if zipf_s is None:
            idx = g.integers(0, n, size=nh)
        else:
            perm = g.permutation(n)
            idx = perm[zipf_ranks(n, zipf_s, nh, g) - 1]
        out[is_hit] = keys.astype(np.uint64)[idx]
    nm = nq - nh
    if nm:
        miss = np.empty(0, np.uint64)
        ku = keys.astype(np.uint64)
        if ku.size > 1 and not np.all(ku[1:] >= ku[:-1]):
            ku = np.sort(ku)
        while miss.size < nm:
            d = _draw_uniform(g, (nm - miss.size) + 16, width_bits)
            d = d[~_in_sorted(d, ku)]
            miss = np.concatenate([miss, d])
        out[~is_hit] = miss[:nm]
    return out.astype(dt)


def _sort_rows(a: np.ndarray) -> np.ndarray:
    """Rows of a (n, kb) uint8 array in lexicographic byte order, duplicates dropped."""
    if a.shape[0] == 0:
        return a
    order = np.lexsort(a.T[::-1])
    a = a[order]
    keep = np.ones(a.shape[0], bool)
    keep[1:] = np.any(a[1:] != a[:-1], axis=1)
    return a[keep]


def byte_keys(n: int, kb: int, seed: int, prefix_bytes: int = 0) -> np.ndarray:
    """n distinct kb-byte keys as an (n, kb) uint8 array in lexicographic
    order: `prefix_bytes` leading bytes shared by every key (drawn once),
    the rest uniform random bytes."""
    if n > 256 ** min(kb - prefix_bytes, 8) // 4:
        raise ValueError("too few free bytes for n distinct keys")
    g = rng(seed)
    prefix = g.integers(0, 256, size=prefix_bytes, dtype=np.uint8)
    out = np.empty((0, kb), np.uint8)
    while out.shape[0] < n:
        d = g.integers(0, 256, size=(n - out.shape[0] + 16, kb), dtype=np.uint8)
        d[:, :prefix_bytes] = prefix
        out = _sort_rows(np.concatenate([out, d]))
    if out.shape[0] > n:
        out = out[np.sort(g.choice(out.shape[0], n, replace=False))]
    return np.ascontiguousarray(out)


def make_byte_queries(keys: np.ndarray, nq: int, hit_frac: float, seed: int,
                      zipf_s: float | None = None) -> np.ndarray:
    """nq kb-byte queries, an (nq, kb) uint8 array: about hit_frac of them
    copies of stored keys (uniform or Zipf(s) over a random key permutation),
    the rest random rows sharing the keys' first byte distribution that are
    not stored keys."""
    g = rng(seed)
    n, kb = keys.shape
    out = np.empty((nq, kb), np.uint8)
    if nq == 0:
        return out
    is_hit = g.random(nq) < (hit_frac if n else 0.0)
    nh = int(is_hit.sum())
    if nh:
        if zipf_s is None:
            idx = g.integers(0, n, size=nh)
        else:
            idx = g.permutation(n)[zipf_ranks(n, zipf_s, nh, g) - 1]
        out[is_hit] = keys[idx]
    nm = nq - nh
    if nm:
        stored = {bytes(r) for r in keys} if n <= 4_000_000 else None
        miss = g.integers(0, 256, size=(nm, kb), dtype=np.uint8)
        if n:
            # keep the keys' leading bytes so that misses land inside the key range
            src = keys[g.integers(0, n, size=nm)]
            lead = g.integers(0, kb // 2 + 1, size=nm)
            for i in range(nm):
                miss[i, :lead[i]] = src[i, :lead[i]]
        if stored is not None:
            for i in range(nm):
                while bytes(miss[i]) in stored:
                    miss[i, -1] ^= 0x5A
                    miss[i, -2] = g.integers(0, 256)
        out[~is_hit] = miss
    return out


def log_uniform_batch_sizes(count: int, seed: int, lo: int = 1, hi: int = 1024) -> np.ndarray:
    """floor(exp(U(ln lo, ln hi))) clamped to [lo, hi]."""
    g = rng(seed)
    b = np.floor(np.exp(g.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    return np.clip(b, lo, hi)


def poisson_arrivals(rate_per_s: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process."""
    g = rng(seed)
    return np.cumsum(g.exponential(1.0 / rate_per_s, size=count))


def geometric_request_sizes(count: int, seed: int, mean: float = 8.0, lo: int = 1,
                            hi: int = 64) -> np.ndarray:
    """Geometric sizes with the given mean, truncated to [lo, hi] by resampling."""
    g = rng(seed)
    p = 1.0 / mean
    out = g.geometric(p, size=count)
    bad = (out < lo) | (out > hi)
    while bad.any():
        out[bad] = g.geometric(p, size=int(bad.sum()))
        bad = (out < lo) | (out > hi)
    return out.astype(np.int64)


def mlp_init_params(seed: int, hidden: int = 32) -> np.ndarray:
    """Random initial parameters of the 1 -> hidden -> hidden -> 1 network in
    the order W1, b1, W2 (row = output unit), b2, w3, b3: first-layer kinks
    spread uniformly over the unit input range, He-scaled later layers."""
    g = rng(seed)
    w1 = g.normal(0.0, 4.0, hidden)
    b1 = -w1 * g.random(hidden)
    w2 = g.normal(0.0, np.sqrt(2.0 / hidden), (hidden, hidden))
    b2 = g.normal(0.0, 0.01, hidden)
    w3 = g.normal(0.0, np.sqrt(2.0 / hidden), hidden)
    b3 = np.zeros(1)
    return np.concatenate([w1, b1, w2.ravel(), b2, w3, b3]).astype(np.float32)
