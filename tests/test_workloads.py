"""The seeded input generators (no GPU)."""
import numpy as np
import pytest

from paper_2604_21117_gb300 import workloads as W


@pytest.mark.parametrize("width", [32, 64])
def test_uniform_keys_distinct_sorted_seeded(width):
    a = W.uniform_keys(10000, width, seed=1)
    b = W.uniform_keys(10000, width, seed=1)
    assert a.dtype == W.key_dtype(width) and a.size == 10000
    assert np.array_equal(a, b)
    assert np.all(np.diff(a.astype(np.float64)) > 0)


def test_lognormal_mixture_keys():
    k = W.lognormal_mixture_keys(50000, seed=3)
    assert k.size == 50000 and np.all(k[1:] > k[:-1])
    # skewed: the middle half of keys spans a small part of the range
    assert (int(k[37500]) - int(k[12500])) < (int(k[-1]) - int(k[0])) / 20


@pytest.mark.parametrize("zipf", [None, 1.1, 0.9])
def test_queries_hit_fraction_and_misses(zipf):
    keys = W.uniform_keys(5000, 64, seed=5)
    q = W.make_queries(keys, 20000, 0.9, seed=6, width_bits=64, zipf_s=zipf)
    hit = np.isin(q, keys)
    assert abs(hit.mean() - 0.9) < 0.02
    qe = W.make_queries(keys, 256, 0.5, seed=7, width_bits=64, exact_hits=True)
    assert int(np.isin(qe, keys).sum()) == 128
    if zipf is not None:
        _, counts = np.unique(q[hit], return_counts=True)
        assert counts.max() > 100  # skewed hits


def test_batch_sizes_and_requests():
    b = W.log_uniform_batch_sizes(10000, seed=1)
    assert b.min() >= 1 and b.max() <= 1024
    s = W.geometric_request_sizes(10000, seed=2)
    assert s.min() >= 1 and s.max() <= 64 and 6.5 < s.mean() < 9.5
    t = W.poisson_arrivals(1e6, 1000, seed=3)
    assert np.all(np.diff(t) > 0) and 0.5e-3 < t[-1] < 2e-3
