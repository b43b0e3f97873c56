"""Pins for the learned-predictor oracle (oracle/learned.py), no GPU.

The learned leaf predictor is not in the paper; these pins tie each oracle
function to mathematics that does not depend on it: exact recovery of
lines, the normal equations of least squares, finite differences of the
loss, hand-evaluated networks, and brute-force windows."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import OracleTree
from oracle import learned as LO
from paper_2604_21117_gb300 import workloads as W


def test_breakpoints_are_quantiles_and_cover_every_key():
    keys = W.uniform_keys(10_000, 64, seed=1)
    b, inv_w = LO.pl_breakpoints(keys, 256)
    assert np.all(b[1:] > b[:-1])
    s = LO.pl_segment(b, keys)
    counts = np.bincount(s, minlength=256)
    assert counts.min() >= 10_000 // 256 and counts.max() <= 10_000 // 256 + 1
    nxt = np.append(b[1:], keys[-1] + np.uint64(1))
    assert np.all((keys >= b[s]) & (keys < nxt[s]))
    assert inv_w.dtype == np.float32 and np.all(inv_w > 0)


def test_pl_fit_recovers_exact_lines():
    """Labels that are an exact line in x per segment give that line back."""
    keys = np.arange(0, 64 * 8, dtype=np.uint64) * np.uint64(1000)
    b, inv_w = LO.pl_breakpoints(keys, 8)
    s, x = LO.pl_x(b, inv_w, keys)
    a_true = np.linspace(-3.0, 5.0, 8)
    c_true = np.linspace(10.0, 80.0, 8)
    y = a_true[s] * x.astype(np.float64) + c_true[s]
    _, _, slope, icpt = LO.pl_fit(keys, y, 8)
    assert np.allclose(slope, a_true, rtol=1e-6, atol=1e-5)
    assert np.allclose(icpt, c_true, rtol=1e-6, atol=1e-5)


def test_pl_fit_satisfies_normal_equations():
    keys = W.lognormal_mixture_keys(20_000, seed=2)
    o = OracleTree(keys, keys, 32)
    _, _, leaf, _ = o.search(keys)
    b, inv_w, slope, icpt = LO.pl_fit(keys, leaf, 64)
    s, x = LO.pl_x(b, inv_w, keys)
    xd, y = x.astype(np.float64), leaf.astype(np.float64)
    for j in range(64):
        m = s == j
        r = y[m] - (float(slope[j]) * xd[m] + float(icpt[j]))
        # residual orthogonal to 1 and x, up to the fp32 rounding of the line
        scale = np.abs(y[m]).max() * m.sum() * 1e-6 + 1e-3
        assert abs(r.sum()) < scale and abs((r * xd[m]).sum()) < scale


def test_pl_predict_is_fp32_line_rounded_half_even():
    b = np.array([0, 100], np.uint64)
    inv_w = np.array([1 / 100, 1 / 100], np.float32)
    slope = np.array([2.0, 0.0], np.float32)
    icpt = np.array([0.5, 3.0], np.float32)
    q = np.array([0, 25, 50, 150, 10**6], np.uint64)
    got = LO.pl_predict(b, inv_w, slope, icpt, q, L=10)
    # x = 0 -> 0.5 -> rint 0 (half to even); x = .25 -> 1.0; x = .5 -> 1.5 -> 2;
    # segment 1 is flat at 3.0; far keys stay in the last segment
    assert list(got) == [0, 1, 2, 3, 3]
    assert list(LO.pl_predict(b, inv_w, np.float32([1000, 0]), np.float32([0, 0]), q[:1] + 99, L=10)) == [9]


def test_mlp_forward_hand_evaluated():
    p = np.zeros(LO.N_PARAMS)
    W1, b1, W2, b2, w3, b3 = 0, 32, 64, 64 + 1024, 64 + 1024 + 32, 64 + 1024 + 64
    p[W1 + 0] = 1.0         # h1_0 = relu(x)
    p[W2 + 0 * 32 + 0] = 2.0  # h2_0 = relu(2 h1_0)
    p[w3 + 0] = 3.0         # y = 3 h2_0 + b3
    p[b3] = 0.5
    y, _ = LO.mlp_forward(p, np.array([0.25, -1.0, 1.0]))
    assert np.allclose(y, [0.5 + 1.5, 0.5, 0.5 + 6.0])
    assert LO.N_PARAMS == 1153


def test_mlp_gradient_matches_central_differences():
    g = W.rng(3)
    p = g.normal(0, 0.5, LO.N_PARAMS)
    x = g.random(64)
    t = g.random(64)
    ana = LO.mlp_grad(p, x, t)
    _, (_, z1, _, z2, _) = LO.mlp_forward(p, x)
    assert np.min(np.abs(z1)) > 1e-5 and np.min(np.abs(z2)) > 1e-5  # away from ReLU kinks
    eps = 1e-6
    num = np.empty_like(p)
    for i in range(p.size):
        d = np.zeros_like(p)
        d[i] = eps
        num[i] = (LO.mlp_loss(p + d, x, t) - LO.mlp_loss(p - d, x, t)) / (2 * eps)
    assert np.allclose(ana, num, rtol=1e-5, atol=1e-8)


def test_mlp_x_rank_coordinate():
    """The first stage maps a key to its rank fraction: exactly s/64 at the
    s-th breakpoint, 0 below the smallest key, at most 1, non-decreasing in
    the key, and within one segment (1/64) of rank/n whatever the key
    distribution."""
    for keys in (W.uniform_keys(10_000, 64, seed=11), W.lognormal_mixture_keys(10_000, seed=12)):
        b, inv_w = LO.mlp_stage1(keys)
        assert b.size == 64 and np.array_equal(b, keys[(np.arange(64) * keys.size) // 64])
        xb = LO.mlp_x(b, b, inv_w)
        assert xb.dtype == np.float32 and np.array_equal(xb, (np.arange(64) / 64).astype(np.float32))
        x = LO.mlp_x(keys, b, inv_w)
        assert np.all(np.diff(x.astype(np.float64)) >= 0)
        assert x.min() >= 0 and x.max() <= 1
        rank = np.arange(keys.size) / keys.size
        assert np.max(np.abs(x - rank)) <= 1 / 64 + 1e-6
        assert LO.mlp_x(np.array([0], np.uint64), b, inv_w)[0] == 0.0 or keys[0] == 0


def test_range_errors_brute_force():
    g = W.rng(9)
    L = 1000
    leaf = g.integers(0, L, 5000)
    hat = np.clip(leaf + g.integers(-30, 31, 5000), 0, L - 1)
    got = LO.range_errors(hat, leaf, L, 16)
    for r in range(16):
        sel = [abs(int(h) - int(l)) for h, l in zip(hat, leaf) if r * L <= int(h) * 16 < (r + 1) * L]
        assert got[r] == (max(sel) if sel else 0)
    assert got.max() == LO.max_error(hat, leaf)


def test_window_leaf_and_max_error_brute_force():
    leaf_max = np.array([10, 20, 30, 40, 50], np.uint64)
    q = np.array([5, 15, 35, 45, 60, 30], np.uint64)
    true_leaf = [0, 1, 3, 4, 4, 2]
    for err in range(0, 5):
        for hat in range(0, 5):
            got = LO.window_leaf(leaf_max, q, np.full(q.size, hat), err)
            for i, tl in enumerate(true_leaf):
                inside = max(0, hat - err) <= tl <= min(4, hat + err)
                assert got[i] == (tl if inside else -1)
    assert LO.max_error(np.array([0, 3, 2]), np.array([1, 1, 2])) == 2
