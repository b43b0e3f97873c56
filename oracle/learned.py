"""CPU oracle for the learned leaf predictor -- TEST INFRASTRUCTURE ONLY.

The paper has no learned component; this restates, in plain numpy, the
definitions the GPU library documents in include/btree_gb300.h for its
learned leaf predictor, so that the GPU fitting, training and inference
kernels can be checked:

* training pairs: every stored key with the index of the leaf holding it
  (the leaf index is the tree's own output, see OracleTree.search);
* PL model: S segments split at key quantiles b_s = k[floor(s*n/S)], a
  least-squares line per segment on x = fp32(fp64(q - b_s)) * inv_w_s;
* MLP model 1 -> 32 -> 32 -> 1 with ReLU on a rank coordinate (two stages):
  the first stage is 64 breakpoints at key quantiles, as the PL model's, and
  x = fp32(fp32(s) + min(fp32(fp64(q - b_s)) * inv_w_s, 1)) * (1/64); trained
  on the target leaf / (L - 1) with mean squared error;
* prediction leaf_hat = rint(clamp(pred)) decided in fp32 exactly as the GPU
  does (separately rounded multiply and add for PL);
* max_err = max over stored keys of |leaf_hat - leaf|.

fp64 throughout except where the GPU's fp32 decision has to be reproduced.
"""
from __future__ import annotations

import numpy as np

H = 32  # hidden width of the MLP
N_PARAMS = H + H + H * H + H + H + 1  # W1, b1, W2, b2, w3, b3 = 1153


# ----------------------------------------------------------- PL model

def pl_breakpoints(keys: np.ndarray, segments: int):
    """b_s = keys[floor(s*n/S)] and inv_w_s = fp32(1 / fp64(width_s)), where
    width_s = b_{s+1} - b_s and the last width reaches one past the largest key."""
    k = keys.astype(np.uint64)
    n = k.size
    S = segments
    idx = (np.arange(S, dtype=np.int64) * n) // S
    b = k[idx]
    nxt = np.empty(S, np.uint64)
    nxt[:-1] = b[1:]
    nxt[-1] = k[-1] + np.uint64(1) if k[-1] != np.uint64(2**64 - 1) else k[-1]
    width = nxt - b
    width = np.maximum(width, np.uint64(1))
    inv_w = (1.0 / width.astype(np.float64)).astype(np.float32)
    return b, inv_w


def pl_segment(b: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Largest s with b_s <= q (0 if q is below b_0)."""
    s = np.searchsorted(b, q.astype(np.uint64), side="right") - 1
    return np.maximum(s, 0)


def pl_x(b, inv_w, q):
    """fp32 local coordinate of q in its segment: fp32(fp64(q - b_s)) * inv_w_s."""
    q = q.astype(np.uint64)
    s = pl_segment(b, q)
    base = b[s]
    diff = np.where(q >= base, q - base, np.uint64(0))
    x = diff.astype(np.float64).astype(np.float32) * inv_w[s]  # fp32 multiply
    return s, x.astype(np.float32)


def pl_fit(keys, leaf, segments: int):
    """Least-squares line per segment (closed form, fp64), stored as fp32."""
    b, inv_w = pl_breakpoints(keys, segments)
    s, x = pl_x(b, inv_w, keys)
    y = leaf.astype(np.float64)
    xd = x.astype(np.float64)
    slope = np.zeros(segments, np.float64)
    icpt = np.zeros(segments, np.float64)
    for j in range(segments):
        m = s == j
        if not m.any():
            continue
        xs, ys = xd[m], y[m]
        if xs.size >= 2 and np.ptp(xs) > 0:
            A = np.stack([xs, np.ones_like(xs)], axis=1)
            (a, c), *_ = np.linalg.lstsq(A, ys, rcond=None)
        else:
            a, c = 0.0, ys.mean()
        slope[j], icpt[j] = a, c
    return b, inv_w, slope.astype(np.float32), icpt.astype(np.float32)


def pl_predict(b, inv_w, slope, icpt, q, L: int) -> np.ndarray:
    """leaf_hat = rint(clamp(fp32(fp32(slope*x) + icpt), 0, L-1))."""
    s, x = pl_x(b, inv_w, q)
    pred = (slope[s] * x).astype(np.float32)      # fp32 multiply, rounded
    pred = (pred + icpt[s]).astype(np.float32)     # fp32 add, rounded
    pred = np.clip(pred, np.float32(0), np.float32(L - 1))
    return np.rint(pred).astype(np.int64)


# ---------------------------------------------------------- MLP model

def mlp_unpack(p: np.ndarray):
    p = np.asarray(p, np.float64)
    assert p.size == N_PARAMS
    o = 0
    W1 = p[o:o + H]; o += H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H   # W2[j, k]: unit j of layer 2 from unit k
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def mlp_forward(p, x):
    W1, b1, W2, b2, w3, b3 = mlp_unpack(p)
    x = np.asarray(x, np.float64)
    z1 = np.outer(x, W1) + b1           # (B, H)
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2                 # (B, H)
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3                    # (B,)
    return y, (x, z1, h1, z2, h2)


def mlp_loss(p, x, t):
    y, _ = mlp_forward(p, x)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def mlp_grad(p, x, t):
    """Gradient of the mean squared error by backpropagation (fp64)."""
    W1, b1, W2, b2, w3, b3 = mlp_unpack(p)
    y, (x, z1, h1, z2, h2) = mlp_forward(p, x)
    B = x.size
    dy = 2.0 * (y - np.asarray(t, np.float64)) / B          # (B,)
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    dh2 = np.outer(dy, w3)
    dz2 = dh2 * (z2 > 0)
    g_W2 = dz2.T @ h1                                        # (H, H)
    g_b2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    g_W1 = dz1.T @ x
    g_b1 = dz1.sum(axis=0)
    return np.concatenate([g_W1, g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])


MLP_STAGE1 = 64  # breakpoints of the MLP's first stage


def mlp_stage1(keys: np.ndarray):
    """The first stage's breakpoints: the PL breakpoints of 64 segments."""
    return pl_breakpoints(keys, MLP_STAGE1)


def mlp_x(keys_or_q, b, inv_w):
    """The MLP's input, in fp32 as the GPU computes it: segment s of q among
    the first stage's breakpoints, u = min(fp32(fp64(q - b_s)) * inv_w_s, 1),
    x = fp32(fp32(s) + u) * (1/64)."""
    q = np.asarray(keys_or_q).astype(np.uint64)
    s, u = pl_x(b, inv_w, q)
    u = np.minimum(u, np.float32(1.0)).astype(np.float32)
    t = (s.astype(np.float32) + u).astype(np.float32)
    return (t * np.float32(1.0 / MLP_STAGE1)).astype(np.float32)


def max_error(leaf_hat: np.ndarray, leaf: np.ndarray) -> int:
    return int(np.max(np.abs(leaf_hat.astype(np.int64) - leaf.astype(np.int64)))) if leaf.size else 0


def range_errors(leaf_hat: np.ndarray, leaf: np.ndarray, L: int, ranges: int = 256) -> np.ndarray:
    """Largest |leaf_hat - leaf| per range r of leaf_hat, where range r holds
    leaf_hat in [r*L/ranges, (r+1)*L/ranges)."""
    h = leaf_hat.astype(np.int64)
    r = (h * ranges) // L
    d = np.abs(h - leaf.astype(np.int64))
    out = np.zeros(ranges, np.int64)
    np.maximum.at(out, r, d)
    return out


def window_leaf(leaf_max: np.ndarray, q, leaf_hat, err: int):
    """The leaf whose key range holds q, searched only in the window
    [leaf_hat - err, leaf_hat + err]; -1 where q's leaf lies outside it
    (the fallback case)."""
    L = leaf_max.size
    q = np.asarray(q).astype(np.uint64)
    lo = np.clip(leaf_hat - err, 0, L - 1)
    hi = np.clip(leaf_hat + err, 0, L - 1)
    true_leaf = np.minimum(np.searchsorted(leaf_max, q, side="left"), L - 1)
    ok = (true_leaf >= lo) & (true_leaf <= hi)
    return np.where(ok, true_leaf, -1)
