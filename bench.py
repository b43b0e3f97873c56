#!/usr/bin/env python3
"""Benchmark of the batched level-wise B+ tree point search on GB300.

Workload (default): one static tree of 2^24 distinct uniform uint64 keys,
fanout 32, uint64 rank values; batches of 2^20 point lookups at 90% hits
(uniform).  One step = one pass of the whole search path over one batch:
the on-device partition of the batch by key, then the level-wise descent, leaf
probe and scatter to input order.  Inputs are resident in HBM when a step
starts.  By default two steps are in flight: steps alternate between two
streams, each with its own workspace and outputs, and the tree's launch
shapes are capped (bt_tree_set_corun) so that one batch's partition runs
beside the previous batch's descent; the same steps one at a time on one
stream are reported beside it (``one_stream``).  By default the L2 is not
flushed between steps: the 282 MB tree is
larger than the 129 MB L2 and four batches rotate, so a step finds its batch
evicted and only the hot upper tree levels cached, as in steady serving;
the same loop with a 256 MB buffer overwritten before every step is
reported beside it (``l2_write_flushed``).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(the plain pointer B+ tree searched one query at a time) on the host cores
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2604_21117_gb300 import workloads as W  # noqa: E402

METRIC = "batched B+tree lookups/s at 2^24 keys, learned vs plain; p99 µs; HBM GB/s"
UNIT = "lookups/s"
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes (read + write) of one k_descend launch on the default workload,
# from one ncu capture of it (summarised under profiles/); valid only while
# the descent's source (desc_pipe.cu and descent.cuh) hashes to the same value.
NCU_DESCEND_TRAFFIC = {"descend_src_sha256": "9f8dc9871dc2dfda", "bytes_per_launch": 223253760}


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--keys", type=int, default=1 << 24)
    p.add_argument("--batch", type=int, default=1 << 20)
    p.add_argument("--fanout", type=int, default=32)
    p.add_argument("--hit", type=float, default=0.9)
    p.add_argument("--zipf", type=float, default=None)
    p.add_argument("--sort-bits", type=int, default=-1)
    p.add_argument("--streams", type=int, choices=[1, 2], default=2,
                   help="steps in flight: 2 alternates two streams (each with its own workspace and "
                        "outputs), so one batch's partition runs beside the previous batch's descent")
    p.add_argument("--corun", default="0,1",
                   help="resident blocks per SM of the descent and the partition with --streams 2 "
                        "(0 = as many as fit)")
    p.add_argument("--l2", choices=["write", "read", "none"], default="none",
                   help="between timed steps: nothing (default: the 282 MB tree already exceeds the L2 and "
                        "the batches rotate), overwrite a 256 MB buffer, or read one")
    p.add_argument("--staging", type=int, default=2,
                   help="descent: 2 = pipelined (bulk-copy leaf staging overlapped with the next chunk), "
                        "0 = synchronous 16-byte cp.async, 1 = synchronous bulk copy")
    p.add_argument("--inner", type=int, default=2,
                   help="pipelined: inner levels through L1 (0), staged (1), staged only for partitioned batches (2)")
    p.add_argument("--ballot", type=int, default=0, help="pipelined: leaf rank by binary search (0) or ballot (1)")
    p.add_argument("--l2-window", type=int, default=64 << 20,
                   help="bytes of the L2 persistence window on the inner levels (0 = none)")
    p.add_argument("--no-designs", action="store_true", help="skip the A/B of the descent designs")
    p.add_argument("--lane-queries", type=int, default=1, help="queries per lane of the descent (1 or 2)")
    p.add_argument("--warps", type=int, default=0, help="descent warps per block (0 = library default)")
    p.add_argument("--pin", type=int, default=-1, help="pinned top-level bytes (-1 = library default)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip e2e / small-batch latency legs")
    p.add_argument("--no-learned", action="store_true", help="skip the learned-vs-plain leg")
    p.add_argument("--no-batching", action="store_true", help="skip the multi-tree batching leg")
    p.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    p.add_argument("--no-range", action="store_true", help="skip the range-partitioned leg")
    p.add_argument("--no-paper-keys", action="store_true", help="skip the 32-byte-key leg")
    p.add_argument("--no-sweeps", action="store_true", help="skip the batch-size and tree-size sweeps")
    return p.parse_args(argv)


# ------------------------------------------------------------ workload

def workload_name(a) -> str:
    dist = "uniform" if a.zipf is None else f"Zipf(s={a.zipf})"
    return (f"plain level-wise search: {a.keys} distinct uniform uint64 keys, fanout {a.fanout}, "
            f"uint64 values, batch {a.batch}, {int(round(a.hit * 100))}% hits, {dist} queries")


def workload_config(a, world: int) -> dict:
    """The workload both arms run (the same dict in both JSON lines)."""
    return {"workload": workload_name(a), "keys": a.keys, "fanout": a.fanout, "batch": a.batch,
            "hit_frac": a.hit, "query_dist": "uniform" if a.zipf is None else f"zipf{a.zipf}",
            "l2": ("GPU arm: not flushed between steps (the 282 MB tree exceeds the 129 MB L2; batches "
                   "rotate); a 256 MB write-flushed loop is reported beside it" if a.l2 == "none" else
                   f"GPU arm: L2 {a.l2}-flushed (256 MB) before every timed step"),
            "parallelism": (f"replicas: one batch of {world} x {a.batch} queries split evenly over {world} GPUs, "
                            "each holding the whole tree" if world > 1 else "single GPU")}


def make_tree_data(a):
    keys = W.uniform_keys(a.keys, 64, seed=W.SEED_BASE + 2)
    vals = W.rank_values(a.keys, 64)
    return keys, vals


def make_batches(a, keys, count: int, rank: int = 0, world: int = 1):
    """`count` batches of a.batch queries for this rank.  With several ranks
    every rank draws the same global batch of world * a.batch queries and
    takes its even slice of it (the replicas' split of one batch)."""
    from paper_2604_21117_gb300.replicas import even_slice
    out = []
    for i in range(count):
        g = W.make_queries(keys, a.batch * world, a.hit, seed=W.SEED_BASE + 2 + 1000 * (i + 1), width_bits=64,
                           zipf_s=a.zipf)
        s, c = even_slice(g.size, world, rank)
        out.append(np.ascontiguousarray(g[s:s + c]))
    return out


def level_node_max(keys: np.ndarray, level_nodes: list[int]) -> list[np.ndarray]:
    """Largest key under every node of every level (root first), from the
    sorted keys and the level sizes of the even bulk load."""
    n = keys.size
    L = level_nodes[-1]
    base, rem = divmod(n, L)
    i = np.arange(L, dtype=np.int64)
    ends = (i + 1) * base + np.minimum(i + 1, rem)
    node_max = keys[ends - 1]
    out = [node_max]
    for l in range(len(level_nodes) - 2, -1, -1):
        N, C = level_nodes[l], level_nodes[l + 1]
        b, r = divmod(C, N)
        j = np.arange(N, dtype=np.int64)
        node_max = node_max[(j + 1) * b + np.minimum(j + 1, r) - 1]
        out.insert(0, node_max)
    return out


def touched(keys: np.ndarray, level_nodes: list[int], m: int, q: np.ndarray, val_bytes: int = 8):
    """Distinct nodes per level on the batch's root-to-leaf paths and
    distinct 32-byte leaf-value sectors its hits read."""
    q = q.astype(np.uint64)
    maxes = level_node_max(keys, level_nodes)
    counts = []
    leaf = None
    for l, mx in enumerate(maxes):
        idx = np.minimum(np.searchsorted(mx, q, side="left"), level_nodes[l] - 1)
        counts.append(int(np.unique(idx).size))
        leaf = idx
    n = keys.size
    L = level_nodes[-1]
    base, rem = divmod(n, L)
    first = leaf * base + np.minimum(leaf, rem)
    rank = np.searchsorted(keys, q, side="left")
    inb = rank < n
    hit = np.zeros(q.size, bool)
    hit[inb] = keys[rank[inb]] == q[inb]
    slot = rank[hit] - first[hit]
    sectors = np.unique(((leaf[hit] * m + slot) * val_bytes) // 32).size
    return counts, int(sectors)


def rank_touched(n: int, level_nodes: list[int], m: int, rank: np.ndarray, hit: np.ndarray, val_bytes: int):
    """touched() for queries given by their lower-bound rank among the n sorted
    keys (any key type): a query goes to the first node whose largest key has
    rank >= its own, since q <= key[r] exactly when lower_bound(q) <= r.
    Returns the distinct nodes per level and the distinct 32-byte value
    sectors read by the hits."""
    node_max_rank = [x.astype(np.int64) for x in level_node_max(np.arange(n, dtype=np.uint64), level_nodes)]
    counts = [int(np.unique(np.minimum(np.searchsorted(mr, rank), mr.size - 1)).size) for mr in node_max_rank]
    leaf = np.minimum(np.searchsorted(node_max_rank[-1], rank), node_max_rank[-1].size - 1)
    first = np.concatenate([[0], node_max_rank[-1][:-1] + 1])
    slot = rank - first[leaf]
    sect = int(np.unique(((leaf[hit] * m + slot[hit]) * val_bytes) // 32).size)
    return counts, sect


def descend_algorithmic_bytes(counts, sectors, m, kb, vb, B) -> int:
    """Bytes the descent must move at least: every distinct node's key block
    once, every distinct value sector once, the sorted queries and their
    positions in, the values and found flags out."""
    return sum(counts) * m * kb + sectors * 32 + B * (kb + 4) + B * (vb + 1)


# ------------------------------------------------------------- helpers

def iqm(x) -> float:
    """Interquartile mean: the mean of the middle half of the sorted samples
    (the paper's Eq. 2 reports this statistic)."""
    s = sorted(x)
    n = len(s)
    lo, hi = n // 4, n - n // 4
    mid = s[lo:hi] if hi > lo else s
    return float(sum(mid) / len(mid))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(p[1]) for _, p in self.samples if num(p[1]) is not None]
        mx = [num(p[2]) for _, p in self.samples if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, p in self.samples:
            for nm, v in zip(names, p[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def src_sha256() -> str:
    """Hash of the descent's source: the pipelined kernel's file and the
    helpers it includes."""
    h = hashlib.sha256()
    for name in ("desc_pipe.cu", "descent.cuh"):
        with open(os.path.join(ROOT, "paper_2604_21117_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------ dist

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(world: int, backend: str):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def reduce_max(x: float, world: int, device=None) -> float:
    """Max of a float over the ranks (identity at world size 1)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------- CPU oracle

CPU_SAMPLE = 1 << 16  # queries per CPU-oracle repeat, in both arms


def cpu_model() -> str:
    """The host CPU's model name (or its implementer/part codes on Arm)."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        return "unknown"
    for line in info.splitlines():
        if line.lower().startswith(("model name", "hardware")):
            return line.split(":", 1)[1].strip()
    imp = part = None
    for line in info.splitlines():
        if line.startswith("CPU implementer"):
            imp = line.split(":", 1)[1].strip()
        elif line.startswith("CPU part"):
            part = line.split(":", 1)[1].strip()
    return f"Arm implementer {imp}, part {part}" if imp else "unknown"


def cpu_baseline(keys, vals, m, q, repeats: int = 100):
    """The CPU oracle (pointer B+ tree, each query descending from the root)
    on the first CPU_SAMPLE queries of a batch, split evenly over T threads
    for T in {1, 2, 4, 8, 16, all cores}; every T timed `repeats` times and
    summarised by the IQM (the paper's Eq. 2) and the interquartile range,
    as the paper's 1- and 16-thread CPU comparison (Sec. V-C, V-F)."""
    import oracle
    t0 = time.perf_counter()
    tree = oracle.OracleTree(keys, vals, m)
    build_s = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    sample = q[: min(q.size, CPU_SAMPLE)]
    threads = sorted({1, 2, 4, 8, 16, cores} & set(range(1, cores + 1)) | {cores})
    table = {}
    for T in threads:
        tree.search_mt(sample, T)  # warm-up
        ts = []
        for _ in range(repeats):
            t1 = time.perf_counter()
            tree.search_mt(sample, T)
            ts.append(time.perf_counter() - t1)
        q25, q75 = np.percentile(ts, [25, 75])
        table[str(T)] = {"lookups_per_s": sample.size / iqm(ts), "iqm_ms": 1e3 * iqm(ts),
                         "iqr_ms": 1e3 * float(q75 - q25)}
    tree.close()
    return {"value": table[str(cores)]["lookups_per_s"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "value_1thread": table["1"]["lookups_per_s"], "threads": table,
            "cpu_model": cpu_model(), "hardware_concurrency": cores,
            "sample": (f"the first {sample.size} queries of one batch, split evenly over T threads; "
                       f"{repeats} repeats per T, IQM (Eq. 2) and IQR; oracle tree build {build_s:.1f} s "
                       "untimed; value = all cores")}


# ------------------------------------------------------ designs leg

DESIGNS = (
    ("pipelined, inner staged, binary search, L2 window", dict(staging=2, inner=1, ballot=0, l2=64 << 20, lq=1)),
    ("pipelined, inner staged, ballot + popc, L2 window", dict(staging=2, inner=1, ballot=1, l2=64 << 20, lq=1)),
    ("pipelined, inner through L1, binary search, L2 window", dict(staging=2, inner=0, ballot=0, l2=64 << 20, lq=1)),
    ("pipelined, inner staged, binary search, no L2 window", dict(staging=2, inner=1, ballot=0, l2=0, lq=1)),
    ("synchronous cp.async (every level staged, waited)", dict(staging=0, inner=0, ballot=0, l2=0, lq=1)),
    ("synchronous bulk copy", dict(staging=1, inner=0, ballot=0, l2=0, lq=1)),
    ("synchronous, two queries per lane", dict(staging=0, inner=0, ballot=0, l2=0, lq=2)),
    # not the paper's method: no sort, each warp takes 32 queries as they come
    ("no sort: the batch as given, pipelined, inner through L1", dict(staging=2, inner=0, ballot=0, l2=64 << 20,
                                                                      lq=1, sort_bits=0)),
)


def designs_leg(a, bt, tree, dq, out_v, out_f, ws, nb, stream, alg, pool, steps: int = 40):
    """A/B of the descent designs on the same batches (sorted, except the
    design that skips the sort): mean descent and step time (CUDA events),
    and the descent's achieved GB/s of the sorted batch's algorithmic bytes;
    each design's results are checked against the default design's on the
    last batch."""
    import torch
    B = a.batch
    peak, _ = measured_peaks()
    out = {}
    ref_v = ref_f = None
    for label, d in DESIGNS:
        bt.bt_tree_set_staging(tree.handle, d["staging"])
        bt.bt_tree_set_lane_queries(tree.handle, d["lq"])
        bt.bt_tree_set_descent(tree.handle, d["inner"], d["ballot"])
        bt.bt_tree_set_l2_window(tree.handle, d["l2"])
        sb = d.get("sort_bits", a.sort_bits)
        for i in range(3):
            bt.bt_search_batch_ex(tree.handle, dq[i % pool], B, out_v, out_f, ws, nb, sb, None, stream)
        ev = []
        for i in range(steps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[1].record(stream)  # create it; recorded again inside the call
            e[0].record(stream)
            bt.bt_search_batch_ex(tree.handle, dq[i % pool], B, out_v, out_f, ws, nb, sb, None, stream, e[1])
            e[2].record(stream)
            ev.append(e)
        torch.cuda.synchronize()
        desc = [e[1].elapsed_time(e[2]) for e in ev]
        step = [e[0].elapsed_time(e[2]) for e in ev]
        byts = statistics.fmean(alg[i % pool][2] for i in range(steps))
        gbs = byts / (statistics.fmean(desc) / 1e3) / 1e9
        v = out_v.cpu().numpy()
        f = out_f.cpu().numpy()
        if ref_v is None:
            ref_v, ref_f, same = v, f, True
        else:
            same = bool(np.array_equal(v, ref_v) and np.array_equal(f, ref_f))
        out[label] = {"descend_us": 1e3 * statistics.fmean(desc), "step_us": 1e3 * statistics.fmean(step),
                      "descend_gbs": gbs, "descend_frac_of_peak": gbs / peak, "same_results": same}
    bt.bt_tree_set_staging(tree.handle, a.staging)
    bt.bt_tree_set_lane_queries(tree.handle, a.lane_queries)
    bt.bt_tree_set_descent(tree.handle, a.inner, a.ballot)
    bt.bt_tree_set_l2_window(tree.handle, a.l2_window)
    return out


# ------------------------------------------------------ learned leg

# Device cycles of the spin each small timed call is queued behind (about
# 50 us at 2 GHz: longer than the host takes to submit the call).
SPIN_CYCLES = 100_000


def _time_calls(fn, steps, flush, stream, submit=False):
    """Per-call CUDA-event times (us) of fn(): the device's time for the call.
    With `flush`, the L2 is flushed before each call (the 256 MB write also
    keeps the device busy while the host submits the call); without it each
    call is queued behind a short device spin, so that the host's submission
    falls outside the timed region.  submit=True times without the spin:
    submission plus device time, as a caller that waits on each call sees."""
    import torch
    out = []
    with torch.cuda.stream(stream):
        for i in range(steps):
            if flush is not None:
                flush.fill_(i)
            elif not submit:
                torch.cuda._sleep(SPIN_CYCLES)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            out.append((e0, e1))
            if flush is None and i % 50 == 49:
                torch.cuda.synchronize()  # keeps the queue of spins short
    torch.cuda.synchronize()
    return sorted(1e3 * x.elapsed_time(y) for x, y in out)


def learned_leg(a, bt, flush, stream):
    """Plain level-wise search against the learned leaf predictor (PL with
    256 segments, MLP 1-32-32-1) on 2^24 keys from a mixture of three
    lognormals (the configured workload) and, for contrast, 2^24 uniform
    keys; fanout 32, 90% hits, batches of 1024 and 2^20."""
    n = 1 << 24
    out = {}
    for label, keys in (("lognormal", lambda: W.lognormal_mixture_keys(n, seed=W.SEED_BASE + 4)),
                        ("uniform", lambda: W.uniform_keys(n, 64, seed=W.SEED_BASE + 2))):
        out[label] = _learned_case(bt, flush, stream, keys(), label)
    return out


def _learned_case(bt, flush, stream, keys, label):
    import torch
    n = keys.size
    vals = W.rank_values(n, 64)
    tree = bt.BTree(keys, vals, 32)
    res = {"workload": f"{n} {label} uint64 keys, fanout 32, 90% hits"}
    t0 = time.perf_counter()
    pl = bt.bt_model_train(tree.handle, bt.BT_MODEL_PL, segments=256)
    t_pl = time.perf_counter() - t0
    t0 = time.perf_counter()
    mlp = bt.bt_model_train(tree.handle, bt.BT_MODEL_MLP, h_init=W.mlp_init_params(W.SEED_BASE + 5),
                            steps=2000, batch=16384, lr=2e-3, seed=W.SEED_BASE + 6)
    t_mlp = time.perf_counter() - t0
    ipl, imlp = bt.bt_model_get_info(pl), bt.bt_model_get_info(mlp)
    res["models"] = {"pl256": {"max_err_leaves": int(ipl.max_err), "fit_s": t_pl},
                     "mlp": {"max_err_leaves": int(imlp.max_err), "train_s": t_mlp, "steps": 2000,
                             "batch": 16384, "final_mse": float(imlp.final_loss)}}
    for B, steps in ((1024, 300), (1 << 20, 50)):
        q = torch.from_numpy(W.make_queries(keys, B, 0.9, seed=W.SEED_BASE + 7 + B, width_bits=64)).cuda()
        nb = tree.workspace_bytes(B)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        outs = {k: tree.alloc_outputs(B) for k in ("plain", "pl256", "mlp")}
        calls = {
            "plain": lambda: bt.bt_search_batch(tree.handle, q, B, *outs["plain"], ws, nb, stream),
            "pl256": lambda: bt.bt_learned_search_batch(tree.handle, pl, q, B, *outs["pl256"], ws, nb, stream),
            "mlp": lambda: bt.bt_learned_search_batch(tree.handle, mlp, q, B, *outs["mlp"], ws, nb, stream),
        }
        row = {}
        for name, fn in calls.items():
            for _ in range(3):
                fn()
            us = _time_calls(fn, steps, flush if B > 4096 else None, stream)
            row[name] = {"lookups_per_s": B / (statistics.fmean(us) / 1e6), "p50_us": us[len(us) // 2],
                         "p99_us": us[min(len(us) - 1, int(0.99 * len(us)))]}
        pv, pf = (x.cpu().numpy() for x in outs["plain"])
        for name in ("pl256", "mlp"):
            lv, lf = (x.cpu().numpy() for x in outs[name])
            row[name]["bit_exact_vs_plain"] = bool(np.array_equal(lv, pv) and np.array_equal(lf, pf))
            row[name]["speedup_vs_plain"] = row[name]["lookups_per_s"] / row["plain"]["lookups_per_s"]
        # share of warps the model window served (the rest fell back to the descent)
        sq = torch.empty_like(q)
        si = torch.empty(B, dtype=torch.int32, device="cuda")
        bt.bt_sort_batch(tree.handle, q, B, -1, sq, si, ws, nb, stream)
        for name, mdl in (("pl256", pl), ("mlp", mlp)):
            st = torch.zeros(2, dtype=torch.int64, device="cuda")
            v, f = tree.alloc_outputs(B)
            bt.bt_learned_descend_sorted(tree.handle, mdl, sq, si, B, v, f, st, stream)
            s0, s1 = (int(x) for x in st.cpu().numpy())
            row[name]["window_served_frac"] = s0 / max(1, s0 + s1)
        res[f"batch_{B}"] = row
    bt.bt_model_free(pl)
    bt.bt_model_free(mlp)
    tree.close()
    return res


# ------------------------------------------------------ paper key format leg

def _steps_in_turn(bt, tree, q, B, out, ws, nb, steps: int = 100):
    """Lookups/s of `steps` searches of one batch issued back to back with
    nothing flushed between them: on one stream, and with two in flight on
    two streams (each with its own workspace and outputs, the partition held
    to one block per SM, as the main loop's two-in-flight steps)."""
    import torch
    outs = [out, tree.alloc_outputs(B)]
    wss = [ws, torch.empty_like(ws)]
    sts = [torch.cuda.Stream(), torch.cuda.Stream()]
    res = {}
    for label, nst, corun in (("one_stream", 1, (0, 0)), ("two_in_flight", 2, (0, 1))):
        bt.bt_tree_set_corun(tree.handle, *corun)
        for i in range(4):
            bt.bt_search_batch(tree.handle, q, B, *outs[i % nst], wss[i % nst], nb, sts[i % nst])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sts[0])
        sts[1].wait_event(e0)
        for i in range(steps):
            bt.bt_search_batch(tree.handle, q, B, *outs[i % nst], wss[i % nst], nb, sts[i % nst])
        sts[0].wait_stream(sts[1])
        e1.record(sts[0])
        torch.cuda.synchronize()
        res[label] = {"lookups_per_s": B * steps / (e0.elapsed_time(e1) / 1e3),
                      "us_per_batch": 1e3 * e0.elapsed_time(e1) / steps}
    bt.bt_tree_set_corun(tree.handle, 0, 0)
    res["note"] = "nothing flushed between steps; two_in_flight: partition at one block per SM"
    return res


def paper_keys_leg(a, bt, flush, stream, peak):
    """The paper's own tree and key format (Sec. V): 2^20 entries of 32-byte
    keys (lexicographic byte order) with 8-byte data, fanout 16; batches of
    1000 queries (the paper's batch size) and 2^20, uniform over the keys,
    90% hits.  Lookups/s through bt_search_batch, the descent's achieved
    bandwidth against its algorithmic bytes, a check of every result against
    numpy's binary search over the keys (byte order), and the byte-key
    oracle on the host cores as this workload's CPU baseline."""
    import torch
    n, m = 1 << 20, 16
    keys = W.byte_keys(n, 32, seed=W.SEED_BASE + 8)
    vals = W.rank_values(n, 64)
    kv = keys.view("V32").ravel()
    tree = bt.BTree(keys, vals, m)
    res = {"workload": f"{n} distinct 32-byte keys (uniform random bytes), 8-byte values, fanout {m}, "
                       "90% hits, uniform queries"}
    for B, steps in ((1000, 300), (1 << 20, 50)):
        qh = W.make_byte_queries(keys, B, 0.9, seed=W.SEED_BASE + 9 + B)
        q = torch.from_numpy(qh).cuda()
        nb = tree.workspace_bytes(B)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
        v, f = tree.alloc_outputs(B)
        fn = lambda: bt.bt_search_batch(tree.handle, q, B, v, f, ws, nb, stream)
        for _ in range(3):
            fn()
        us = _time_calls(fn, steps, flush if B > 4096 else None, stream)
        rank = np.searchsorted(kv, qh.view("V32").ravel())
        hit = rank < n
        hit[hit] = kv[rank[hit]] == qh.view("V32").ravel()[hit]
        want_v = np.full(B, np.uint64(2**64 - 1))
        want_v[hit] = vals[rank[hit]]
        row = {"lookups_per_s": B / (statistics.fmean(us) / 1e6), "p50_us": us[len(us) // 2],
               "p99_us": us[min(len(us) - 1, int(0.99 * len(us)))],
               "correct": bool(np.array_equal(v.cpu().numpy(), want_v) and
                               np.array_equal(f.cpu().numpy(), hit.astype(np.uint8)))}
        if B > 4096:
            row["l2"] = "flushed before every call"
            row["steps_in_turn"] = _steps_in_turn(bt, tree, q, B, (v, f), ws, nb)
            # the descent alone on the batch partitioned on log2 B bits, against its
            # algorithmic bytes
            sq = torch.empty_like(q)
            si = torch.empty(B, dtype=torch.int32, device="cuda")
            bt.bt_sort_batch(tree.handle, q, B, B.bit_length() - 1, sq, si, ws, nb, stream)
            dfn = lambda: bt.bt_descend_sorted(tree.handle, sq, si, B, v, f, None, stream)
            dus = _time_calls(dfn, steps, flush, stream)
            counts, sect = rank_touched(n, tree.level_nodes, m, rank, hit, 8)
            alg = descend_algorithmic_bytes(counts, int(sect), m, 32, 8, B)
            d_mean = statistics.fmean(dus)
            row["descend_us"] = d_mean
            row["roofline"] = {"bound": "hbm", "achieved": alg / (d_mean / 1e6) / 1e9, "peak": peak,
                               "unit": "GB/s", "frac": alg / (d_mean / 1e6) / 1e9 / peak,
                               "algorithmic_bytes_per_launch": alg, "distinct_nodes_per_level": counts}
        # the same search over the paper's node layout (Eq. 1: whole nodes of 40 m bytes)
        bt.bt_paper_layout_build(tree.handle)
        pfn = lambda: bt.bt_paper_search_batch(tree.handle, q, B, v, f, ws, nb, stream)
        for _ in range(3):
            pfn()
        pus = _time_calls(pfn, steps, flush if B > 4096 else None, stream)
        prow = {"lookups_per_s": B / (statistics.fmean(pus) / 1e6), "p50_us": pus[len(pus) // 2],
                "correct": bool(np.array_equal(v.cpu().numpy(), want_v) and
                                np.array_equal(f.cpu().numpy(), hit.astype(np.uint8)))}
        if B > 4096:
            pdfn = lambda: bt.bt_paper_descend_sorted(tree.handle, sq, si, B, v, f, stream)
            pdus = _time_calls(pdfn, steps, flush, stream)
            nbytes = bt.bt_paper_node_bytes(m, bt.BT_B32)
            palg = sum(counts) * nbytes + B * (32 + 4) + B * (8 + 1)
            pd = statistics.fmean(pdus)
            prow["descend_us"] = pd
            prow["roofline"] = {"bound": "hbm", "achieved": palg / (pd / 1e6) / 1e9, "peak": peak, "unit": "GB/s",
                                "frac": palg / (pd / 1e6) / 1e9 / peak, "algorithmic_bytes_per_launch": palg,
                                "node_bytes": nbytes}
        row["paper_layout"] = prow
        res[f"batch_{B}"] = row
    tree.close()
    # CPU baseline for this workload: the byte-key oracle, all host cores
    from oracle.bytes_keys import OracleBytesTree
    o = OracleBytesTree(keys, vals, m)
    sample = W.make_byte_queries(keys, 1 << 18, 0.9, seed=W.SEED_BASE + 10)
    t0 = time.perf_counter()
    o.search_mt(sample, os.cpu_count() or 1)
    dt = time.perf_counter() - t0
    res["cpu_baseline"] = {"value": sample.shape[0] / dt, "unit": "lookups/s", "cores": os.cpu_count() or 1,
                           "kind": "oracle", "sample": f"{sample.shape[0]} queries of the same mix"}
    o.close()
    return res


# ------------------------------------------------------ sweeps

def sweep_leg(a, bt, stream, keys, vals, tree):
    """The configured sweeps: batch sizes 1, 16, 64, 256, 1024 and 2^20 on the
    2^24-key tree (uniform and Zipf(1.1) queries, 90% hits), and tree sizes
    10 to 2e7 keys (fanout 32) at batch 1024.  Lookups/s and p50/p99 of
    bt_search_batch per call (the device's time: small calls are queued
    behind a device spin, see _time_calls), every result checked against
    numpy's binary search over the keys."""
    import torch

    def run(t, k, v, B, z, seed, calls):
        qh = W.make_queries(k, B, 0.9, seed=seed, width_bits=64, zipf_s=z)
        q = torch.from_numpy(qh).cuda()
        nb = t.workspace_bytes(B)
        ws = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
        ov, of = t.alloc_outputs(B)
        fn = lambda: bt.bt_search_batch(t.handle, q, B, ov, of, ws, nb, stream)
        for _ in range(3):
            fn()
        us = _time_calls(fn, calls, None, stream)
        pos = np.searchsorted(k, qh)
        hit = (pos < k.size) & (k[np.minimum(pos, k.size - 1)] == qh)
        ok = bool(np.array_equal(of.cpu().numpy().astype(bool), hit) and
                  np.array_equal(ov.cpu().numpy()[hit], v[pos[hit]]))
        return {"lookups_per_s": B / (statistics.fmean(us) / 1e6), "p50_us": us[len(us) // 2],
                "p99_us": us[min(len(us) - 1, int(0.99 * len(us)))], "correct": ok}

    out = {"timing": "device time per call: each call queued behind a device spin, so that the host's "
                     "submission is not timed",
           "batch_sweep": {"workload": f"{keys.size} uniform uint64 keys, fanout {a.fanout}, 90% hits"},
           "tree_sweep": {"workload": "uniform uint64 keys, fanout 32, batch 1024 uniform queries, 90% hits"}}
    for dist, z in (("uniform", None), ("zipf1.1", 1.1)):
        row = {}
        for B in (1, 16, 64, 256, 1024, 1 << 20):
            row[f"b{B}"] = run(tree, keys, vals, B, z, W.SEED_BASE + 20 + B, 30 if B > 4096 else 300)
        out["batch_sweep"][dist] = row
    for n in (10, 1000, 100_000, 1_000_000, 20_000_000):
        k = W.uniform_keys(n, 64, seed=W.SEED_BASE + 30 + n)
        v = W.rank_values(n, 64)
        t = bt.BTree(k, v, 32)
        out["tree_sweep"][f"n{n}"] = run(t, k, v, 1024, None, W.SEED_BASE + 31, 300) | {"height": t.height}
        t.close()
    return out


# ------------------------------------------------------ batching leg

def _work_list(bt, keysets, nbatches, seed):
    """A work list of nbatches batches (sizes log-uniform in 1..1024) over the
    trees, Zipf(0.9) queries with 80% hits: (descriptors, flat queries)."""
    g = W.rng(seed)
    counts = W.log_uniform_batch_sizes(nbatches, seed=seed + 1)
    tids = g.integers(0, len(keysets), size=nbatches)
    pools = {}
    for ti in range(len(keysets)):
        need = int(counts[tids == ti].sum())
        pools[ti] = W.make_queries(keysets[ti], need, 0.8, seed=seed + 10 + ti, width_bits=64, zipf_s=0.9)
    used = {ti: 0 for ti in pools}
    desc = np.zeros(nbatches, bt.BATCH_DESC_DTYPE)
    parts, off = [], 0
    for b in range(nbatches):
        c, ti = int(counts[b]), int(tids[b])
        parts.append(pools[ti][used[ti]:used[ti] + c])
        used[ti] += c
        desc[b] = (ti, c, off)
        off += c
    return desc, np.concatenate(parts)


def batching_leg(a, bt, stream, nbatches: int = 10_000):
    """One graph-captured persistent launch over a work list of many small
    batches addressed to 4 resident trees (1e3, 1e5, 1e6, 2e7 uint64 keys,
    fanout and launch settings chosen per tree by the autotuner, the
    forest's launch shape by the forest autotuner on a separate sample work
    list); batch sizes log-uniform in [1, 1024]; Zipf(0.9) queries with 80%
    hits."""
    import torch
    sizes = [1000, 100_000, 1_000_000, 20_000_000]
    trees, keysets, tunes = [], [], []
    t0 = time.perf_counter()
    for i, n in enumerate(sizes):
        keys = W.uniform_keys(n, 64, seed=W.SEED_BASE + 20 + i)
        vals = W.rank_values(n, 64)
        sample = W.make_queries(keys, 1024, 0.8, seed=W.SEED_BASE + 30 + i, width_bits=64, zipf_s=0.9)
        h, best = bt.bt_autotune(keys, vals, torch.from_numpy(sample).cuda(), sample.size)
        trees.append(bt.BTree(None, None, handle=h))
        keysets.append(keys)
        tunes.append({"keys": n, "fanout": int(best.fanout), "warps_per_block": int(best.warps_per_block),
                      "pin_bytes": int(best.pin_bytes), "staging": int(best.staging),
                      "lane_queries": int(best.lane_queries), "inner_staged": int(best.inner_staged),
                      "sample_us": float(best.us_per_batch)})
    tune_s = time.perf_counter() - t0
    desc, allq = _work_list(bt, keysets, nbatches, W.SEED_BASE + 40)
    total = int(allq.size)
    dq = torch.from_numpy(allq).cuda()
    d_desc = torch.from_numpy(desc.view(np.uint8)).cuda()
    forest = bt.bt_forest_create(trees)
    v = torch.empty(total, dtype=torch.uint64, device="cuda")
    f = torch.empty(total, dtype=torch.uint8, device="cuda")
    wsb = bt.bt_forest_workspace_bytes(nbatches)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    cur = torch.cuda.current_stream()

    def time_graph(reps=20):
        with torch.cuda.stream(s):
            bt.bt_forest_search(forest, d_desc, nbatches, dq, v, f, ws, wsb, 0, s)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            bt.bt_forest_search(forest, d_desc, nbatches, dq, v, f, ws, wsb, 0, torch.cuda.current_stream())
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in ev:
            e0.record(cur)
            graph.replay()
            e1.record(cur)
        torch.cuda.synchronize()
        return sorted(1e3 * x.elapsed_time(y) for x, y in ev)

    us_tree = time_graph()  # each tree's own tuned settings, the forest's default shape
    # the forest autotuner on a separate sample work list (1000 batches, other seed)
    sdesc, sq = _work_list(bt, keysets, 1000, W.SEED_BASE + 90)
    sv = torch.empty(sq.size, dtype=torch.uint64, device="cuda")
    sf = torch.empty(sq.size, dtype=torch.uint8, device="cuda")
    swsb = bt.bt_forest_workspace_bytes(1000)
    sws = torch.empty(swsb, dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    ft = bt.bt_forest_autotune(forest, torch.from_numpy(sdesc.view(np.uint8)).cuda(), 1000,
                               torch.from_numpy(sq).cuda(), sv, sf, sws, swsb)
    ftune_s = time.perf_counter() - t0
    us = time_graph()
    # correctness of the graph replay against the per-tree single-batch path
    vv, ff = v.cpu().numpy(), f.cpu().numpy()
    ok = True
    for b in range(0, nbatches, 97):
        c, o, ti = int(desc[b]["count"]), int(desc[b]["offset"]), int(desc[b]["tree"])
        if c == 0:
            continue
        rv, rf = trees[ti].search(dq[o:o + c])
        ok &= bool(np.array_equal(rv.cpu().numpy(), vv[o:o + c]) and np.array_equal(rf.cpu().numpy(), ff[o:o + c]))
    # the same work list as one bt_search_batch launch sequence per batch
    outs = [trees[int(desc[b]["tree"])].alloc_outputs(max(1, int(desc[b]["count"]))) for b in range(nbatches)]
    wss = {}
    for ti, t in enumerate(trees):
        nbt = t.workspace_bytes(1024)
        wss[ti] = (torch.empty(nbt, dtype=torch.uint8, device="cuda"), nbt)

    def per_batch():
        for b in range(nbatches):
            c, o, ti = int(desc[b]["count"]), int(desc[b]["offset"]), int(desc[b]["tree"])
            if c:
                bt.bt_search_batch(trees[ti].handle, dq[o:o + c], c, *outs[b], *wss[ti], cur)
    per_batch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(cur)
    per_batch()
    e1.record(cur)
    torch.cuda.synchronize()
    per_batch_wall = time.perf_counter() - t0
    per_batch_us = 1e3 * e0.elapsed_time(e1)
    bt.bt_forest_free(forest)
    for t in trees:
        t.close()
    counts = desc["count"]
    return {"workload": f"{nbatches} batches, sizes log-uniform 1..1024, over trees of {sizes} uint64 keys, "
                        "Zipf(0.9) queries, 80% hits",
            "queries": total, "autotune": tunes, "autotune_s": tune_s,
            "forest_tune": {"warps_per_block": int(ft.warps_per_block), "pin_budget": int(ft.pin_budget),
                            "pin_applied": int(ft.pin_applied), "lane_queries": int(ft.lane_queries),
                            "staging": int(ft.staging), "sample_us": float(ft.us), "tune_s": ftune_s,
                            "sample": "1000 batches of the same mix, another seed"},
            "graph_launch": {"lookups_per_s": total / (statistics.fmean(us) / 1e6), "p50_us": us[len(us) // 2],
                             "p99_us": us[min(len(us) - 1, int(0.99 * len(us)))], "launches_per_work_list": 2},
            "graph_launch_tree_settings": {"lookups_per_s": total / (statistics.fmean(us_tree) / 1e6),
                                           "p50_us": us_tree[len(us_tree) // 2]},
            "per_batch_launches": {"lookups_per_s": total / (per_batch_us / 1e6), "device_us": per_batch_us,
                                   "host_wall_s": per_batch_wall, "launches": int((counts > 0).sum())},
            "bit_exact_vs_single_tree_path": ok}


# ------------------------------------------------------- range-split leg

def range_leg(a, bt, keys, vals, dq, ref, stream, steps: int = 30):
    """Range-partitioned trees on one GPU (bt_range_build / bt_range_search):
    the default tree's keys split into P contiguous key ranges, each its own
    tree; a batch is routed to its parts, each part searched, the results
    returned in input order.  Lookups/s per P against the single tree, and
    the results of one batch against the single tree's."""
    import torch
    B = a.batch
    out = {"workload": f"{a.keys} uniform uint64 keys split into P key ranges, fanout {a.fanout}, "
                       f"batches of {B} queries (the default workload's)", "parts": {}}
    for P in (1, 2, 4, 8):
        r = bt.bt_range_build(keys, vals, a.fanout, P, stream=stream)
        nb = bt.bt_range_workspace_bytes(r, B)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        v = torch.empty(B, dtype=torch.uint64, device="cuda")
        f = torch.empty(B, dtype=torch.uint8, device="cuda")
        for i in range(3):
            bt.bt_range_search(r, dq[i % len(dq)], B, v, f, ws, nb, stream)
        torch.cuda.synchronize()
        ev = []
        for i in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bt.bt_range_search(r, dq[i % len(dq)], B, v, f, ws, nb, stream)
            e1.record(stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        us = sorted(1e3 * x.elapsed_time(y) for x, y in ev)
        bt.bt_range_search(r, dq[0], B, v, f, ws, nb, stream)
        torch.cuda.synchronize()
        same = bool(np.array_equal(v.cpu().numpy(), ref[0]) and np.array_equal(f.cpu().numpy(), ref[1]))
        out["parts"][str(P)] = {"lookups_per_s": B / (statistics.fmean(us) / 1e6), "p50_us": us[len(us) // 2],
                                "bit_exact_vs_single_tree": same}
        bt.bt_range_free(r)
    return out


# ------------------------------------------------------- serving leg

def serving_leg(a, bt, rates=(1e6, 5e6, 20e6, 50e6, 100e6), seconds: float = 0.25):
    """Continuous batching under Poisson arrivals: 2 resident trees (1e6 and
    2e7 uint64 keys, fanout 32), requests of 1..64 lookups (geometric, mean
    8), 50 us batching deadline, memory-capped admission; plain search
    against the learned (PL-256) search."""
    sizes = [1_000_000, 20_000_000]
    trees, keysets, models = [], [], []
    for i, n in enumerate(sizes):
        keys = W.uniform_keys(n, 64, seed=W.SEED_BASE + 60 + i)
        trees.append(bt.BTree(keys, W.rank_values(n, 64), 32))
        keysets.append(keys)
        models.append(bt.bt_model_train(trees[-1].handle, bt.BT_MODEL_PL, segments=256))
    out = {"workload": "2 trees (1e6, 2e7 uint64 keys, fanout 32); Poisson arrivals; requests of 1..64 lookups "
                       "(geometric, mean 8), 80% hits; 50 us deadline; 8 slots; 16 MB in-flight cap",
           "rates": {}}
    for rate in rates:
        nreq = max(1000, int(rate / 8.0 * seconds))
        seed = W.SEED_BASE + 70 + int(rate // 1e6)
        cnt = W.geometric_request_sizes(nreq, seed=seed).astype(np.uint32)
        tid = W.rng(seed).integers(0, 2, size=nreq).astype(np.uint32)
        pools = [W.make_queries(keysets[i], int(cnt[tid == i].sum()), 0.8, seed=seed + 1 + i, width_bits=64)
                 for i in range(2)]
        base = [0, pools[0].size]
        allk = np.concatenate(pools)
        koff = np.empty(nreq, np.uint64)
        cur = [0, 0]
        for r in range(nreq):
            i = int(tid[r])
            koff[r] = base[i] + cur[i]
            cur[i] += int(cnt[r])
        t_arr = W.poisson_arrivals(rate / 8.0, nreq, seed=seed + 3)
        row = {"requests": nreq, "lookups": int(allk.size)}
        ref = None
        for mode in ("plain", "learned"):
            srv = bt.bt_server_create(trees, models if mode == "learned" else None, slots=8, max_batch=8192,
                                      deadline_us=50.0, mem_cap_bytes=16 << 20)
            vals = np.zeros(allk.size, np.uint64)
            found = np.zeros(allk.size, np.uint8)
            wall = bt.bt_server_run_trace(srv, t_arr, tid, cnt, koff, allk, vals, found)
            st = bt.bt_server_get_stats(srv)
            bt.bt_server_destroy(srv)
            row[mode] = {"lookups_per_s": allk.size / wall, "offered_lookups_per_s": rate,
                         "p50_us": float(st.p50_us), "p99_us": float(st.p99_us), "batches": int(st.batches),
                         "mean_batch": allk.size / max(1, st.batches), "max_inflight": int(st.max_inflight)}
            if ref is None:
                ref = (vals, found)
            else:
                row[mode]["bit_exact_vs_plain"] = bool(np.array_equal(vals, ref[0]) and np.array_equal(found, ref[1]))
        out["rates"][f"{rate / 1e6:g}M"] = row
    for m in models:
        bt.bt_model_free(m)
    for t in trees:
        t.close()
    return out


# ---------------------------------------------------------- our arm

def run_ours(a):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    from paper_2604_21117_gb300 import build_lib
    build_lib.build()
    from paper_2604_21117_gb300 import btree as bt

    keys, vals = make_tree_data(a)
    pool = 4
    batches = make_batches(a, keys, pool, rank, world)
    tree = bt.BTree(keys, vals, a.fanout)
    bt.bt_tree_set_staging(tree.handle, a.staging)
    bt.bt_tree_set_lane_queries(tree.handle, a.lane_queries)
    bt.bt_tree_set_descent(tree.handle, a.inner, a.ballot)
    if a.l2_window > 0:
        bt.bt_tree_set_l2_window(tree.handle, a.l2_window)
    if a.warps > 0 or a.pin >= 0:
        bt.bt_tree_set_launch(tree.handle, a.warps if a.warps > 0 else 8, a.pin if a.pin >= 0 else 16384)
    m, kb, vb, B = a.fanout, 8, 8, a.batch

    alg = []
    for qb in batches:
        counts, sectors = touched(keys, tree.level_nodes, m, qb)
        alg.append((counts, sectors, descend_algorithmic_bytes(counts, sectors, m, kb, vb, B)))

    dq = [torch.from_numpy(qb).cuda() for qb in batches]
    sq = torch.empty(B, dtype=torch.uint64, device="cuda")
    si = torch.empty(B, dtype=torch.int32, device="cuda")
    out_v = torch.empty(B, dtype=torch.uint64, device="cuda")
    out_f = torch.empty(B, dtype=torch.uint8, device="cuda")
    nb = tree.workspace_bytes(B)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    flush.fill_(0)
    flush_sink = torch.empty(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    sort_bits = a.sort_bits

    def clear_l2(i):
        if a.l2 == "write":
            flush.fill_(i)
        elif a.l2 == "read":  # leaves clean lines: no write-back inside the step
            flush_sink.copy_(flush.sum(dtype=torch.int64))

    def step(i, phase_event=None):
        # one whole search of batch i: partition, descent, leaf probe, scatter
        bt.bt_search_batch_ex(tree.handle, dq[i % pool], B, out_v, out_f, ws, nb, sort_bits, None, stream,
                              phase_event)

    sampler = ClockSampler(local)
    sampler.start()
    for i in range(a.warmup):
        clear_l2(i)
        step(i)
    torch.cuda.synchronize()

    K = a.steps

    def timed_loop(clear, phases=True):
        # phases: also record an event between the partition and the descent
        # (it keeps the descent from starting under the partition's tail, so
        # the step itself is timed without it)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
        for e in ev:  # create the events (the middle one is recorded inside the call)
            for x in e:
                x.record(stream)
        barrier(world)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for i in range(K):
            clear(i)
            e0, e1, e2 = ev[i]
            e0.record(stream)
            step(i, e1 if phases else None)
            e2.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return ([e[0].elapsed_time(e[2]) for e in ev], [e[0].elapsed_time(e[1]) for e in ev] if phases else None,
                [e[1].elapsed_time(e[2]) for e in ev] if phases else None, time.perf_counter() - w0)

    # the second stream's workspace and outputs
    ws2 = torch.empty(nb, dtype=torch.uint8, device="cuda")
    out_v2 = torch.empty(B, dtype=torch.uint64, device="cuda")
    out_f2 = torch.empty(B, dtype=torch.uint8, device="cuda")
    bufs = [(out_v, out_f, ws), (out_v2, out_f2, ws2)]
    pstreams = [torch.cuda.Stream(), torch.cuda.Stream()]
    corun = tuple(int(x) for x in a.corun.split(","))

    def pipelined_loop():
        # step i on stream i % 2 with buffer set i % 2; the total runs from an
        # event on stream 0 (stream 1 waits for it) to stream 0's join of stream 1
        per = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        t0e.record(pstreams[0])
        pstreams[1].wait_event(t0e)
        for i in range(K):
            st, (ov, of, w) = pstreams[i % 2], bufs[i % 2]
            with torch.cuda.stream(st):
                clear_l2(i)
            per[i][0].record(st)
            bt.bt_search_batch_ex(tree.handle, dq[i % pool], B, ov, of, w, nb, sort_bits, None, st)
            per[i][1].record(st)
        pstreams[0].wait_stream(pstreams[1])
        t1e.record(pstreams[0])
        torch.cuda.synchronize()
        barrier(world)
        return t0e.elapsed_time(t1e), [e0.elapsed_time(e1) for e0, e1 in per], time.perf_counter() - w0

    # one stream, nothing capped: each step alone (and the phase split)
    one_ms, _, _, one_wall = timed_loop(clear_l2, phases=False)
    phase_step_ms, sort_ms, desc_ms, _ = timed_loop(clear_l2)
    if a.streams == 2:
        bt.bt_tree_set_corun(tree.handle, corun[0], corun[1])
        for i in range(a.warmup):  # warm up the capped launch shapes on both streams
            st, (ov, of, w) = pstreams[i % 2], bufs[i % 2]
            bt.bt_search_batch_ex(tree.handle, dq[i % pool], B, ov, of, w, nb, sort_bits, None, st)
        torch.cuda.synchronize()
        total_ms, step_ms, wall = pipelined_loop()
        bt.bt_tree_set_corun(tree.handle, 0, 0)
        last_out = bufs[(K - 1) % 2]
    else:
        total_ms, step_ms, wall = sum(one_ms), one_ms, one_wall
        last_out = bufs[0]
    total_s = total_ms / 1e3
    total_s_max = reduce_max(total_s, world, device="cuda")
    value = B * K * world / total_s_max
    one_total_max = reduce_max(sum(one_ms) / 1e3, world, device="cuda")
    out_v, out_f = last_out[0], last_out[1]

    # correctness spot check of the last step against the plain definition
    if world > 1:
        # the ranks' results of the last batch, reassembled in input order
        from paper_2604_21117_gb300.replicas import gather_in_input_order
        gv = gather_in_input_order(out_v.view(torch.int64), B * world, world, rank)
        gf = gather_in_input_order(out_f.to(torch.int64), B * world, world, rank)
        got_v = gv.cpu().numpy().view(np.uint64)
        got_f = gf.cpu().numpy().astype(np.uint8)
        i_last = (K - 1) % pool
        last = W.make_queries(keys, B * world, a.hit, seed=W.SEED_BASE + 2 + 1000 * (i_last + 1), width_bits=64,
                              zipf_s=a.zipf)
    else:
        last = batches[(K - 1) % pool]
        got_v = out_v.cpu().numpy()
        got_f = out_f.cpu().numpy()
    pos = np.searchsorted(keys, last)
    hit = (pos < keys.size) & (keys[np.minimum(pos, keys.size - 1)] == last)
    ok = bool(np.array_equal(got_f.astype(bool), hit) and np.array_equal(got_v[hit], vals[pos[hit]]))

    # bytes and roofline of the dominant kernel (the descent)
    desc_bytes = [alg[i % pool][2] for i in range(K)]
    node_bytes = [sum(alg[i % pool][0]) * m * kb + alg[i % pool][1] * 32 for i in range(K)]
    achieved = statistics.fmean(desc_bytes) / (statistics.fmean(desc_ms) / 1e3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = None
    default_workload = (a.keys == 1 << 24 and a.batch == 1 << 20 and a.fanout == 32 and a.zipf is None
                        and abs(a.hit - 0.9) < 1e-9)
    if (NCU_DESCEND_TRAFFIC["descend_src_sha256"] == src_sha256() and default_workload and a.lane_queries == 1
            and a.staging == 2 and a.inner in (1, 2) and a.ballot == 0 and a.l2_window == 64 << 20 and a.warps <= 0
            and a.pin < 0 and a.sort_bits < 0):
        traffic = NCU_DESCEND_TRAFFIC["bytes_per_launch"]
    step_gbs = statistics.fmean(node_bytes) / (total_s / K) / 1e9  # per batch, at the whole job's rate
    sort_k = bt.bt_sort_launches(tree.handle, B, sort_bits)
    # our kernels per step: the partition's kernels, then the descent
    launches_per_step = sort_k + 1
    sdev = sorted(step_ms)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": a.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded uniform keys and query mix)",
        "config": workload_config(a, world),
        "launch": {"sort_bits": "auto" if sort_bits < 0 else sort_bits,
                   "staging": {0: "synchronous cp.async", 1: "synchronous bulk copy",
                               2: "pipelined bulk-copy leaves"}[a.staging],
                   "inner_levels": {0: "through L1", 1: "staged (cp.async)",
                                    2: "staged (cp.async) for partitioned batches, else through L1"}[a.inner],
                   "leaf_rank": "ballot + popc" if a.ballot else "binary search",
                   "l2_window_bytes": a.l2_window, "lane_queries": a.lane_queries,
                   "steps_in_flight": a.streams,
                   "corun_blocks_per_sm": ({"descent": corun[0], "partition": corun[1]} if a.streams == 2
                                           else None),
                   "l2": {"write": "flushed before every timed step (256 MB device write)",
                          "read": "flushed before every timed step (256 MB device read)",
                          "none": "not flushed: the 282 MB tree exceeds the 129 MB L2 and 4 batches "
                                  "rotate"}[a.l2]},
        "p50_us": 1e3 * sdev[len(sdev) // 2], "p99_us": 1e3 * sdev[min(len(sdev) - 1, int(0.99 * len(sdev)))],
        "iqm_us": 1e3 * iqm(step_ms),
        "latency_note": ("p50/p99/iqm: each step's own time on its stream, with the other stream's step "
                         "running beside it" if a.streams == 2 else "each step alone"),
        "one_stream": {"value": B * K * world / one_total_max, "ms_per_step": statistics.fmean(one_ms),
                       "p50_us": 1e3 * sorted(one_ms)[len(one_ms) // 2],
                       "note": "the same steps one at a time on one stream, launch shapes uncapped"},
        "phase_ms": {"sort": statistics.fmean(sort_ms), "descend": statistics.fmean(desc_ms),
                     "step_with_phase_event": statistics.fmean(phase_step_ms),
                     "note": "one stream, launch shapes uncapped, an event between the phases (which keeps "
                             "the descent from starting under the partition's tail)"},
        "hbm_gbs": step_gbs,
        "roofline": {"kernel": "k_descend (level-wise descent + leaf probe + scatter)", "bound": "hbm",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": f"{peak_kind} (hbm_gbs)", "traffic": traffic,
                     "algorithmic_bytes_per_launch": statistics.fmean(desc_bytes),
                     "distinct_nodes_per_level": alg[0][0], "distinct_value_sectors": alg[0][1],
                     # the whole search per batch (sort + descent): bytes of the distinct
                     # nodes the batch touches (and its value sectors) over the step time
                     "per_batch": {"what": "distinct node bytes + value sectors per batch / (whole job time / steps)",
                                   "bytes": statistics.fmean(node_bytes), "achieved": step_gbs,
                                   "frac": step_gbs / peak},
                     "target": {"frac": 0.5, "applies_to": "per_batch (the whole search, sort included)",
                                "met": step_gbs / peak >= 0.5, "descent_kernel_alone_met": achieved / peak >= 0.5}},
        "gpu_launches": launches_per_step * K,
        "correct_last_step": ok, "wall_s_timed_loop": wall,
    }

    if a.l2 != "write":
        # the same loop with a 256 MB buffer overwritten before every step: the
        # L2 then starts each step full of dirty lines that must be written back
        w_step, w_sort, w_desc, _ = timed_loop(lambda i: flush.fill_(i))
        w_tot = reduce_max(sum(w_step) / 1e3, world, device="cuda")
        line["l2_write_flushed"] = {"value": B * K * world / w_tot, "ms_per_step": statistics.fmean(w_step),
                                    "phase_ms": {"sort": statistics.fmean(w_sort),
                                                 "descend": statistics.fmean(w_desc)}}

    # the same step replayed from CUDA graphs (one per batch of the pool),
    # the way a serving loop would issue it: no host launch cost per kernel
    graphs = []
    cap = torch.cuda.Stream()
    cap.wait_stream(stream)
    with torch.cuda.stream(cap):
        for p_ in range(pool):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                bt.bt_search_batch_ex(tree.handle, dq[p_], B, out_v, out_f, ws, nb, sort_bits, None, cap)
            graphs.append(g)
    stream.wait_stream(cap)
    torch.cuda.synchronize()
    for i in range(3):
        graphs[i % pool].replay()
    gev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    for i in range(K):
        clear_l2(i)
        gev[i][0].record(stream)
        graphs[i % pool].replay()
        gev[i][1].record(stream)
    torch.cuda.synchronize()
    g_ms = [e[0].elapsed_time(e[1]) for e in gev]
    g_tot = reduce_max(sum(g_ms) / 1e3, world, device="cuda")
    line["graph_replay"] = {"value": B * K * world / g_tot, "unit": UNIT, "ms_per_step": statistics.fmean(g_ms),
                            "p99_us": 1e3 * sorted(g_ms)[min(K - 1, int(0.99 * K))]}

    if not a.no_extras:
        # end to end through the host-buffer entry point: H2D of the queries,
        # search, D2H of values and found flags, every step
        hq = torch.from_numpy(batches[0]).pin_memory()
        hv = torch.empty(B, dtype=torch.uint64).pin_memory()
        hf = torch.empty(B, dtype=torch.uint8).pin_memory()
        nbh = bt.bt_search_host_workspace_bytes(tree.handle, B)
        wsh = torch.empty(nbh, dtype=torch.uint8, device="cuda")
        for _ in range(3):
            bt.bt_search_batch_host(tree.handle, hq, B, hv, hf, wsh, nbh, stream)
        torch.cuda.synchronize()
        Ke = max(10, min(K, 200))
        tt = []
        for i in range(Ke):
            clear_l2(i)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bt.bt_search_batch_host(tree.handle, hq, B, hv, hf, wsh, nbh, stream)
            e1.record(stream)
            e1.synchronize()
            tt.append(e0.elapsed_time(e1))
        e2e_s = reduce_max(sum(tt) / 1e3, world, device="cuda")
        serial = B * Ke * world / e2e_s
        # the same calls pipelined the way a host keeps a GPU busy (Sec. V-B,
        # Fig. 7): four streams, each with its own pinned buffers and
        # workspace, steps issued in turn, so that steps' copies in, copies
        # out and kernels overlap; the launch shapes are capped as in the
        # two-in-flight loop, so that one step's partition runs beside
        # another's descent.  Every step still copies its queries in and its
        # values and found flags out.
        NS = 4
        if a.streams == 2:
            bt.bt_tree_set_corun(tree.handle, corun[0], corun[1])
        streams = [torch.cuda.Stream() for _ in range(NS)]
        bufs = []
        for j in range(NS):
            bufs.append((torch.from_numpy(batches[j % pool]).pin_memory(),
                         torch.empty(B, dtype=torch.uint64).pin_memory(),
                         torch.empty(B, dtype=torch.uint8).pin_memory(),
                         torch.empty(nbh, dtype=torch.uint8, device="cuda")))
        for j in range(2 * NS):
            h = bufs[j % NS]
            bt.bt_search_batch_host(tree.handle, h[0], B, h[1], h[2], h[3], nbh, streams[j % NS])
        torch.cuda.synchronize()
        barrier(world)
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        fin = [torch.cuda.Event() for _ in range(NS)]
        p0.record(stream)
        for j in range(NS):
            streams[j].wait_event(p0)
        for j in range(Ke):
            h = bufs[j % NS]
            bt.bt_search_batch_host(tree.handle, h[0], B, h[1], h[2], h[3], nbh, streams[j % NS])
        for j in range(NS):
            fin[j].record(streams[j])
            stream.wait_event(fin[j])
        p1.record(stream)
        torch.cuda.synchronize()
        pipe_s = reduce_max(p0.elapsed_time(p1) / 1e3, world, device="cuda")
        bt.bt_tree_set_corun(tree.handle, 0, 0)
        pipelined = B * Ke * world / pipe_s
        line["e2e"] = {"value": pipelined, "unit": UNIT, "h2d_bytes_per_step": B * kb,
                       "d2h_bytes_per_step": B * (vb + 1), "steps": Ke,
                       "entry_point": f"bt_search_batch_host (pinned host buffers), {NS} streams in turn"
                                      + (f", launch shapes capped as in the two-in-flight loop {corun}"
                                         if a.streams == 2 else ""),
                       "serial_value": serial, "serial_p50_us": 1e3 * sorted(tt)[len(tt) // 2],
                       "l2": "serial: flushed before every step; pipelined: not flushed (steps overlap; the "
                             "282 MB tree exceeds the 129 MB L2)"}
        # small-batch latency (the paper's batch sizes go to 1000)
        lat = {}
        for b in (1, 1024):
            qs = torch.from_numpy(batches[1][:b].copy()).cuda()
            v1 = torch.empty(b, dtype=torch.uint64, device="cuda")
            f1 = torch.empty(b, dtype=torch.uint8, device="cuda")
            n1 = tree.workspace_bytes(b)
            w1 = torch.empty(max(n1, 1), dtype=torch.uint8, device="cuda")
            for _ in range(20):
                bt.bt_search_batch(tree.handle, qs, b, v1, f1, w1, n1, stream)
            fn = lambda: bt.bt_search_batch(tree.handle, qs, b, v1, f1, w1, n1, stream)
            us = _time_calls(fn, 500, None, stream)
            su = _time_calls(fn, 500, None, stream, submit=True)
            lat[f"b{b}"] = {"p50_us": us[len(us) // 2], "p99_us": us[int(0.99 * len(us))],
                            "lookups_per_s": b / (statistics.fmean(us) / 1e6),
                            "with_submission": {"p50_us": su[len(su) // 2], "p99_us": su[int(0.99 * len(su))]}}
        lat["timing"] = ("device time of each call (queued behind a device spin, so that the host's "
                         "submission is not timed); with_submission: the host's submission included")
        line["small_batch_latency"] = lat

    if not a.no_designs:
        line["designs"] = designs_leg(a, bt, tree, dq, out_v, out_f, ws, nb, stream, alg, pool)
    if not a.no_extras and not a.no_sweeps:
        line["sweeps"] = sweep_leg(a, bt, stream, keys, vals, tree)
    if not a.no_extras and not a.no_paper_keys:
        line["paper_keys"] = paper_keys_leg(a, bt, flush, stream, peak)
    if not a.no_extras and not a.no_learned:
        line["learned"] = learned_leg(a, bt, flush, stream)
    if not a.no_extras and not a.no_batching:
        line["batching"] = batching_leg(a, bt, stream)
    if not a.no_extras and not a.no_serving:
        line["serving"] = serving_leg(a, bt)
    if not a.no_extras and not a.no_range:
        # the single tree's results of batch 0, for the range leg's check
        bt.bt_search_batch(tree.handle, dq[0], B, out_v, out_f, ws, nb, stream)
        torch.cuda.synchronize()
        ref0 = (out_v.cpu().numpy().copy(), out_f.cpu().numpy().copy())
        line["range_split"] = range_leg(a, bt, keys, vals, dq, ref0, stream)

    sampler.stop()
    line["clocks"] = sampler.summary()

    if rank == 0 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(keys, vals, m, batches[0])
    if rank == 0:
        print(json.dumps(line), flush=True)
    tree.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------ reference arm

def run_reference(a):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    keys, vals = make_tree_data(a)
    q = make_batches(a, keys, 1)[0]
    tree = oracle.OracleTree(keys, vals, a.fanout)
    cores = os.cpu_count() or 1
    sample = min(q.size, CPU_SAMPLE)
    qs = q[:sample]
    for _ in range(a.warmup):
        tree.search_mt(qs, cores)
    ts = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        tree.search_mt(qs, cores)
        ts.append(time.perf_counter() - t0)
    total = sum(ts)
    value = sample * a.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (seeded uniform keys and query mix)",
        "config": workload_config(a, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "hardware_concurrency": cores,
                         "sample": f"each step: the first {sample} queries of the batch (the same sample as "
                                   f"the GPU arm's cpu_baseline), split evenly over {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    tree.close()
    print(json.dumps(line), flush=True)


def main(argv=None):
    a = parse_args(argv)
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
