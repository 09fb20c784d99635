#!/usr/bin/env python
"""Benchmark of Strassen's block-recursive inversion on GB300.

One step = one inversion of one synthetic matrix through the library's C ABI
(the whole recursion: leaves, level products, subtractions).  The metric is
the effective rate 2 n^3 / t (the exact flop count of the method, since the
six products per level and the 2 L^3 leaves sum to 2 n^3).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--n N --leaf L] [--impl ours|reference]

Workloads:
  plain_fp64   A = G G^T / n + I (G ~ N(0,1), seeded), n = 32768, leaf 512,
               every product in FP64 (the plain method at scale).
  small_fp64   U(-1,1) + n on the diagonal, n = 1024, leaf 128.

With N > 1 (torchrun) every rank inverts its own matrix (independent
replicas, weak scaling); `value` is the sum of all ranks' flops over the
slowest rank's time.  `--impl reference` times the CPU oracle on this
host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2n³/t TFLOP/s vs FP64/BF16 peak at residual ≤1e-10; served req/s with p50/p99"
T_START = time.perf_counter()
# The batched and serving sub-records of the default run start only before
# these many seconds of run time (the limit for the whole run is 1800 s; the
# batched sub-record takes about 35 s, the serving one about 25 s, and the
# serving run aborts after 60 s without progress).
BATCHED_DEADLINE_S = 1600.0
SERVE_DEADLINE_S = 1650.0

SEED_BASE = 0x5EED0000

WORKLOADS = {
    "plain_fp64": dict(n=32768, leaf=512, precision="fp64", family="spd_gram", seed=SEED_BASE + 1,
                       desc="plain method, one FP64 SPD matrix A = G G^T/n + I, n = 32768, leaf 512"),
    "small_fp64": dict(n=1024, leaf=128, precision="fp64", family="sdd", seed=SEED_BASE,
                       desc="plain method, one FP64 SDD matrix (U(-1,1) + n I), n = 1024, leaf 128"),
    "batched_fp64": dict(n=1024, leaf=0, precision="fp64", family="batch_sdd", seed=SEED_BASE + 3,
                         desc="4096 independent FP64 matrices, orders log-uniform in [32, 1024] rounded to "
                              "multiples of 32, each U(-1,1) + n I; one spin_invert_batched call (CUDA graph)"),
    "batched_mixed": dict(n=1024, leaf=0, precision="bf16x3", family="batch_sdd", seed=SEED_BASE + 3,
                          desc="the batching workload (4096 matrices, orders log-uniform in [32, 1024], multiples "
                               "of 32, each U(-1,1) + n I) in the mixed form: tensor-core level products batched "
                               "over each order bucket, FP64 leaves, Newton-Schulz to residual <= 1e-10"),
    "serve": dict(n=8192, leaf=0, precision="mixed", family="serve", seed=SEED_BASE + 4,
                  desc="serving: Poisson arrivals at 200 req/s, n log-uniform in [64, 8192], A = G G^T/n + alpha I "
                       "(alpha uniform in [0.1, 1]); half the requests ask for residual <= 1e-13, half for "
                       "<= 1e-10; admission by device-memory footprint under a 150 GB budget, 8 slots"),
    "mixed_digits": dict(n=32768, leaf=128, precision="digits", family="householder", seed=SEED_BASE + 2,
                         desc="as mixed_bf16x3 but the level products are 4-slice BF16 digit products with exact "
                              "FP32 runs (~2^-30), so the first residual usually certifies the result"),
    "mixed_bf16x3": dict(n=32768, leaf=128, precision="bf16x3", family="householder", seed=SEED_BASE + 2,
                         desc="mixed precision, one SPD matrix A = Q diag(d) Q^T (64 Householder reflectors, "
                              "d log-uniform in [1, 1e3]), n = 32768: BF16x3 tensor-core level products, FP64 "
                              "leaves, FP64-class top-two Schur complements and residual, Newton-Schulz to 1e-10"),
}


BATCH_COUNT = 4096
BATCH_LEAF_CANDIDATES = (32, 64, 128, 256)
PERSIST_MAX_LEAF = 64  # largest leaf of the persistent batch kernel
BATCH_TILE_CANDIDATES = (64, 32, 16)  # largest product tile of a bucket, persistent schedule


def measured_peaks() -> dict:
    """Measured peaks of this machine (HBM GB/s, BF16 TFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="plain_fp64", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=0, help="override the order (development runs)")
    ap.add_argument("--leaf", type=int, default=-1, help="override the leaf order")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--probes", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="plain_fp64: skip the mixed-precision sub-record")
    ap.add_argument("--no-batched", action="store_true", help="plain_fp64: skip the batched sub-record")
    ap.add_argument("--no-serve", action="store_true", help="plain_fp64: skip the serving sub-record")
    ap.add_argument("--serve-sub-seconds", type=float, default=15.0,
                    help="plain_fp64: arrival window of the serving sub-record (s)")
    ap.add_argument("--mixed-steps", type=int, default=3, help="plain_fp64: timed steps of the mixed sub-record "
                    "(at most --steps)")
    ap.add_argument("--mixed-warmup", type=int, default=2, help="plain_fp64: warm-up steps of the mixed sub-record "
                    "(at most --warmup, at least 1)")
    ap.add_argument("--schedule", default="default", choices=["default", "lockstep", "persistent"],
                    help="single-matrix workloads: II and C21 on a second stream where it pays (default), "
                         "one stream (lockstep) or the second stream at every order (persistent)")
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT,
                    help="batched workloads: matrices per batch (smaller for profiler captures)")
    ap.add_argument("--batch-schedule", default="default", choices=["default", "lockstep", "persistent"],
                    help="batched workloads, plain form: one persistent launch (default) or lockstep launches")
    ap.add_argument("--profile-json", default="", help="write per-launch records here")
    ap.add_argument("--leaf-times", default="", help="comma-separated leaf orders: time one leaf inversion "
                    "(spin_leaf_inverse on its default cluster) per order and print the per-pivot-step times")
    ap.add_argument("--leaf-batch", default="", help="L:count -- time count leaves of order L <= 128 side by side "
                    "(one batched leaf launch, one CTA each) and print the per-pivot-step time and cycles")
    ap.add_argument("--leaf-sweep", default="", help="comma-separated orders: time every candidate leaf "
                    "(the U-shaped block-size sweep) with spin_autotune_leaf and print one JSON line")
    ap.add_argument("--gemm-probe", type=int, default=0, help="time one digit-slice (6 slices) and one bf16x3 "
                    "tensor-core product of this order and print one JSON line")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="serving: arrival window (s)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="serving: Poisson arrival rate (req/s)")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-max-batch", type=int, default=0,
                    help="serving: requests per batched launch group (0: the library default, 64; 1: off)")
    ap.add_argument("--serve-priority-order", type=int, default=1024,
                    help="serving: requests of order <= this run on high-priority streams (0: off)")
    ap.add_argument("--fp64-levels", type=int, default=2,
                    help="mixed workloads: top recursion levels with FP64-class Schur complements")
    ap.add_argument("--pretransform", type=int, default=0, choices=[0, 1, 2],
                    help="single-matrix workloads: random butterfly transform around the recursion "
                         "(1: always, 2: after a breakdown); the default workloads need none")
    ap.add_argument("--oracle-sizes", default="", help="reference arm: also time one oracle inversion at each of "
                    "these orders (all host threads, plus one thread at the smallest) and add them to the line")
    ap.add_argument("--serve-fp64-path", default="mixed", choices=["mixed", "plain"],
                    help="path for the 1e-13 requests: mixed precision refined to 1e-13, or the plain FP64 method")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ inputs --

def make_input(w: dict, n: int, device):
    """(A on the device, known-inverse handle or None)."""
    from paper_1801_04723_gb300 import inputs

    if w["family"] == "spd_gram":
        return inputs.spd_gram_device(n, w["seed"], device), None
    if w["family"] == "sdd":
        return inputs.sdd_device(n, w["seed"], device), None
    if w["family"] == "householder":
        A, V, d = inputs.householder_spd_device(n, w["seed"], device, reflectors=64, cond=1e3)
        return A, (V, d)
    raise ValueError(w["family"])


def known_inverse_error(X, known, cols: int = 8) -> float:
    """max over sampled columns j of ||X e_j - Q diag(1/d) Q^T e_j|| / ||Q diag(1/d) Q^T e_j||."""
    import numpy as np

    from paper_1801_04723_gb300 import inputs

    V, d = known
    n = X.shape[0]
    js = np.linspace(0, n - 1, cols).astype(int)
    E = np.zeros((n, cols))
    E[js, np.arange(cols)] = 1.0
    ref = inputs.householder_apply(V, 1.0 / d, E)
    got = X[:, js].double().cpu().numpy()
    return float(np.max(np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)))


def freivalds_rel(A, X, k: int, seed: int) -> float:
    """Relative residual estimate sqrt(mean ||(AX - I) v||^2) / (||A||_F ||X||_F)
    with k N(0,1) probe vectors (E||Rv||^2 = ||R||_F^2), FP64 on the device."""
    import torch
    from paper_1801_04723_gb300 import inputs

    n = A.shape[0]
    V = inputs.normal_torch(seed, n, k, 0, A.device)
    R = A @ (X @ V) - V
    est = math.sqrt(float((R * R).sum()) / k)
    return est / (float(torch.linalg.norm(A)) * float(torch.linalg.norm(X)))


# --------------------------------------------------------------- baseline --

def host_sample(w: dict, n_s: int):
    from paper_1801_04723_gb300 import inputs

    if w["family"] in ("spd_gram", "serve"):
        return inputs.spd_gram(n_s, seed=w["seed"])
    if w["family"] == "householder":
        return inputs.householder_spd(n_s, seed=w["seed"], reflectors=64, cond=1e3)[0]
    return inputs.sdd(n_s, seed=w["seed"])


def sample_leaf(w: dict, n_s: int) -> int:
    if w["leaf"] > 0:
        return min(w["leaf"], n_s)
    return n_s if n_s <= 128 else 64


def cpu_baseline(w: dict, seconds_hint: float = 15.0) -> dict:
    """The oracle, as it stands, on this host's cores: one inversion of a
    bounded sample of the workload (same family and leaf, smaller order)."""
    import numpy as np

    import oracle
    from paper_1801_04723_gb300 import inputs

    n_s = 4096 if w["n"] >= 4096 else w["n"]
    leaf = sample_leaf(w, n_s)
    A = host_sample(w, n_s)
    oracle.strassen_inv(np.eye(8), 2)  # build / load outside the timing
    t0 = time.perf_counter()
    oracle.strassen_inv(A, leaf)
    dt = time.perf_counter() - t0
    out = {"value": 2.0 * n_s ** 3 / dt / 1e12, "unit": "TFLOP/s", "cores": oracle.num_threads(),
           "kind": "oracle", "sample": f"one inversion, n={n_s}, leaf {leaf}, {w['family']} input, "
                                       f"{dt:.1f} s on {oracle.num_threads()} threads"}
    if w["n"] > n_s:
        # the method's work is 2 n^3 at any leaf: the full order's time by n^3
        out["extrapolated"] = {"n": w["n"], "seconds": dt * (w["n"] / n_s) ** 3, "label": "extrapolated",
                               "how": f"sample time x (n / {n_s})^3"}
    return out


def run_reference_serve(args, w: dict):
    """The oracle serving the same request trace one request at a time on the
    host's cores, on a bounded prefix of the trace (about 20 s of work)."""
    import numpy as np

    import oracle
    from paper_1801_04723_gb300 import inputs

    trace = inputs.serve_trace(w["seed"], rate=args.serve_rate, duration=args.serve_seconds, lo=64,
                               hi=min(8192, w["n"]))
    oracle.strassen_inv(np.eye(8), 2)
    lat, flops, t_used, skipped = [], 0.0, 0.0, 0
    rate = 5e9  # flop/s guess until the first requests are timed
    for j, (t, n, alpha, mixed) in enumerate(trace):
        if t_used > 20.0:
            break
        if t_used + 2.0 * float(n) ** 3 / rate > 30.0:  # keep the sample bounded
            skipped += 1
            continue
        A = inputs.spd_gram(n, seed=w["seed"] + 7919 * (j + 1), alpha=alpha)
        leaf = n if n <= 128 else 128
        t0 = time.perf_counter()
        oracle.strassen_inv(A, leaf)
        dt = time.perf_counter() - t0
        t_used += dt
        lat.append(dt * 1e3)
        flops += 2.0 * float(n) ** 3
        rate = flops / t_used
    val = len(lat) / t_used
    lat.sort()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "req/s", "n_gpus": args.gpus, "steps": 1,
        "warmup": 0, "ms_per_step": t_used * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "serve", "rate_req_s": args.serve_rate, "requests_sampled": len(lat)},
        "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
        "cpu_baseline": {"value": val, "unit": "req/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"first {len(lat)} requests of the trace ({skipped} predicted to overrun a 30 s "
                                   f"budget skipped), served one at a time by the oracle "
                                   f"({flops / t_used / 1e12:.4f} TFLOP/s)"},
        "e2e": {"value": val, "unit": "req/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args, w: dict, n: int, leaf: int):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_1801_04723_gb300 import inputs

    if w["family"] == "serve":
        return run_reference_serve(args, w)

    n_s = min(n, 4096)
    leaf_s = sample_leaf(w, n_s)
    A = host_sample(w, n_s)
    oracle.strassen_inv(np.eye(8), 2)
    for _ in range(args.warmup):
        oracle.strassen_inv(A, leaf_s)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.strassen_inv(A, leaf_s)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    val = 2.0 * n_s ** 3 / dt / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "leaf": leaf, "precision": w["precision"],
                   "sample_n": n_s, "sample_leaf": leaf_s},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"one oracle inversion per step at n={n_s}, leaf {leaf_s} (bounded sample "
                                   f"of the n={n} workload)"},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    if args.oracle_sizes:
        line["oracle_sizes"] = oracle_size_sweep(w, [int(v) for v in args.oracle_sizes.split(",") if v])
    print(json.dumps(line), flush=True)
    return 0


def oracle_size_sweep(w: dict, sizes: list) -> list:
    """One oracle inversion per order on all host threads, and one more on a
    single thread at the smallest order."""
    import oracle

    out = []
    threads = oracle.num_threads()
    for i, m in enumerate(sorted(sizes)):
        leaf_m = sample_leaf(w, m)
        A = host_sample(w, m)
        for t in ([threads, 1] if i == 0 else [threads]):
            oracle.set_threads(t)
            t0 = time.perf_counter()
            oracle.strassen_inv(A, leaf_m)
            dt = time.perf_counter() - t0
            out.append({"n": m, "leaf": leaf_m, "threads": t, "s": dt, "tflops": 2.0 * m ** 3 / dt / 1e12})
    oracle.set_threads(threads)
    return out


# -------------------------------------------------------------------- ours --

class SingleWork:
    """One matrix per rank: spin_invert_ex on a device-resident input."""

    def __init__(self, spin, w, n, leaf, device, pretransform=0, fp64_levels=2, schedule="default"):
        import torch

        self.spin, self.w, self.n, self.leaf = spin, w, n, leaf
        self.schedule = schedule
        self.pt = pretransform
        self.fl = fp64_levels
        self.A, self.known = make_input(w, n, device)
        self.X = torch.empty_like(self.A)
        self.flops = 2.0 * float(n) ** 3
        self.Ah = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        self.Ah.copy_(self.A)
        self.Xh = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        self.h2d = self.d2h = 8 * n * n

    def step(self):
        self.spin.invert(self.A, leaf=self.leaf, precision=self.w["precision"], out=self.X, blocking=False,
                         pretransform=self.pt, rbt_seed=SEED_BASE + 5, fp64_levels=self.fl, schedule=self.schedule)

    def launches(self, recs, steps):
        return len(recs)

    def finish(self):
        return self.spin.sync(check=False)

    def e2e_step(self):
        self.spin.invert_host(self.Ah.numpy(), leaf=self.leaf, precision=self.w["precision"], out=self.Xh.numpy(),
                              pretransform=self.pt, rbt_seed=SEED_BASE + 5, schedule=self.schedule)

    def accuracy(self, probes):
        out = {"rel_residual_est": freivalds_rel(self.A, self.X, probes, SEED_BASE + 77) if probes > 0 else None}
        if self.known is not None:
            out["err_vs_known_inverse"] = known_inverse_error(self.X, self.known)
        return out


class BatchWork:
    """Thousands of matrices of uneven order: one spin_invert_batched call."""

    def __init__(self, spin, w, n, leaf, device, count, schedule="default"):
        import torch

        from paper_1801_04723_gb300 import inputs

        self.spin, self.leaf = spin, leaf
        self.precision = w["precision"]
        # the plain batch runs as one persistent launch unless lockstep is asked for
        self.schedule = schedule
        persistent = self.precision == "fp64" and schedule != "lockstep"
        cands = tuple(c for c in BATCH_LEAF_CANDIDATES if c <= PERSIST_MAX_LEAF) if persistent \
            else BATCH_LEAF_CANDIDATES
        self.orders = [int(v) for v in inputs.batch_orders(count, seed=w["seed"], lo=32, hi=min(1024, n))]
        self.As = [inputs.sdd_device(m, w["seed"] + 1000 * 3 + j, device) for j, m in enumerate(self.orders)]
        self.Xs = [torch.empty_like(a) for a in self.As]
        self.flops = sum(2.0 * float(m) ** 3 for m in self.orders)
        self.Ahs = [a.cpu().pin_memory() for a in self.As]
        self.Xhs = [torch.empty_like(a) for a in self.Ahs]
        self.h2d = self.d2h = sum(8 * m * m for m in self.orders)
        self.info = None
        self.tuned = None
        if leaf == 0:
            # per order bucket, the fastest leaf on a bucket of the same size
            # (outside the timed region); leaf 0 then uses the records
            t0 = time.perf_counter()
            if persistent:
                # leaf and largest product tile per order bucket, on the persistent kernel
                rec = spin.autotune_batched_persistent(self.orders, leaves=cands, tiles=BATCH_TILE_CANDIDATES)
                tiles = {}
                for m in sorted(set(self.orders)):
                    tiles.setdefault(str(rec[m][1]), []).append(m)
            else:
                rec = spin.autotune_batched_leaf(self.orders, self.precision, candidates=cands)
            chosen = {}
            for m in sorted(set(self.orders)):
                chosen.setdefault(str(rec[m][0]), []).append(m)
            self.tuned = {"candidates": list(cands), "leaf_orders": chosen,
                          **({"tile_candidates": list(BATCH_TILE_CANDIDATES), "tile_orders": tiles}
                             if persistent else {}),
                          "tuning_s": time.perf_counter() - t0}

    def step(self):
        _, self.info = self.spin.invert_batched(self.As, leaf=self.leaf, outs=self.Xs, blocking=False,
                                                precision=self.precision, schedule=self.schedule)

    def launches(self, recs, steps):
        return self.spin.batched_stats()["kernels"] * steps

    def schedule_desc(self):
        if self.precision == "fp64" and self.schedule != "lockstep":
            return "persistent: one launch over a device-side task list (leaves <= 64 on one CTA, product tiles)"
        return "lockstep: per order bucket one launch per product and per leaf, buckets on 8 streams"

    def finish(self):
        import torch

        torch.cuda.synchronize()
        bad = int((self.info != 0).sum())
        out = {"status": 0 if bad == 0 else 2, "refine_iters": 0, "rel_residual": -1.0, "failed": bad}
        if self.precision != "fp64":
            ri = self.spin.batched_refine_info()
            out["refine_iters"], out["rel_residual"] = ri["refine_iters"], ri["worst_rel_residual"]
        return out

    def e2e_step(self):
        import torch

        for a, ah in zip(self.As, self.Ahs):
            a.copy_(ah, non_blocking=True)
        self.spin.invert_batched(self.As, leaf=self.leaf, outs=self.Xs, blocking=False, precision=self.precision,
                                 schedule=self.schedule)
        for x, xh in zip(self.Xs, self.Xhs):
            xh.copy_(x, non_blocking=True)
        torch.cuda.synchronize()

    def accuracy(self, probes):
        worst = 0.0
        for j in range(0, len(self.As), max(1, len(self.As) // 16)):
            worst = max(worst, freivalds_rel(self.As[j], self.Xs[j], 4, SEED_BASE + 77))
        return {"rel_residual_est": worst, "rel_residual_note": "max over 16 sampled matrices, 4 probes each"}


def replica_rate(ms_local: float, flops_local: float, world: int, device):
    """Replicas (one matrix per rank, no collective on the data path): the
    job's time is the slowest rank's, its work the sum over ranks.  Returns
    (ms, TFLOP/s of the whole job)."""
    if world <= 1:
        return ms_local, flops_local / (ms_local * 1e-3) / 1e12
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    f = torch.tensor([flops_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(f, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return ms, float(f.item()) / (ms * 1e-3) / 1e12


def time_work(spin, work, steps: int, warmup: int, stream, barrier, local: int) -> dict:
    """Warm-up calls through host buffers (each one also an end-to-end
    measurement: pinned host memory, H2D of the inputs and D2H of the results
    inside), then exactly `steps` device-resident steps between CUDA events
    on the launching stream, with launch records and nvidia-smi clock samples
    taken over the timed region."""
    import torch

    e2e_times = []
    for _ in range(warmup):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        work.e2e_step()
        e2e_times.append(time.perf_counter() - t0)
    if warmup == 0:
        work.step()  # at least one warm call
        work.finish()
    # Steps under a second: the launch records come from a second pass of the
    # same steps, so that the timed region runs as a user's calls do
    # (repeated calls replay the captured schedule; recording events around
    # every launch would run it launch by launch).  Longer steps record in
    # the timed region, where the records cost nothing measurable.
    separate = bool(e2e_times) and statistics.median(e2e_times) < 1.0
    with ClockSampler(local) as clk:
        barrier()
        if not separate:
            spin.profile_start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            work.step()
        e1.record(stream)
        barrier()
        recs = None if separate else spin.profile_collect()
        info = work.finish()
    if separate:
        barrier()
        spin.profile_start()
        for _ in range(steps):
            work.step()
        barrier()
        recs = spin.profile_collect()
        work.finish()
    return {"ms_local": e0.elapsed_time(e1) / steps, "e2e_times": e2e_times, "recs": recs, "info": info,
            "clocks": clk.summary(), "records": "separate pass of the same steps" if separate else "timed region"}


def kernel_table(recs) -> dict:
    by_kind: dict = {}
    for r in recs:
        d = by_kind.setdefault(r["kind"], {"ms": 0.0, "flops": 0.0, "bytes": 0.0, "launches": 0})
        d["ms"] += r["ms"]
        d["flops"] += r["flops"]
        d["bytes"] += r["bytes"]
        d["launches"] += 1
    return by_kind


def tensor_peak(peaks: dict):
    """Tensor-core kernels timed inside a long step: the sustained BF16 peak."""
    peak = peaks.get("bf16_tflops_sustained")
    if peak is None:
        return 1700.0, "fallback 1.7 PFLOP/s sustained BF16 (of fallback)"
    return peak, "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)"


def top_roofline(by_kind: dict, ms_step: float, steps: int, peaks: dict, peak_fp64: float):
    if not by_kind:
        return None
    top = max(by_kind, key=lambda k: by_kind[k]["ms"])
    d = by_kind[top]
    achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
    if top in ("gemm_tc", "residual", "update"):
        peak, src = tensor_peak(peaks)
        return {"kernel": top, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "peak_source": src,
                "flops_counted": "BF16 tensor-core products actually issued (slice pairs x 2mnk)",
                "launches": d["launches"], "share_of_step": d["ms"] / (ms_step * steps)}
    return {"kernel": top, "bound": "alu", "achieved": achieved, "peak": peak_fp64, "unit": "TFLOP/s",
            "frac": achieved / peak_fp64, "traffic": None,
            "traffic_note": ("gemm_f64: ncu dram read+write was 0.96 GB for a 4096^3 launch and 12.7 GB for "
                             "8192^3 (algorithmic 0.40 and 1.61 GB); it does not grow in proportion to the "
                             "flops, and this workload's launches were not captured" if top == "gemm_f64"
                             else "not captured"),
            "peak_source": "FP64 FMA rate measured live by spin_probe_fp64_peak on this GPU",
            "launches": d["launches"], "share_of_step": d["ms"] / (ms_step * steps)}


def run_ours(args, w: dict, n: int, leaf: int):
    import torch

    import paper_1801_04723_gb300 as spin

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=device)
    spin.build()
    spin.lib()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    if w["family"] == "batch_sdd":
        work = BatchWork(spin, w, n, leaf, device, args.batch_count, args.batch_schedule)
    else:
        work = SingleWork(spin, w, n, leaf, device, args.pretransform, args.fp64_levels, args.schedule)
    stream = torch.cuda.current_stream()
    flops = work.flops

    # FP64 peak, live: the DFMA probe (the plain path's roofline denominator)
    # and the DMMA probe beside it, with the SM clock sampled meanwhile
    with ClockSampler(local) as pclk:
        dfma = [spin.probe_fp64_peak() for _ in range(3)]
        dmma = [spin.probe_fp64_mma_peak() for _ in range(3)]
    peak_fp64 = max(dfma)
    probe = {"dfma_tflops": max(dfma), "dmma_tflops": max(dmma), "clocks": pclk.summary(),
             "how": "spin_probe_fp64_peak (8 DFMA chains per thread) and spin_probe_fp64_mma_peak (8 mma.sync "
                    "m8n8k4 f64 chains per warp), 4 x 256 threads per SM, best of 3 launches, 3 calls each"}
    t = time_work(spin, work, args.steps, args.warmup, stream, barrier, local)
    recs, info = t["recs"], t["info"]
    ms, value = replica_rate(t["ms_local"], flops, world, device)
    acc = work.accuracy(args.probes)

    mixed = batched = served = None
    # seconds since the start of the process at the end of each phase
    timeline = {"plain_s": time.perf_counter() - T_START}
    # A sub-record that fails is reported as such; the plain line (measured
    # above) is printed either way.
    def guarded(fn):
        try:
            return fn()
        except Exception as e:  # noqa: BLE001 -- reported in the line
            print(f"[bench] sub-record failed: {e!r}", file=sys.stderr, flush=True)
            return {"error": repr(e)[:400]}

    if args.workload == "plain_fp64" and not args.no_mixed:
        mixed = guarded(lambda: mixed_subrecord(args, spin, work, n, ms, device, stream, barrier, local, world,
                                                peak_fp64))
        timeline["mixed_s"] = time.perf_counter() - T_START
    # the batching and serving forms, while the run stays well inside its
    # time limit (the plain steps take most of it)
    if args.workload == "plain_fp64" and not args.no_batched and world == 1:
        if time.perf_counter() - T_START < BATCHED_DEADLINE_S:
            batched = guarded(lambda: batched_subrecord(args, spin, device, stream, barrier, local, world,
                                                        peak_fp64))
            timeline["batched_s"] = time.perf_counter() - T_START
        else:
            batched = {"skipped": f"run time above {BATCHED_DEADLINE_S:.0f} s"}
    if args.workload == "plain_fp64" and not args.no_serve and world == 1:
        if time.perf_counter() - T_START < SERVE_DEADLINE_S:
            def serve_sub():
                sargs = argparse.Namespace(**vars(args))
                sargs.serve_seconds = args.serve_sub_seconds
                out = run_serve(sargs, dict(WORKLOADS["serve"]), sub=True)
                return {k: v for k, v in out.items()
                        if k not in ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data")}
            served = guarded(serve_sub)
            timeline["serve_s"] = time.perf_counter() - T_START
        else:
            served = {"skipped": f"run time above {SERVE_DEADLINE_S:.0f} s"}

    if rank != 0:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel, from the in-region launch records
    by_kind = kernel_table(recs)
    peaks = measured_peaks()
    roof = None
    if isinstance(work, BatchWork) and work.precision == "fp64":
        # the batch replays one CUDA graph: no per-launch events; the whole
        # graph is FP64-pipe bound (batched products and leaves)
        roof = {"kernel": ("persistent_batch_kernel (product tiles and leaves, one launch)"
                           if work.schedule != "lockstep" else
                           "batched graph (gemm_f64_batched_kernel + leaf_gj_cta_kernel)"), "bound": "alu",
                "achieved": value / world, "peak": peak_fp64, "unit": "TFLOP/s", "frac": value / world / peak_fp64,
                "traffic": None, "peak_source": "FP64 FMA rate measured live by spin_probe_fp64_peak on this GPU"}
    elif isinstance(work, BatchWork):
        # mixed batch: graph + refinement launches, no per-launch events; the
        # effective rate against the FP64 peak is what the form buys
        roof = {"kernel": "mixed batch (tc_gemm_kernel batched + leaves + refinement), whole call", "bound": "alu",
                "achieved": value / world, "peak": peak_fp64, "unit": "TFLOP/s", "frac": value / world / peak_fp64,
                "traffic": None, "peak_source": "FP64 FMA rate measured live by spin_probe_fp64_peak on this GPU",
                "note": "effective 2n^3/t over the FP64 peak (above 1 means the tensor-core form beats FP64)"}
    top_roof = top_roofline(by_kind, ms, args.steps, peaks, peak_fp64)
    if top_roof is not None:
        roof = top_roof
    e2e_times = t["e2e_times"]
    e2e_ok = e2e_times[1:] if len(e2e_times) > 1 else e2e_times
    e2e_t = statistics.median(e2e_ok) if e2e_ok else None
    batch = isinstance(work, BatchWork)
    config = {"workload": args.workload, "n": n, "leaf": leaf, "precision": w["precision"],
              **({"pretransform": args.pretransform} if args.pretransform else {}),
              **({"fp64_levels": args.fp64_levels} if w["precision"] != "fp64" else {}),
              "matrices_per_gpu": len(work.orders) if batch else 1, "parallelism": f"replicas{world}",
              "desc": w["desc"], "launch_records": t["records"]}
    if batch:
        config["l2"] = f"inputs larger than L2 ({work.h2d / 1e9:.1f} GB of matrices)"
        config["orders"] = {"min": min(work.orders), "max": max(work.orders), "distinct": len(set(work.orders))}
        config["schedule"] = work.schedule_desc()
        if work.tuned is not None:
            config["leaf"] = "autotuned per order"
            config["leaf_autotune"] = work.tuned
    else:
        config["l2"] = (f"inputs larger than L2 ({8 * n * n / 1e9:.1f} GB per matrix)" if n >= 4096 else
                        "inputs smaller than L2; no flush between steps")
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if w["precision"] == "fp64" else ("bf16x3+f64" if w["precision"] == "bf16x3" else "bf16-digits+f64"), "data": "synthetic",
        "config": config,
        "clocks": t["clocks"],
        "e2e": {"value": flops / e2e_t / 1e12 if e2e_t else None, "unit": "TFLOP/s",
                "h2d_bytes_per_step": work.h2d, "d2h_bytes_per_step": work.d2h,
                "how": "host buffers (pinned), copies inside the timed call, warm-up steps 2..W, host wall clock"},
        "cold": {"first_call_ms": e2e_times[0] * 1e3 if e2e_times else None,
                 "how": "the first end-to-end call of the process: workspace allocation, module load and "
                        "copies included"},
        "gpu_launches": work.launches(recs, args.steps) + (mixed.get("gpu_launches", 0) if mixed else 0)
        + sum(batched[k]["gpu_launches"] for k in ("batched_fp64", "batched_mixed") if batched and k in batched),
        "roofline": roof,
        "status": info["status"],
        "refine_iters": info.get("refine_iters"),
        "rel_residual_lib": info.get("rel_residual"),
        "fp64_peak_tflops": peak_fp64,
        "fp64_probe": probe,
        "frac_of_fp64_peak": value / world / peak_fp64,
        "bf16_peak_tflops": peaks.get("bf16_tflops"),
        "frac_of_bf16_peak": value / world / peaks["bf16_tflops"] if peaks.get("bf16_tflops") else None,
        "kernels": {k: {"launches": v["launches"], "ms": v["ms"], "tflops": v["flops"] / max(v["ms"], 1e-9) / 1e9}
                    for k, v in by_kind.items()},
    }
    line.update(acc)
    if mixed is not None:
        line["mixed"] = mixed
    if batched is not None:
        line["batched"] = batched
    if served is not None:
        line["serve"] = served
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    timeline["end_s"] = time.perf_counter() - T_START
    line["timeline"] = timeline
    if args.profile_json:
        with open(args.profile_json, "w") as f:
            json.dump(recs, f)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def mixed_subrecord(args, spin, plain_work, n: int, plain_ms: float, device, stream, barrier, local: int,
                    world: int, peak_fp64: float) -> dict:
    """The mixed-precision form on the same GPU in the same process: one SPD
    matrix of order n with known inverse (A = Q diag(d) Q^T, 64 Householder
    reflectors, d log-uniform in [1, 1e3]), BF16x3 tensor-core level
    products, FP64 leaves, FP64-class top-two Schur complements and residual,
    Newton-Schulz to residual <= 1e-10; timed like the plain form (CUDA events
    over the steps, e2e through spin_invert_host) and compared with it."""
    import gc

    import torch

    # the plain form's buffers (A, X, pinned host copies) are not needed any more
    for name in ("A", "X", "Ah", "Xh"):
        if hasattr(plain_work, name):
            setattr(plain_work, name, None)
    gc.collect()
    torch.cuda.empty_cache()
    wm = dict(WORKLOADS["mixed_bf16x3"])
    wm["n"] = n
    leaf_m = wm["leaf"]
    steps = max(1, min(args.steps, args.mixed_steps))
    warmup = max(1, min(args.warmup, args.mixed_warmup))
    work = SingleWork(spin, wm, n, leaf_m, device, 0, args.fp64_levels)
    t = time_work(spin, work, steps, warmup, stream, barrier, local)
    ms, value = replica_rate(t["ms_local"], work.flops, world, device)
    acc = work.accuracy(args.probes)
    by_kind = kernel_table(t["recs"])
    roof = top_roofline(by_kind, ms, steps, measured_peaks(), peak_fp64)
    e2e_times = t["e2e_times"]
    e2e_ok = e2e_times[1:] if len(e2e_times) > 1 else e2e_times
    e2e_t = statistics.median(e2e_ok) if e2e_ok else None
    info = t["info"]
    return {
        "workload": "mixed_bf16x3", "desc": wm["desc"], "n": n, "leaf": leaf_m, "precision": "bf16x3",
        "fp64_levels": args.fp64_levels, "tol": 1e-10, "steps": steps, "warmup": warmup,
        "value": value, "unit": "TFLOP/s", "ms_per_step": ms,
        "speedup_vs_plain": plain_ms / ms,
        "status": info["status"], "refine_iters": info.get("refine_iters"),
        "rel_residual_lib": info.get("rel_residual"),
        **acc,
        "clocks": t["clocks"],
        "e2e": {"value": work.flops / e2e_t / 1e12 if e2e_t else None, "unit": "TFLOP/s",
                "h2d_bytes_per_step": work.h2d, "d2h_bytes_per_step": work.d2h,
                "how": "spin_invert_host on pinned host buffers, copies inside the timed call, warm-up steps "
                       "2..W (step 1 if W = 1), host wall clock"},
        "cold": {"first_call_ms": e2e_times[0] * 1e3 if e2e_times else None},
        "roofline": roof,
        "gpu_launches": len(t["recs"]),
        "launch_records": t["records"],
        "kernels": {k: {"launches": v["launches"], "ms": v["ms"], "tflops": v["flops"] / max(v["ms"], 1e-9) / 1e9}
                    for k, v in by_kind.items()},
    }


def batched_subrecord(args, spin, device, stream, barrier, local: int, world: int, peak_fp64: float) -> dict:
    """The batching workload (4096 matrices of orders 32..1024) on the same
    GPU in the same process, FP64 and mixed, each with its leaves autotuned
    per order bucket before the timed steps; the mixed batch is compared
    with the FP64 batch."""
    import gc

    import torch

    out = {}
    steps, warmup = max(1, min(args.steps, 3)), max(3, min(args.warmup, 3))
    for name in ("batched_fp64", "batched_mixed"):
        wb = dict(WORKLOADS[name])
        work = BatchWork(spin, wb, wb["n"], 0, device, BATCH_COUNT, args.batch_schedule)
        t = time_work(spin, work, steps, warmup, stream, barrier, local)
        ms, value = replica_rate(t["ms_local"], work.flops, world, device)
        fin = t["info"]
        acc = work.accuracy(args.probes)
        e2e_ok = t["e2e_times"][1:] if len(t["e2e_times"]) > 1 else t["e2e_times"]
        e2e_t = statistics.median(e2e_ok) if e2e_ok else None
        out[name] = {
            "desc": wb["desc"], "precision": wb["precision"], "matrices": len(work.orders),
            "orders": {"min": min(work.orders), "max": max(work.orders), "distinct": len(set(work.orders))},
            "leaf_autotune": work.tuned, "schedule": work.schedule_desc(), "steps": steps, "warmup": warmup,
            "value": value, "unit": "TFLOP/s", "ms_per_step": ms, "frac_of_fp64_peak": value / world / peak_fp64,
            "failed": fin["failed"], "refine_iters": fin["refine_iters"], "worst_rel_residual_lib": fin["rel_residual"],
            **acc,
            "clocks": t["clocks"],
            "e2e": {"value": work.flops / e2e_t / 1e12 if e2e_t else None, "unit": "TFLOP/s",
                    "h2d_bytes_per_step": work.h2d, "d2h_bytes_per_step": work.d2h,
                    "how": "pinned host buffers, copies inside the timed call, warm-up steps 2..W, host wall clock"},
            "gpu_launches": work.launches(t["recs"], steps),
        }
        del work, t
        gc.collect()
        torch.cuda.empty_cache()
    out["mixed_speedup_vs_fp64_batch"] = out["batched_fp64"]["ms_per_step"] / out["batched_mixed"]["ms_per_step"]
    return out


def run_serve(args, w: dict, sub: bool = False):
    """Serving benchmark: replay a Poisson arrival trace against spin_serve_*.

    A producer thread generates every request's matrix on the device ahead
    of its arrival time (a bounded look-ahead in bytes); the main thread
    submits each at its arrival time and polls finished requests.  Every
    arrival of the trace is accounted for: submitted (then served or failed),
    shed by the server's queue bound, or not generated (a generation failure,
    reported, never silently dropped).  Latency is taken from the arrival
    time in the trace (the server's own submit-to-finish latency is reported
    beside it)."""
    import queue
    import threading

    # many distinct matrix sizes come and go: let the caching allocator grow
    # and shrink segments instead of fragmenting fixed ones
    os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "expandable_segments:True")
    import torch

    import paper_1801_04723_gb300 as spin
    from paper_1801_04723_gb300 import inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    spin.build()
    spin.lib()
    trace = inputs.serve_trace(w["seed"] + 1000 * rank, rate=args.serve_rate, duration=args.serve_seconds,
                               lo=64, hi=min(8192, w["n"]))
    # the client's input generation must keep up with the trace while the
    # server saturates the GPU: its kernels go ahead of the server's pending blocks
    lo_prio, hi_prio = torch.cuda.Stream.priority_range()
    gen_stream = torch.cuda.Stream(device, priority=hi_prio)

    def make(j, n, alpha):
        # G G^T / n on the TF32 tensor cores (input preparation only: the
        # product's rounding is far below alpha >= 0.1, so A stays SPD), then
        # symmetrised in FP64
        with torch.cuda.stream(gen_stream):
            prev = torch.backends.cuda.matmul.allow_tf32
            torch.backends.cuda.matmul.allow_tf32 = True
            try:
                G = inputs.normal_torch(w["seed"] + 7919 * (j + 1), n, n, 0, device, torch.float32)
                A = (G @ G.T).double() / float(n)
            finally:
                torch.backends.cuda.matmul.allow_tf32 = prev
            A = 0.5 * (A + A.T)
            A.diagonal().add_(alpha)
            del G
            ev = torch.cuda.Event()
            ev.record(gen_stream)
        return A, ev

    lookahead_bytes = 4 << 30
    ready = queue.Queue()
    cond = threading.Condition()
    state = {"ahead": 0, "gen_retries": 0, "gen_failed": [], "error": None}

    def producer():
        try:
            for j, (t, n, alpha, mixed) in enumerate(trace):
                nb = 8 * n * n
                with cond:  # bounded look-ahead in bytes
                    while state["ahead"] > 0 and state["ahead"] + nb > lookahead_bytes:
                        cond.wait(timeout=0.05)
                A = ev = None
                for attempt in range(200):
                    try:
                        A, ev = make(j, n, alpha)
                        break
                    except torch.OutOfMemoryError:
                        # the client's memory frees as results are polled: wait, then retry
                        state["gen_retries"] += 1
                        torch.cuda.empty_cache()
                        time.sleep(0.05)
                if A is None:
                    state["gen_failed"].append(j)
                    ready.put((j, t, n, mixed, None, None))
                    continue
                with cond:
                    state["ahead"] += nb
                ready.put((j, t, n, mixed, A, ev))
        except BaseException as e:  # reported by the main loop, which then stops
            state["error"] = repr(e)
        finally:
            ready.put(None)

    # Offered load beyond what the GPU serves makes the queue grow; requests
    # whose A would take the queued bytes above 48 GB are shed (the A of
    # queued requests stays in the client's device memory).
    srv = spin.Server(hbm_budget_bytes=150 << 30, max_slots=args.serve_slots, max_queued_bytes=48 << 30,
                      priority_order=args.serve_priority_order, max_batch=args.serve_max_batch)
    pending = {}
    done = []
    shed = 0
    submit_lag = {}
    # warm the kernels once (both paths, batched and single) outside the measured window
    for prec, tol in (("bf16x3", 1e-10), ("fp64", 1e-13), ("bf16x3", 1e-13)):
        for nw in (256, 1536):
            Aw, ev = make(10 ** 6, nw, 0.5)
            ev.synchronize()
            tk = srv.submit(Aw, precision=prec, tol=tol)
            while srv.poll(tk, discard=True) is None:
                time.sleep(0.001)
    st0 = srv.stats()
    th = threading.Thread(target=producer, daemon=True)
    th.start()
    t0 = time.perf_counter()

    def collect():
        for tk in list(pending):
            got = srv.poll(tk, discard=True)
            if got is not None:
                j, n, t_arr = pending.pop(tk)
                r = got[1]
                r["n"] = n
                r["latency_from_arrival_ms"] = r["latency_ms"] + submit_lag[tk]
                done.append(r)

    submitted = 0
    # Finished requests are polled on every pass of the loop, also while the
    # client waits for the producer: results that nobody polls hold the
    # server's budget, and the producer may be waiting for that memory.
    # A run that makes no progress for stall_s aborts with its counters.
    stall_s = 60.0 if sub else 300.0
    progress = {"t": time.perf_counter(), "done": 0, "last_print": time.perf_counter()}

    def check_progress(where):
        now = time.perf_counter()
        if len(done) != progress["done"] or submitted != progress.get("submitted"):
            progress.update(t=now, done=len(done), submitted=submitted)
        if now - progress["last_print"] > 10.0:
            progress["last_print"] = now
            free, _ = torch.cuda.mem_get_info()
            print(f"[serve] t={now - t0:.0f}s submitted={submitted} done={len(done)} pending={len(pending)} "
                  f"shed={shed} ahead={state['ahead'] >> 20} MB device_free={free >> 30} GB "
                  f"server={srv.stats()}", file=sys.stderr, flush=True)
        if now - progress["t"] > stall_s:
            raise RuntimeError(f"serving run made no progress for {stall_s:.0f} s ({where}): submitted={submitted} "
                               f"done={len(done)} pending={len(pending)} shed={shed} "
                               f"generation_retries={state['gen_retries']} server={srv.stats()}")

    def next_item():
        while True:
            collect()
            try:
                return ready.get(timeout=0.002)
            except queue.Empty:
                check_progress("waiting for input generation")

    with ClockSampler(local) as clk:
        while True:
            item = next_item()
            if item is None:
                break
            j, t_arr, n, mixed, A, ev = item
            if A is None:
                continue  # counted as not generated
            while time.perf_counter() - t0 < t_arr:
                collect()  # poll finished requests while waiting for the next arrival
                time.sleep(0.0005)
            check_progress("submitting")
            ev.synchronize()
            if mixed:
                prec, tol = "bf16x3", 1e-10
            else:
                prec, tol = ("bf16x3" if args.serve_fp64_path == "mixed" else "fp64"), 1e-13
            t_sub = time.perf_counter() - t0
            tk = srv.submit(A, precision=prec, tol=tol)
            with cond:
                state["ahead"] -= 8 * n * n
                cond.notify_all()
            del A
            if tk is None:
                shed += 1
                continue
            submitted += 1
            submit_lag[tk] = (t_sub - t_arr) * 1e3
            pending[tk] = (j, n, t_arr)
        t_last_arrival = time.perf_counter() - t0
        while pending:
            collect()
            check_progress("draining")
            time.sleep(0.001)
        makespan = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    if state["error"] is not None:
        raise RuntimeError(f"input generation failed: {state['error']}")
    arrivals = len(trace)
    not_generated = len(state["gen_failed"])
    assert arrivals == submitted + shed + not_generated, (arrivals, submitted, shed, not_generated)
    assert len(done) == submitted
    lat = sorted(r["latency_from_arrival_ms"] for r in done)
    lat_srv = sorted(r["latency_ms"] for r in done)
    bad = sum(1 for r in done if r["status"] != 0)
    failed_status = {}
    for r in done:
        if r["status"] != 0:
            failed_status[str(r["status"])] = failed_status.get(str(r["status"]), 0) + 1
    failed_detail = [{k: r[k] for k in ("status", "n", "precision", "refine_iters", "rel_residual")}
                     for r in done if r["status"] != 0][:20]

    def pct(v, q):
        return v[min(len(v) - 1, int(q * len(v)))] if v else None

    flops_trace = sum(2.0 * float(n) ** 3 for _, n, _, _ in trace)
    flops_done = sum(2.0 * float(r["n"]) ** 3 for r in done if r["status"] == 0)
    served_ok = sum(1 for r in done if r["status"] == 0)
    line = {
        "metric": METRIC, "value": served_ok / makespan, "unit": "req/s", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": makespan * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3+f64", "data": "synthetic",
        "config": {"workload": "serve", "rate_req_s": args.serve_rate, "arrival_window_s": args.serve_seconds,
                   "requests": arrivals, "n_range": [64, min(8192, w["n"])], "slots": args.serve_slots,
                   "priority_order": args.serve_priority_order, "max_batch": args.serve_max_batch,
                   "hbm_budget_gb": 150, "fp64_class_path": args.serve_fp64_path, "desc": w["desc"],
                   "inputs": "A = G G^T / n + alpha I generated on the device ahead of arrival (G G^T on TF32 "
                             "tensor cores, symmetrised in FP64; a high-priority stream), at most 4 GB ahead"},
        "arrivals": arrivals, "submitted": submitted, "served": served_ok, "failed": bad, "shed": shed,
        "client_lag_s": {"p50": pct(sorted(submit_lag.values()), 0.5) / 1e3 if submit_lag else None,
                         "max": max(submit_lag.values()) / 1e3 if submit_lag else None,
                         "note": "submit time minus arrival time in the trace (input generation falling behind)"},
        "not_generated": not_generated, "generation_retries": state["gen_retries"],
        "p50_ms": pct(lat, 0.50), "p99_ms": pct(lat, 0.99), "max_ms": lat[-1] if lat else None,
        "latency_from": "arrival time in the trace (p50_ms, p99_ms, max_ms)",
        "server_p50_ms": pct(lat_srv, 0.50), "server_p99_ms": pct(lat_srv, 0.99),
        "offered_req_s": arrivals / args.serve_seconds,
        "offered_tflops": flops_trace / args.serve_seconds / 1e12,
        "served_tflops": flops_done / makespan / 1e12,
        "drain_s_after_last_arrival": makespan - t_last_arrival,
        "failed_status": failed_status, "failed_detail": failed_detail,
        "peak_running": st["peak_running"], "deferred": st["deferred"] - st0["deferred"],
        "batching": {"groups": st["groups"] - st0["groups"], "requests_in_groups": st["grouped"] - st0["grouped"],
                     "largest_group": st["max_group"]},
        "clocks": clk.summary(),
        "e2e": {"value": served_ok / makespan, "unit": "req/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "how": "requests submitted from device memory; results left on the device"},
        "gpu_launches": None,
    }
    if sub:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_gemm_probe(args):
    """One digit-slice (6 slices, 21 pairs: the refinement residual's form)
    and one bf16x3 tensor-core product of order n, each timed 3 times after a
    warm-up (CUDA events, splits included), with the SM clock sampled over
    the timed calls: the kernel variant switches (SPIN_TC_WIDE, SPIN_TC_PAIR)
    are compared this way, clock and all."""
    import torch

    import paper_1801_04723_gb300 as spin
    from paper_1801_04723_gb300 import inputs

    spin.build()
    n = args.gemm_probe
    A = inputs.sdd_device(n, SEED_BASE + 11, "cuda")
    B = inputs.sdd_device(n, SEED_BASE + 12, "cuda")
    D = torch.empty_like(A)
    out = {"probe": "tensor-core products", "n": n,
           "variant": {k: os.environ.get(k, "") for k in ("SPIN_TC_WIDE", "SPIN_TC_PAIR", "SPIN_TC_PERSIST")}}
    for name, fn, pairs in (("ozaki6", lambda: spin.gemm_ozaki(A, B, slices=6, out=D), 21),
                            ("bf16x3", lambda: spin.gemm_bf16x3(A, B, out=D), 3)):
        fn()  # warm
        torch.cuda.synchronize()
        times = []
        with ClockSampler(0) as clk:
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        out[name] = {"ms_with_splits": ms, "bf16_tflops_incl_splits": pairs * 2.0 * n ** 3 / (ms * 1e-3) / 1e12,
                     "clocks": clk.summary()}
    out["device_error"] = spin.take_device_error()
    print(json.dumps(out), flush=True)
    return 0


def run_leaf_sweep(args):
    import torch

    import paper_1801_04723_gb300 as spin

    spin.build()
    prec = "fp64" if args.workload in ("plain_fp64", "small_fp64", "batched_fp64") else "bf16x3"
    cands = (64, 128, 256, 512, 1024, 2048)
    out = {"sweep": "leaf", "precision": prec, "candidates": list(cands), "results": []}
    for n in [int(v) for v in args.leaf_sweep.split(",") if v]:
        best, ms = spin.autotune_leaf(n, prec, cands)
        out["results"].append({"n": n, "best_leaf": best,
                               "ms": {str(k): v for k, v in ms.items()},
                               "tflops": {str(k): 2.0 * n ** 3 / (v * 1e-3) / 1e12 for k, v in ms.items()}})
    torch.cuda.synchronize()
    print(json.dumps(out), flush=True)
    return 0


def run_leaf_times(args):
    """The leaf kernel alone: CUDA events around one spin_leaf_inverse launch
    per order (best of 5 after 2 warm-ups), on a seeded diagonally dominant
    matrix; per pivot step = time / L.  These are the per-step times the
    cost model's leaf constants come from."""
    import torch

    import paper_1801_04723_gb300 as spin
    from paper_1801_04723_gb300 import inputs

    spin.build()
    out = {"leaf_times": [], "how": "CUDA events around one spin_leaf_inverse launch, best of 5 after 2 warm-ups"}
    for L in [int(v) for v in args.leaf_times.split(",") if v]:
        A = torch.from_numpy(inputs.sdd(L, seed=inputs.SEED_BASE + L)).to("cuda:0")
        X = torch.empty_like(A)
        for _ in range(2):
            spin.leaf_inverse(A, out=X)
        best = float("inf")
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            spin.leaf_inverse(A, out=X)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out["leaf_times"].append({"L": L, "ms": best, "us_per_step": best * 1e3 / L})
    print(json.dumps(out), flush=True)
    return 0


def run_leaf_batch(args):
    """Many leaves side by side: `count` matrices of order L <= 128 through
    spin_invert_batched (plain FP64), where every matrix is one leaf, so a
    call is one leaf_gj_batched_kernel launch (one CTA per matrix) plus a
    status scatter.  CUDA events around each call, best of 5 after 2 warm-ups;
    per pivot step = time / L; with the SM clock sampled meanwhile."""
    import torch

    import paper_1801_04723_gb300 as spin
    from paper_1801_04723_gb300 import inputs

    spin.build()
    L, count = (int(v) for v in args.leaf_batch.split(":"))
    As = [torch.from_numpy(inputs.sdd(L, seed=inputs.SEED_BASE + 9000 + i)).to("cuda:0") for i in range(count)]
    Xs = [torch.empty_like(a) for a in As]
    for _ in range(2):
        spin.invert_batched(As, outs=Xs, schedule="lockstep")
    torch.cuda.synchronize()
    best = float("inf")
    with ClockSampler(0) as clk:
        for _ in range(3):
            # five calls back to back between the events: the host's
            # marshalling of the next call overlaps the previous call's kernel
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                _, info = spin.invert_batched(As, outs=Xs, blocking=False, schedule="lockstep")
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 5)
    assert int(info.abs().sum()) == 0
    c = clk.summary()
    mhz = c["sm_mhz"] or 2070.0
    per_step_us = best * 1e3 / L
    out = {"leaf_batch": {"L": L, "count": count, "ms": best, "us_per_step": per_step_us,
                          "cycles_per_step": per_step_us * mhz, "fma_per_step_per_leaf": L * L,
                          "fp64_bound_cycles_per_step": L * L / 2.0,
                          "how": "CUDA events around 5 back-to-back spin_invert_batched calls (per call), best of "
                                 "3 after 2 warm-ups"},
           "clocks": c}
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.leaf_times:
        return run_leaf_times(args)
    if args.leaf_batch:
        return run_leaf_batch(args)
    if args.leaf_sweep:
        return run_leaf_sweep(args)
    if args.gemm_probe:
        return run_gemm_probe(args)
    w = dict(WORKLOADS[args.workload])
    n = args.n if args.n > 0 else w["n"]
    leaf = args.leaf if args.leaf >= 0 else w["leaf"]
    w["n"], w["leaf"] = n, leaf
    if args.impl == "reference":
        return run_reference(args, w, n, leaf)
    if w["family"] == "serve":
        return run_serve(args, w)
    return run_ours(args, w, n, leaf)


if __name__ == "__main__":
    sys.exit(main())
