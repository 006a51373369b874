#!/usr/bin/env python
"""Benchmark: exact posteriors of all n(n-1) edges, n=26 binary variables,
in-degree d<=4, m=2000 samples (full 2^26 subset lattice), DP arrays in FP32
log2 domain with FP64 scores and normaliser.  Metric: subset-DP cells/s
(cells = n * 2^n per job).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp32|fp64] [--workload large|mid|small] [--shard]

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
replica of the job on its own GPU (no collective on the data path); value =
cells of all ranks / max time over ranks.  With --shard the ranks instead
split one job (paper_1408_1664_gb300.shard: an NCCL all-gather per exchange
step, an all-reduce of the posteriors); value = cells of the job / max time.
"--impl reference" times the CPU FP64 oracle (the only reference that exists)
on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1408_1664_gb300 import datagen  # noqa: E402

WORKLOADS = {
    "large": ("n26_d4_binary_m2000", datagen.config_large),
    "mid": ("n20_d4_arity3_m1000", datagen.config_mid),
    "small": ("n12_d3_binary_m200", datagen.config_small),
}
METRIC = "subset-DP cells/s"
UNIT = "cells/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--workload", default="large", choices=list(WORKLOADS))
    ap.add_argument("--no-fp64-extra", action="store_true",
                    help="skip the secondary FP64-path measurement")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--sweep", action="store_true",
                    help="the n and d sweep of the paper's experiments (prints one JSON table)")
    ap.add_argument("--subset-n", type=int, default=0,
                    help="use only the first N variables of the workload (profiling)")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the 256-job batched workload (prints its JSON object)")
    ap.add_argument("--batch-reps", type=int, default=5,
                    help="timed runs of the batch")
    ap.add_argument("--batch-graph", action="store_true",
                    help="with --batched-only: the graph form instead of the persistent launch")
    ap.add_argument("--degree", type=int, default=0,
                    help="override the workload's in-degree bound d (profiling)")
    ap.add_argument("--shard", action="store_true",
                    help="one job split over the ranks (strong scaling) instead of replicas")
    ap.add_argument("--divide-a", action="store_true",
                    help="with --shard: each rank holds only its slabs of A")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


# --------------------------------------------------------------- clocks --
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons, pw = [], [], set(), []
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names[1:], f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------ roofline helpers --
def measured_peaks() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


KERNEL_SOURCES = ("bn_kernels.cu", "bn_tile13.cu", "bn_levels.cu", "bn_device.cuh")


def kernel_source_sha(files=KERNEL_SOURCES) -> str:
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_1408_1664_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def committed_traffic(kernel: str, workload: str, precision: str):
    """dram bytes per launch from a committed ncu summary, only if it was
    taken on the current source of the kernel: each line names the files the
    kernel is compiled from (src=a+b) and their hash at the capture."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
        if (kv.get("kernel") == kernel and kv.get("workload") == workload
                and kv.get("precision") == precision and "src" in kv
                and kv.get("src_sha") == kernel_source_sha(tuple(kv["src"].split("+")))):
            return float(kv["dram_bytes_per_launch"])
    return None


def committed_fp64_ops() -> float | None:
    """FP64 pipe operations (DFMA + DADD + DMUL, per thread) per subset-DP
    cell of the FP64 path, from the committed ncu count in
    profiles/fp64_ops.txt, only while the kernels' sources hash as at the
    capture."""
    path = os.path.join(ROOT, "profiles", "fp64_ops.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kv = dict(tok.split("=", 1) for tok in line.split() if "=" in tok)
        if ("ops_per_cell" in kv and "src" in kv
                and kv.get("src_sha") == kernel_source_sha(tuple(kv["src"].split("+")))):
            return float(kv["ops_per_cell"])
    return None


def stage_table(n: int, d: int, es: int) -> dict:
    """Per kernel: algorithmic HBM bytes per launch, launches per job and how
    to read its device time from bn_stats.  "bytes" counts only the method's
    own arrays (A written once; A read by F and by R'; F and R' written and
    read once; the halves of F and R' read for every endpoint v: the minimal
    traffic of the five steps).  "bytes_with_intermediates" adds what this
    implementation moves besides: the up-zeta column sums and the down-zeta
    phase-1 rows W, which the method does not have."""
    from math import comb
    N = 2 ** n
    A_bytes = n * N / 2 * es                      # A: n 2^(n-1) values, written once
    # F / R' launches, one per level: row tiles of 16 subsets (FP32, n >= 5) or
    # 8 subsets (FP64, n >= 4), else warp tiles of 32 subsets
    rows = (es == 4 and n >= 5) or (es == 8 and n >= 4)
    nh = (n - (4 if es == 4 else 3) + 1) if rows else (n - min(n, 5) + 1)
    fwd, bwd = ("k_forward_rows", "k_backward_rows") if rows else ("k_forward_level",
                                                                   "k_backward_level")
    fr = (A_bytes + 2 * N * es) / nh              # A read once, F written and read once
    tab = {
        fwd: {"bytes": fr, "bytes_with_intermediates": fr, "launches": nh,
              "ms": lambda h: h["ms_forward"]},
        bwd: {"bytes": fr, "bytes_with_intermediates": fr, "launches": nh,
              "ms": lambda h: h["ms_backward"]},
    }
    if n >= 14:
        h = n - 1 - 13
        ncol = sum(comb(13, k) for k in range(min(d, 13) + 1))
        K = sum(comb(n - 1, k) for k in range(min(d, n - 1) + 1))
        C_bytes = n * 2 ** h * ncol * es          # column sums handed to the tile kernel
        tab["k_upzeta13"] = {"bytes": A_bytes, "bytes_with_intermediates": A_bytes + C_bytes,
                             "launches": 1,
                             "ms": lambda h: h["ms_upzeta"] - h["ms_upzeta_sums"]}
        tab["k_upzeta13_cols"] = {"bytes": 0.0,
                                  "bytes_with_intermediates": C_bytes + 2 * n * K * es,
                                  "launches": 1, "ms": lambda h: h["ms_upzeta_sums"]}
        # every endpoint v in one launch: the halves of F and R' read per v
        # (the method's bytes), one row of W per tile written (intermediate)
        tab["k_gamma13_p1"] = {"bytes": n * N * es,
                               "bytes_with_intermediates": n * (N + 2 ** h * ncol) * es,
                               "launches": 1, "ms": lambda h: h["ms_gamma_p1"]}
    else:
        tab["k_upzeta"] = {"bytes": A_bytes, "bytes_with_intermediates": A_bytes, "launches": 1,
                           "ms": lambda h: h["ms_upzeta"]}
        tab["k_gamma_p1"] = {"bytes": n * N * es, "bytes_with_intermediates": n * N * es,
                             "launches": 1, "ms": lambda h: h["ms_gamma_p1"]}
    return tab


def probe_peaks() -> dict:
    """Arithmetic rates measured on this GPU with CUDA events
    (_build/libbnpeaks.so): FP64 and FP32 FMA flop/s, MUFU ex2 ops/s and
    CUDA's FP64 exp() per second."""
    import ctypes as C

    from paper_1408_1664_gb300 import build as lib_build

    lib = C.CDLL(lib_build.LIB_PEAKS)
    out = {}
    for name, key in (("bn_peak_fp64_fma", "fp64_fma_flops"), ("bn_peak_fp32_fma", "fp32_fma_flops"),
                      ("bn_peak_ex2_f32", "ex2_f32_per_s"), ("bn_peak_exp_f64", "exp_f64_per_s")):
        fn = getattr(lib, name)
        fn.restype = C.c_int
        fn.argtypes = [C.c_int, C.POINTER(C.c_double)]
        v = C.c_double(0.0)
        out[key] = v.value if fn(4, C.byref(v)) == 0 else None
    return out


# ------------------------------------------------------------- replicas --
def replica_value(local_s: float, units_per_rank: float, dist=None, device="cpu"):
    """Independent replicas, one per rank: the job time is the maximum over
    ranks, and the value is the units of all ranks over that time.  Returns
    (max seconds, units per second).  `dist` is torch.distributed (None for
    one process); `device` holds the reduction tensor (the rank's GPU under
    NCCL, the CPU under gloo)."""
    world = 1
    if dist is not None:
        import torch
        t = torch.tensor([float(local_s)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local_s = float(t.item())
        world = dist.get_world_size()
    return local_s, world * units_per_rank / local_s


# ------------------------------------------------------------- CPU oracle --
def oracle_sample(ds, d, budget_s: float):
    """Time the oracle on sub-problems (the first n_s variables of the same
    data) of growing n_s until one run takes a sizeable share of the budget.
    Returns (cells/s, n_s, seconds, cores)."""
    from oracle import oracle as orc

    cores = orc.num_threads()
    best = None
    n_s = min(12, ds.n)
    spent = 0.0
    while True:
        sub = np.ascontiguousarray(ds.data[:, :n_s])
        t0 = time.perf_counter()
        orc.edge_posteriors(sub, ds.arity[:n_s], d)
        dt = time.perf_counter() - t0
        spent += dt
        best = (n_s * 2 ** n_s / dt, n_s, dt, cores)
        # each +1 variable roughly doubles (and more) the work
        if n_s >= ds.n or spent + 2.6 * dt > budget_s or dt > budget_s / 3:
            return best
        n_s += 1


def host_mem_available() -> int:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def oracle_full_run(ds, d, gpu_posts: dict) -> dict | None:
    """One full oracle run on the whole workload (all n variables), timed on
    the host cores, with its max abs error against each GPU result.  None when
    the host lacks the memory (A, F, R and four 2^n scratch arrays per
    thread, in doubles)."""
    from oracle import oracle as orc

    orc.build()
    n = ds.n
    need = 8 * (n * 2 ** n + 2 * 2 ** n + 4 * 2 ** n * orc.num_threads())
    if host_mem_available() < 1.2 * need:
        return None
    t0 = time.perf_counter()
    ref = orc.edge_posteriors(ds.data, ds.arity, d)
    dt = time.perf_counter() - t0
    out = {"value": n * 2 ** n / dt, "unit": UNIT, "cores": orc.num_threads(),
           "kind": "oracle",
           "sample": (f"one full oracle run on the whole workload (n={n}, d={d}, m={ds.m}): "
                      f"{n * 2 ** n} cells in {dt:.2f} s"),
           "seconds": dt}
    for k, p in gpu_posts.items():
        out[f"max_abs_err_{k}_vs_oracle"] = float(np.abs(p - ref["post"]).max())
    return out


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    name, fn = WORKLOADS[args.workload]
    ds, d = fn()
    from oracle import oracle as orc

    orc.build()
    # pick the sample size once (about 5 s per step), then time K steps
    rate, n_s, dt, cores = oracle_sample(ds, d, budget_s=12.0)
    sub = np.ascontiguousarray(ds.data[:, :n_s])
    for _ in range(args.warmup):
        orc.edge_posteriors(sub, ds.arity[:n_s], d)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.edge_posteriors(sub, ds.arity[:n_s], d)
    el = time.perf_counter() - t0
    value = args.steps * n_s * 2 ** n_s / el
    sample = (f"oracle (CPU FP64, OpenMP) on the first {n_s} of the {ds.n} variables of the "
              f"{name} workload (same data, d={d}); {n_s * 2 ** n_s} cells per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "n": ds.n, "d": d, "m": ds.m,
                   "precision": args.precision, "parallelism": f"replicas{world}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- serving --
def serving_trace(duration_s: float, rate: float = 200.0):
    """Seeded Poisson arrivals of small jobs (n 8..22, d=3, binary, m=500)
    with one n=29, m=2000 job every 10 s (at t = 1, 11, 21, ... s)."""
    arr = datagen.poisson_arrivals(rate, duration_s, seed=7)
    jobs = [(float(t),) + datagen.served_job(j) for j, t in enumerate(arr)]
    for b, t in enumerate(np.arange(1.0, duration_s, 10.0)):
        jobs.append((float(t),) + datagen.served_job(b, big=True))
    jobs.sort(key=lambda x: x[0])
    return jobs


def _pct(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if xs else None


def run_serving(binding, device: int, duration_s: float, sat_s: float = 8.0) -> dict:
    """Served FP32 path (bn_submit/bn_poll, 8 slots) against the plain FP64
    one-job-at-a-time path, (1) on the same open-loop arrival trace and (2)
    at saturation: a closed loop that keeps every slot busy (the plain path:
    back to back) for sat_s seconds over the trace's small jobs."""
    trace = serving_trace(duration_s)
    descs = [binding.Job(ds.data, ds.arity, d, precision="fp32") for _, ds, d in trace]
    out = {}
    # served: continuous batching
    lat, res = [], {}
    with binding.Context(device, slots=8) as ctx:
        pending = {}
        k = 0
        t0 = time.perf_counter()
        while k < len(trace) or pending:
            now = time.perf_counter() - t0
            while k < len(trace) and trace[k][0] <= now:
                pending[binding.bn_submit(ctx.h, descs[k])] = k
                k += 1
            for jid in list(pending):
                kk = pending[jid]
                rc, post, _ = binding.bn_poll(ctx.h, jid, trace[kk][1].n)
                if rc == binding.BN_EAGAIN:
                    continue
                if rc != binding.BN_OK:
                    raise binding.BnError(rc, "served job")
                lat.append(time.perf_counter() - t0 - trace[kk][0])
                res[kk] = post
                del pending[jid]
        span = time.perf_counter() - t0
    out["served_fp32"] = {"jobs": len(lat), "jobs_per_s": len(lat) / span,
                          "p50_ms": _pct(lat, 50) * 1e3, "p99_ms": _pct(lat, 99) * 1e3,
                          "slots": 8}
    # plain: FP64, one job at a time, first come first served
    lat64, err = [], 0.0
    with binding.Context(device, slots=1) as ctx:
        t0 = time.perf_counter()
        for kk, (t_arr, ds, d) in enumerate(trace):
            wait = t_arr - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            post, _ = binding.bn_edge_posteriors(ctx.h, binding.Job(ds.data, ds.arity, d,
                                                                    precision="fp64"))
            lat64.append(time.perf_counter() - t0 - t_arr)
            err = max(err, float(np.abs(post - res[kk]).max()))
        span64 = time.perf_counter() - t0
    out["plain_fp64"] = {"jobs": len(lat64), "jobs_per_s": len(lat64) / span64,
                         "p50_ms": _pct(lat64, 50) * 1e3, "p99_ms": _pct(lat64, 99) * 1e3}
    out["max_abs_err_fp32_vs_fp64"] = err
    nbig = sum(1 for _, ds, _ in trace if ds.n == 29)
    out["trace"] = (f"Poisson 200 jobs/s for {duration_s:g} s (seed 7): n~U[8,22], d=3, binary, "
                    f"m=500, plus one n=29, m=2000 job every 10 s ({nbig}); {len(trace)} jobs")
    out["saturation"] = run_saturation(binding, device, trace, sat_s)
    return out


def run_saturation(binding, device: int, trace, seconds: float) -> dict:
    """Closed loop over the trace's small jobs (in trace order, cycling): the
    served FP32 path keeps all 8 slots busy, the plain FP64 path runs one job
    after another.  Offered load = capacity, so jobs/s is each path's
    throughput; latency is submit to result."""
    small = [(ds, d) for _, ds, d in trace if ds.n < 29]
    out = {}
    lat, done, err = [], 0, 0.0
    with binding.Context(device, slots=8) as ctx:
        pending, k = {}, 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < seconds or pending:
            while len(pending) < 8 and time.perf_counter() - t0 < seconds:
                ds, d = small[k % len(small)]
                jid = binding.bn_submit(ctx.h, binding.Job(ds.data, ds.arity, d, precision="fp32"))
                pending[jid] = (k, time.perf_counter())
                k += 1
            for jid in list(pending):
                kk, ts = pending[jid]
                rc, post, _ = binding.bn_poll(ctx.h, jid, small[kk % len(small)][0].n)
                if rc == binding.BN_EAGAIN:
                    continue
                if rc != binding.BN_OK:
                    raise binding.BnError(rc, "served job")
                lat.append(time.perf_counter() - ts)
                done += 1
                del pending[jid]
        span = time.perf_counter() - t0
    out["served_fp32"] = {"jobs": done, "jobs_per_s": done / span,
                          "p50_ms": _pct(lat, 50) * 1e3, "p99_ms": _pct(lat, 99) * 1e3}
    lat64, done64 = [], 0
    with binding.Context(device, slots=1) as ctx:
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < seconds:
            ds, d = small[done64 % len(small)]
            ts = time.perf_counter()
            binding.bn_edge_posteriors(ctx.h, binding.Job(ds.data, ds.arity, d, precision="fp64"))
            lat64.append(time.perf_counter() - ts)
            done64 += 1
        span64 = time.perf_counter() - t0
    out["plain_fp64"] = {"jobs": done64, "jobs_per_s": done64 / span64,
                         "p50_ms": _pct(lat64, 50) * 1e3, "p99_ms": _pct(lat64, 99) * 1e3}
    out["how"] = (f"closed loop for {seconds:g} s over the trace's small jobs (n 8..22): "
                  "served FP32 keeps 8 jobs in flight, plain FP64 runs them back to back")
    return out


# ------------------------------------------------------------- batches --
def run_batched(binding, torch, device: int, jobs_n: int = 256, reps: int = 5) -> dict:
    """The batched workload (job j: seed 1000+j, n~U[10,18], d=3, arity
    U{2,3}, m~U[100,1000]) in FP32: the persistent form (one launch per run),
    the form the autotuner keeps (the faster of persistent and graph), and the
    tuned form end to end -- new data uploaded, run, every result downloaded,
    all inside the timed loop -- against the plain FP64 path running the same
    jobs one at a time."""
    jobs = [datagen.batched_job(j) for j in range(jobs_n)]
    cells = sum(ds.n * 2 ** ds.n for ds, _ in jobs)
    descs = lambda: [binding.Job(ds.data, ds.arity, d, precision="fp32") for ds, d in jobs]
    out = {}

    def device_ms(batch, stream):
        for _ in range(2):
            batch.run(stream)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            batch.run(stream)
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / reps

    stream = torch.cuda.Stream()
    with binding.Context(device, autotune=False) as ctx0:
        with binding.Batch(ctx0.h, descs()) as batch:
            ms = device_ms(batch, stream)
            line = [x for x in batch.describe().splitlines() if x.startswith("persistent")]
            out["batched_fp32_persistent"] = {"jobs": jobs_n, "ms_per_batch": ms,
                                              "jobs_per_s": jobs_n / (ms / 1e3),
                                              "cells_per_s": cells / (ms / 1e3),
                                              "kernel_launches_per_run": 1, "describe": line}
    with binding.Context(device) as ctx:
        t0 = time.perf_counter()
        batch = binding.Batch(ctx.h, descs())
        build_s = time.perf_counter() - t0
        ms = device_ms(batch, stream)
        text = batch.describe().strip().splitlines()
        form = "persistent" if any(x.endswith("in use") for x in text) else "graph"
        out["batched_fp32_tuned"] = {"jobs": jobs_n, "form": form, "ms_per_batch": ms,
                                     "jobs_per_s": jobs_n / (ms / 1e3),
                                     "cells_per_s": cells / (ms / 1e3),
                                     "build_ms_incl_autotune": build_s * 1e3,
                                     "describe": text}
        # end to end: upload (pinned staging, one copy), run, download (one copy)
        up = descs()
        batch.upload(up, stream)
        batch.run(stream)
        res, _ = batch.download()
        t0 = time.perf_counter()
        for _ in range(reps):
            batch.upload(up, stream)
            batch.run(stream)
            res, _ = batch.download()
        e2e_s = (time.perf_counter() - t0) / reps
        h2d = sum(ds.m * ds.n for ds, _ in jobs)
        d2h = sum(ds.n * ds.n * 8 + 8 for ds, _ in jobs)
        out["batched_fp32_tuned_e2e"] = {"ms_per_batch": e2e_s * 1e3, "jobs_per_s": jobs_n / e2e_s,
                                         "h2d_bytes_per_batch": h2d, "d2h_bytes_per_batch": d2h}
        batch.close()
        err = 0.0
        t0 = time.perf_counter()
        for k, (ds, d) in enumerate(jobs):
            post, _ = binding.bn_edge_posteriors(ctx.h, binding.Job(ds.data, ds.arity, d,
                                                                    precision="fp64"))
            err = max(err, float(np.abs(post - res[k]).max()))
        s64 = time.perf_counter() - t0
        out["plain_fp64_one_at_a_time"] = {"jobs": jobs_n, "s": s64, "jobs_per_s": jobs_n / s64,
                                           "cells_per_s": cells / s64,
                                           "how": "bn_edge_posteriors per job: host data in, "
                                                  "host posteriors out"}
        out["max_abs_err_fp32_vs_fp64"] = err
    return out


def run_batched_only(args) -> None:
    """The 256-job batch without autotuning, in its persistent form (one
    launch per precision) or, with --batch-graph, as the graph of launches:
    two warm-up runs and --batch-reps timed runs; used for launch lists and
    for timing either form alone."""
    import torch

    from paper_1408_1664_gb300 import binding

    binding.load(build_if_missing=True)
    jobs = [datagen.batched_job(j) for j in range(256)]
    with binding.Context(0, autotune=False, graph_batch=args.batch_graph) as ctx:
        batch = binding.Batch(ctx.h, [binding.Job(ds.data, ds.arity, d, precision="fp32")
                                      for ds, d in jobs])
        stream = torch.cuda.Stream()
        for _ in range(2):
            batch.run(stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.batch_reps):
            batch.run(stream)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / args.batch_reps
        groups = sum(1 for x in batch.describe().strip().splitlines()
                     if not x.startswith("persistent"))
        batch.close()
    form = "graph" if args.batch_graph else "persistent"
    print(json.dumps({f"batched_{form}_default_schedule": {"jobs": 256, "groups": groups,
                                                   "ms_per_batch": ms,
                                                   "jobs_per_s": 256 / (ms / 1e3)}}))


def run_priors_features(binding, ctx, ds, d: int, prec: str, reps: int = 3) -> dict:
    """The same job with an order prior q_i(|S|) and per-family weights
    (Eq. 4, 7, 12; seeded normal log values, a quarter of the weights zero,
    the empty parent set kept), and one edge feature (the edge whose
    posterior is closest to 1/2) through the single-feature DP (Eqs. 5-9: steps 1-3 twice), both on the job's
    precision.  Device time of the prior run from the library's CUDA events;
    the feature call blocks, so it is timed on the host."""
    import math

    n = ds.n
    K = binding.bn_num_families(n, d)
    rng = np.random.default_rng(77)
    log_q = rng.normal(0.0, 1.5, size=(n, n))
    log_w = rng.normal(0.0, 1.0, size=(n, K))
    log_w[rng.random((n, K)) < 0.25] = -math.inf
    log_w[:, 0] = 0.0
    job = binding.Job(ds.data, ds.arity, d, precision=prec, log_q=log_q, log_w=log_w)
    binding.bn_edge_posteriors(ctx.h, job)
    ms = []
    for _ in range(reps):
        binding.bn_edge_posteriors(ctx.h, job)
        ms.append(ctx.stats()["ms_total"])
    masks, _ = binding.bn_scores(ctx.h, binding.Job(ds.data, ds.arity, d))
    plain = binding.Job(ds.data, ds.arity, d, precision=prec)
    post, _ = binding.bn_edge_posteriors(ctx.h, plain)
    # the edge u -> v whose posterior is closest to 1/2, so that agreement
    # between the two algorithms is not trivial
    dist = np.abs(post - 0.5)
    np.fill_diagonal(dist, np.inf)
    u, v = (int(x) for x in np.unravel_index(int(np.argmin(dist)), dist.shape))
    log_f = np.zeros((n, K))
    log_f[v] = np.where((masks[v] >> u) & 1, 0.0, -math.inf)
    p, _ = binding.bn_feature_posterior(ctx.h, plain, log_f)
    t0 = time.perf_counter()
    for _ in range(reps):
        p, _ = binding.bn_feature_posterior(ctx.h, plain, log_f)
    feat_ms = (time.perf_counter() - t0) / reps * 1e3
    cells = n * 2 ** n
    return {"edge_posteriors_with_prior_and_weights": {
                "ms": statistics.median(ms), "cells_per_s": cells / (statistics.median(ms) / 1e3)},
            "feature_posterior_edge": {
                "edge": f"{u}->{v}", "ms_host": feat_ms, "p": p,
                "all_edges_path_p": float(post[u, v]),
                "abs_diff_vs_edge_path": abs(p - float(post[u, v]))}}


# ---------------------------------------------------------------- sweep --
def run_sweep(args) -> None:
    """Time the FP32 path over the configurations of the paper's experiments
    (Section 4.2, Tables 1-2: d in {2, 4, 6, 8} at n = 25; n = 21..31 at
    d = 4; binary data, m = 500, one seeded random DAG per configuration).
    Each result is checked for 0 <= P <= 1, sum_u P(u->v) <= d and
    P(u->v) + P(v->u) <= 1; up to n = 26 also against the FP64 path."""
    import torch

    from paper_1408_1664_gb300 import binding

    binding.load(build_if_missing=True)
    grid = [(25, d) for d in (2, 4, 6, 8)] + [(n, 4) for n in range(21, 32)]
    rows = []
    with binding.Context(0) as ctx:
        for n, d in grid:
            ds = datagen.random_dag_data(n, 500, 2, min(d, 4), 1.0, seed=500 + 10 * n + d)
            job = binding.Job(ds.data, ds.arity, d, precision="fp32")
            binding.bn_edge_posteriors(ctx.h, job)                       # warm-up
            reps = 3 if n <= 28 else 1
            ts, post, st = [], None, None
            for _ in range(reps):
                post, _ = binding.bn_edge_posteriors(ctx.h, job)
                st = ctx.stats()
                ts.append(st["ms_total"])
            ms = statistics.median(ts)
            eps = 1e-6
            ok = bool(np.all(post >= -eps) and np.all(post <= 1 + eps)
                      and np.all(post.sum(axis=0) <= d + 1e-4)
                      and np.all(post + post.T <= 1 + 1e-4))
            row = {"n": n, "d": d, "m": 500, "ms": ms, "cells_per_s": n * 2 ** n / (ms / 1e3),
                   "properties_ok": ok,
                   "stages_ms": {k: round(st[k], 3) for k in ("ms_scores", "ms_upzeta",
                                                              "ms_upzeta_sums", "ms_forward",
                                                              "ms_backward", "ms_gamma_p1",
                                                              "ms_gamma_p2", "ms_edges")}}
            if n <= 26:
                p64, _ = binding.bn_edge_posteriors(ctx.h, binding.Job(ds.data, ds.arity, d,
                                                                       precision="fp64"))
                row["max_abs_fp32_vs_fp64"] = float(np.abs(post - p64).max())
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
            torch.cuda.empty_cache()
    print(json.dumps({"sweep": "n and d of Section 4.2 (FP32 path, binary, m=500)",
                      "rows": rows}))


# ---------------------------------------------------------------- ours --
def run_ours(args):
    import torch

    from paper_1408_1664_gb300 import binding

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    binding.load(build_if_missing=True)
    name, fn = WORKLOADS[args.workload]
    ds, d = fn()
    if args.subset_n:
        ds = datagen.Dataset(np.ascontiguousarray(ds.data[:, :args.subset_n]),
                             ds.arity[:args.subset_n].copy(), [], ds.seed)
        name = f"{name}_first{args.subset_n}"
    if args.degree:
        d = args.degree
        name = f"{name}_d{d}"
    n = ds.n
    cells = n * 2 ** n
    prec = args.precision
    es = 4 if prec == "fp32" else 8
    ctx = binding.Context(local)
    # a dedicated stream: the library runs on the stream it is given, and the
    # CUDA events below are recorded on the same one
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    data_dev = torch.from_numpy(ds.data).cuda()
    post_dev = torch.empty((n, n), dtype=torch.float64, device="cuda")
    lpd_dev = torch.empty(1, dtype=torch.float64, device="cuda")
    job = binding.Job(data_dev, ds.arity, d, precision=prec, m=ds.m)

    def step():
        binding.bn_edge_posteriors_async(ctx.h, job, post_dev, lpd_dev, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    try:
        props = torch.cuda.get_device_properties(local)
        gpu_id = "GPU-" + str(props.uuid) if getattr(props, "uuid", None) else None
    except Exception:
        gpu_id = None
    sampler = ClockSampler(gpu_id)
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    t_ms = e0.elapsed_time(e1)
    hist = binding.bn_stats_history(ctx.h, min(args.steps, 32))
    t_s, value = replica_value(t_ms / 1e3, args.steps * cells, dist, "cuda")
    t_ms = t_s * 1e3
    post = post_dev.cpu().numpy()

    # roofline of the dominant kernel, from the per-kernel CUDA events of the
    # timed steps
    peak, peak_kind = measured_peaks()
    tab = stage_table(n, d, es)
    launches_per_step = hist[-1]["kernels"] if hist else None
    per_stage = {}
    for k, row in tab.items():
        ms = statistics.mean(row["ms"](h) for h in hist)
        per_stage[k] = {"ms_per_step": ms, "launches_per_step": row["launches"],
                        "alg_bytes_per_launch": row["bytes"],
                        "alg_gbs": row["bytes"] * row["launches"] / (ms / 1e3) / 1e9,
                        "gbs_with_intermediates": (row["bytes_with_intermediates"]
                                                   * row["launches"] / (ms / 1e3) / 1e9)}
    other = {f: statistics.mean(h[f] for h in hist) for f in ("ms_scores", "ms_gamma_p2",
                                                              "ms_edges", "ms_total")}
    # F and R' run beside each other: for the choice of the dominant kernel
    # each counts half of their common wall time (the launch list under ncu,
    # which serialises them, gives the same order)
    pair = ("k_forward_rows", "k_backward_rows", "k_forward_level", "k_backward_level")
    dom = max(tab, key=lambda k: per_stage[k]["ms_per_step"] / (2 if k in pair else 1))
    row = tab[dom]
    avg_launch_s = per_stage[dom]["ms_per_step"] / row["launches"] / 1e3
    achieved = row["bytes"] / avg_launch_s / 1e9
    traffic = committed_traffic(dom, name, prec)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "alg_bytes_per_launch": row["bytes"],
                "avg_launch_ms": avg_launch_s * 1e3,
                "achieved_with_intermediates": (row["bytes_with_intermediates"] / avg_launch_s
                                                / 1e9)}
    job_alg_bytes = hist[-1]["alg_bytes"] if hist else None
    whole = {"alg_bytes_per_step": job_alg_bytes,
             "alg_gbs": job_alg_bytes / (t_ms / args.steps / 1e3) / 1e9 if job_alg_bytes else None}
    whole["frac_of_peak"] = whole["alg_gbs"] / peak if whole["alg_gbs"] else None

    # end to end through the public host API: pinned host data in, host
    # posteriors out, every step
    pinned = torch.from_numpy(ds.data).pin_memory()
    host_data = pinned.numpy()
    post_host = np.zeros((n, n))
    job_h = binding.Job(host_data, ds.arity, d, precision=prec)
    if not args.no_e2e:
        binding.bn_edge_posteriors(ctx.h, job_h, post_host)
    e2e = None
    if not args.no_e2e:
        e2e_steps = max(3, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            binding.bn_edge_posteriors(ctx.h, job_h, post_host)
        e2e_s, e2e_value = replica_value(time.perf_counter() - t0, e2e_steps * cells, dist, "cuda")
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": int(ds.m * n + n),
               "d2h_bytes_per_step": int(n * n * 8 + 8),
               "ms_per_step": e2e_s / e2e_steps * 1e3}

    extra = {}
    post64_host = None
    if not args.no_fp64_extra and prec == "fp32" and rank == 0:
        job64 = binding.Job(data_dev, ds.arity, d, precision="fp64", m=ds.m)
        post64 = torch.empty((n, n), dtype=torch.float64, device="cuda")
        binding.bn_edge_posteriors_async(ctx.h, job64, post64, None, stream)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        k64 = 2
        f0.record(stream)
        for _ in range(k64):
            binding.bn_edge_posteriors_async(ctx.h, job64, post64, None, stream)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / k64
        h64 = binding.bn_stats_history(ctx.h, k64)
        bytes64 = h64[-1]["alg_bytes"]
        post64_host = post64.cpu().numpy()
        err = float(np.abs(post - post64_host).max())
        torch.cuda.synchronize()
        peaks = probe_peaks()
        p64 = peaks.get("fp64_fma_flops")
        extra["fp64_path"] = {
            "measured_rates": peaks,
            "fp64_flops_per_cell_in_job_time_at_fma_peak": (p64 * ms64 / 1e3 / cells
                                                             if p64 else None),
            "value": cells / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
            "alg_gbs": bytes64 / (ms64 / 1e3) / 1e9, "frac_of_hbm_peak": bytes64 / (ms64 / 1e3) / 1e9 / peak,
            "stages_ms": {k: h64[-1][k] for k in ("ms_scores", "ms_upzeta", "ms_forward",
                                                  "ms_backward", "ms_gamma_p1", "ms_gamma_p2",
                                                  "ms_edges")},
            "max_abs_diff_vs_fp32": err}
        # the FP64 path is bound by the FP64 pipe: its operations per cell
        # (ncu count) at the pipe's measured rate (a DFMA, a DADD and a DMUL
        # each take one slot; the FMA probe counts 2 flops per slot)
        opc = committed_fp64_ops()
        if opc and p64:
            achieved = opc * cells / (ms64 / 1e3)
            extra["fp64_path"]["roofline"] = {
                "bound": "alu", "pipe": "fp64", "ops_per_cell": opc,
                "achieved": achieved, "peak": p64 / 2, "unit": "FP64 thread-ops/s",
                "frac": achieved / (p64 / 2), "peak_kind": "measured (bn_peak_fp64_fma)"}

    if rank == 0 and not args.no_serve:
        extra["serving"] = run_serving(binding, local, args.serve_seconds)
        extra["batched"] = run_batched(binding, torch, local)
        extra["priors_and_features"] = run_priors_features(binding, ctx, ds, d, prec)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as orc

        orc.build()
        gpu_posts = {prec: post}
        if post64_host is not None:
            gpu_posts["fp64"] = post64_host
        cpu = oracle_full_run(ds, d, gpu_posts)
        if cpu is None:                        # not enough host memory for the whole job
            rate, n_s, dt, cores = oracle_sample(ds, d, budget_s=25.0)
            cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": (f"oracle skipped: RAM for the whole job; one oracle run on the "
                              f"first {n_s} of the {n} variables of the same data (d={d}, "
                              f"m={ds.m}): {n_s * 2 ** n_s} cells in {dt:.2f} s")}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": name, "n": n, "d": d, "m": ds.m, "arity": int(ds.arity[0]),
                       "precision": prec, "cells_per_job": cells,
                       "parallelism": f"replicas{world}",
                       "l2": "no flush: each step streams a >4 GB DP working set (L2 129 MB)"},
            "roofline": roofline, "whole_job_hbm": whole,
            "stages": per_stage, "stages_other_ms": other,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches_per_step * args.steps) if launches_per_step else None,
            "clocks": clocks, "kernel_src_sha": kernel_source_sha(),
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def run_shard(args):
    """One job of the workload split over all ranks (shard.run_rank: an
    all-gather of each exchange step's levels, an all-reduce of the
    posteriors).  A step is one whole job; the value is its cells over the
    maximum time over ranks (strong scaling: the work per step is fixed).
    Rank 0 checks the split job against the job run whole on its GPU."""
    import torch

    from paper_1408_1664_gb300 import binding
    from paper_1408_1664_gb300 import shard as sh

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    binding.load(build_if_missing=True)
    name, fn = WORKLOADS[args.workload]
    ds, d = fn()
    n = ds.n
    cells = n * 2 ** n
    ctx = binding.Context(local)
    # a dedicated stream (torch's default stream has handle 0, which the
    # library reads as its context's stream): the shard calls, the
    # collectives and the CUDA events below all run on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    job = binding.Job(ds.data, ds.arity, d, precision=args.precision)
    shard = binding.Shard(ctx.h, job, rank, world, divide_a=args.divide_a)
    shard_bytes = shard.bytes()
    nb = sh.max_step_bytes(shard)
    xbytes = sum(sum(sh.step_bytes(shard, hf, hr)) for hf, hr in sh.steps(shard.levels))
    buf = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    gathered = torch.zeros(world * nb, dtype=torch.uint8, device="cuda")
    post = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    lpd = torch.zeros(1, dtype=torch.float64, device="cuda")

    def step():
        if dist is None:
            sh.run_virtual([shard], [buf], [post], lpd, stream)
        else:
            sh.run_rank(shard, dist, buf, gathered, post, lpd, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(None)
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    local_s = e0.elapsed_time(e1) / 1e3
    if dist:
        t = torch.tensor([local_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local_s = float(t.item())
    split_post = post.cpu().numpy()
    shard.close()
    if rank == 0:
        whole, _ = ctx.edge_posteriors(ds.data, ds.arity, d, precision=args.precision)
        line = {
            "metric": METRIC, "value": args.steps * cells / local_s, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": local_s / args.steps * 1e3, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": name, "n": n, "d": d, "m": ds.m,
                       "precision": args.precision, "cells_per_job": cells,
                       "parallelism": f"shard{world}" + ("_divided_A" if args.divide_a else ""),
                       "device_bytes_per_rank": shard_bytes,
                       "packed_bytes_per_rank_per_job": xbytes,
                       "l2": "no flush: each step streams a >4 GB DP working set (L2 129 MB)"},
            "split_vs_whole_max_abs_diff": float(np.abs(split_post - whole).max()),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.shard and args.impl == "ours":
        run_shard(args)
        return
    if args.sweep:
        run_sweep(args)
    elif args.batched_only:
        run_batched_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
