#!/usr/bin/env python
"""Benchmark of the relational hot path on one GB300 (or N, as replicas).

Workload: the 60M-row star schema (fact: fk int32 Zipf(0.8) over a 2M-row
dimension, date int32, qty/price/disc int64 scaled decimals, flag/status
uint8, orderkey int64; dimension: unique scrambled int32 pk, attr int32 in
25 values) and its low-cardinality query: filter date <= 2504, join
fk = pk, group by (flag, status, attr), SUM(qty), SUM(price*(100-disc)),
COUNT(*), AVG(disc).

One step = one tp_execute of that plan: hash build of the dimension, one
fused filter/probe/aggregate pass over the fact columns, finalisation.

  value : fact rows/s with the tables resident in HBM (CUDA events on the
          engine's compute stream, max over ranks)
  e2e   : the same query through the C ABI from host pages: every step copies
          the used columns of both tables host->device inside the timed region
          and reads every result array back
  roofline : the fused kernel's algorithmic bytes per launch over its
          event-timed duration, against the measured HBM copy peak
  cpu_baseline : the CPU oracle on a bounded row sample, host cores

Prints one JSON line on rank 0.  ``--impl reference`` times the CPU oracle
instead (the only reference this project has: the paper ships no code).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fact rows/s & HBM GB/s (join+agg); served p50/p99 latency vs plain"
WORKLOAD = "star-60M-lowcard"
BYTES_PER_FACT_ROW = 4 + 4 + 8 + 8 + 8 + 1 + 1      # date, fk, qty, price, disc, flag, status
BYTES_PER_DIM_ROW = 4 + 4                            # pk, attr
# committed ncu summaries of the dominant kernel, by kernel name: the
# run-time compiled (plan-specialised) staged kernel, or the ahead-of-time one
PROFILE_SUMMARY = {"tpj_dense": os.path.join(ROOT, "profiles", "tpj_dense_star12M.md"),
                   "k_agg_shared_staged": os.path.join(ROOT, "profiles", "k_agg_shared_staged_star12M.md")}
KERNEL_SOURCES = {"tpj_dense": ("kernels.cuh", "device.cuh", "pipeline.cuh", "jit_common.cuh", "jit_dense.cuh",
                                "jit.cu", "staged.cu"),
                  "k_agg_shared_staged": ("kernels.cu", "kernels.cuh", "device.cuh", "pipeline.cuh", "staged.cu")}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="theseus", choices=["theseus", "reference"])
    ap.add_argument("--n-fact", type=int, default=60_000_000)
    ap.add_argument("--n-dim", type=int, default=2_000_000)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-sample-rows", type=int, default=20_000_000)
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary queries")
    ap.add_argument("--legs", default="config1,highcard,star,hashed",
                    help="secondary device-resident legs to run (comma list of config1, highcard, star, hashed; "
                         "highcard-hashed runs only the hashed-table leg of highcard)")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="fact-size scale of the 256-query batched and served mixes (1.0 = the full ~394M rows)")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="arrival window per served rate")
    ap.add_argument("--serve-requests", type=int, default=20_000,
                    help="requests per served rate at most (and of the closed-loop throughput run)")
    ap.add_argument("--no-patterns", action="store_true", help="skip the batched and served measurements")
    ap.add_argument("--no-outofcore", action="store_true", help="skip the out-of-core (paged, spilling) query")
    ap.add_argument("--ooc-fact", type=int, default=600_000_000, help="out-of-core fact rows")
    ap.add_argument("--ooc-dim", type=int, default=150_000_000, help="out-of-core build rows")
    ap.add_argument("--ooc-budgets", default="16,2", help="device budgets (GiB) of the out-of-core runs")
    ap.add_argument("--ooc-steps", type=int, default=2)
    ap.add_argument("--ooc-lip-budget", type=float, default=2.0,
                    help="budget (GiB) of the out-of-core runs with a dimension predicate, lookahead "
                         "filter off and on; 0 skips them")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl != "reference":
        import torch.distributed as dist
        import torch
        # one process per GPU over NCCL; gloo where no GPU is visible (the
        # host-side logic of the replicas)
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world: int, rows_per_rank: int, steps: int, ms_total: float) -> float:
    """Whole-job rows/s of replicas: every rank's rows over the slowest rank's time."""
    return world * rows_per_rank * steps / (ms_total / 1e3)


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def roofline_obj(alg_bytes: float, ms: float, peak: float, bound="hbm", peak_kind="measured", **extra):
    """Algorithmic bytes over a duration against a peak (GB/s)."""
    gbs = alg_bytes / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    d = {"bound": bound, "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak if peak else None,
         "peak_kind": peak_kind, "alg_bytes": int(alg_bytes), "ms": ms}
    d.update(extra)
    return d


def time_plan(torch, stream, eng, p, reps=5, warm=2):
    """(ms per query, the aggregate kernels' ms per query, groups, joined rows)
    of plan p: CUDA events on the engine's stream around reps executions; the
    kernel time comes from the engine's event-timed aggregate launches."""
    for _ in range(warm):
        p.execute().free()
    torch.cuda.synchronize()
    s0 = eng.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = None
    for i in range(reps):
        r = p.execute()
        if i + 1 < reps:
            r.free()
        else:
            res = r
    e1.record(stream)
    torch.cuda.synchronize()
    s1 = eng.stats()
    groups, joined = res.n_groups, int(res.counts().sum()) if res.n_groups else 0
    res.free()
    ms = e0.elapsed_time(e1) / reps
    return ms, (s1["agg_kernel_ms"] - s0["agg_kernel_ms"]) / reps, groups, joined


def kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2508_05029_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, n_rows: int):
    """DRAM bytes per launch from the committed ncu summary of `kernel`, scaled
    to n_rows, or None when the summary is missing or the kernel source
    changed since."""
    try:
        text = open(PROFILE_SUMMARY[kernel]).read()
    except OSError:
        return None
    m_src = re.search(r"source_sha\s*=\s*([0-9a-f]+)", text)
    m_b = re.search(r"dram_bytes_per_launch\s*=\s*(\d+)", text)
    m_r = re.search(r"rows_per_launch\s*=\s*(\d+)", text)
    if not (m_src and m_b and m_r) or m_src.group(1) != kernel_source_hash(kernel):
        return None
    return int(int(m_b.group(1)) * n_rows / int(m_r.group(1)))


def link_peak_gbs(dev, pinned_bytes=2 << 30, page=64 << 20):
    """Host-to-device copy peak of this machine: cudaMemcpyAsync of 64 MiB pinned
    pages (torch tensors), best of three passes."""
    import torch
    h = torch.empty(pinned_bytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(pinned_bytes, dtype=torch.uint8, device=dev)
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for off in range(0, pinned_bytes, page):
            d[off:off + page].copy_(h[off:off + page], non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, pinned_bytes / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del h, d
    return best


# ------------------------------------------------------------- CPU oracle leg
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_oracle(fact, dim, query, sample_rows):
    """The oracle as it stands, one thread, on the first sample_rows fact rows."""
    import oracle
    sub = {k: v[:sample_rows] for k, v in fact.items()}
    t0 = time.perf_counter()
    res = oracle.run_query(sub, dim, query)
    dt = time.perf_counter() - t0
    return sample_rows / dt, dt, res


def _merge_partials(parts):
    """Groups of several oracle results over disjoint row ranges, merged by
    key: counts and exact sums add; AVG is the merged sum over the merged
    count, rounded once (Python's int -> float conversion rounds correctly)."""
    acc = {}
    for r in parts:
        for g in range(r.n_groups):
            k = int(r.keys[g])
            c, sums = acc.get(k, (0, [0] * len(r.aggs)))
            acc[k] = (c + int(r.counts[g]), [sums[a] + r.sum_int(g, a) for a in range(len(r.aggs))])
    keys = sorted(acc)
    return keys, [acc[k][0] for k in keys], [acc[k][1] for k in keys]


def cpu_oracle_threads(fact, dim, query, sample_rows, threads):
    """The oracle on `threads` row ranges of the sample at once (the C calls
    release the GIL, so they run on separate cores), each with its own copy of
    the dimension lookup, and the partial groups merged by key.  Returns
    (rows/s, seconds, merged groups)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    cut = np.linspace(0, sample_rows, threads + 1).astype(np.int64)
    parts = [{k: v[cut[i]:cut[i + 1]] for k, v in fact.items()} for i in range(threads)]
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(lambda f: oracle.run_query(f, dim, query), parts))
    merged = _merge_partials(res)
    dt = time.perf_counter() - t0
    return sample_rows / dt, dt, merged


def cpu_baseline_obj(fact, dim, query, sample_rows, threads=None):
    """cpu_baseline object: the oracle on every host core (row ranges, merged)
    and on one core, both on the same bounded sample; the merged groups are
    checked against the one-core result."""
    threads = threads or host_cores()
    r1, s1, ref = cpu_oracle(fact, dim, query, sample_rows)
    rn, sn, merged = cpu_oracle_threads(fact, dim, query, sample_rows, threads)
    same = merged[0] == [int(k) for k in ref.keys] and merged[1] == [int(c) for c in ref.counts] and \
        all(merged[2][g][a] == ref.sum_int(g, a) for g in range(ref.n_groups) for a in range(len(ref.aggs)))
    return {"value": rn, "unit": "fact rows/s", "cores": threads, "kind": "oracle",
            "sample": f"first {sample_rows} fact rows with the full dimension, {threads} row ranges on "
                      f"{threads} threads merged by key ({sn:.2f} s); merge equals the one-core result: {same}",
            "single_core": {"value": r1, "unit": "fact rows/s", "cores": 1, "seconds": s1}}


def reference_arm(args, world, rank):
    """The CPU oracle as it stands on this host's cores: each step evaluates a
    bounded row sample of the same workload as row ranges on every core,
    merged by key (one core's rate is reported beside it)."""
    if rank != 0:
        return
    from datagen import workloads as W
    q = W.q_lowcard()
    threads = host_cores()
    # size each step's row sample so warm-up plus timed steps take ~2 minutes
    probe_rows = 400_000
    fact, dim = W.config2_tables(n_fact=probe_rows, n_dim=args.n_dim)
    _, secs, _ = cpu_oracle_threads(fact, dim, q, probe_rows, threads)
    per_row = secs / probe_rows
    budget_s = 120.0 / max(1, args.warmup + args.steps)
    sample = int(min(args.n_fact, max(probe_rows, budget_s / per_row)))
    fact, dim = W.config2_tables(n_fact=sample, n_dim=args.n_dim)
    rates = []
    for i in range(args.warmup + args.steps):
        r, _, _ = cpu_oracle_threads(fact, dim, q, sample, threads)
        if i >= args.warmup:
            rates.append(r)
    r1, s1, _ = cpu_oracle(fact, dim, q, min(sample, 4_000_000))
    value = statistics.mean(rates)
    t_step = sample / value
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "fact rows/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "fact_rows": args.n_fact, "dim_rows": args.n_dim,
                   "step_sample_rows": sample},
        "cpu_baseline": {"value": value, "unit": "fact rows/s", "cores": threads, "kind": "oracle",
                         "sample": f"first {sample} fact rows of the workload, full dimension, {threads} row "
                                   f"ranges on {threads} threads merged by key",
                         "single_core": {"value": r1, "unit": "fact rows/s", "cores": 1, "seconds": s1}},
        "e2e": {"value": value, "unit": "fact rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)



# ------------------------------------------------------ batched and served
def _mix_tables(eng, T, W, torch, dev, n_queries, scale, n_dims=None, fact_pages=False):
    """The batched mix: per query its own fact table (lognormal size), a
    dimension (log-uniform size) and a group count; dims shared round-robin
    when n_dims is given.  Fact tables are device-resident, or in the engine's
    pinned pages (streamed per query) with fact_pages.  Returns the tables,
    plans, fact rows and algorithmic bytes (34 B per fact row, 8 B per
    dimension row of each query)."""
    sz = W.config4_sizes(n_queries=n_queries)
    tabs, plans = [], []
    dims = {}
    rows = 0
    alg = 0
    for q in range(n_queries):
        dq = q % n_dims if n_dims else q
        wl = W.config4_query(dq, int(sz["fact"][q]), int(sz["dim"][dq]), int(sz["cutoff"][q]),
                             int(sz["groups"][dq]), fact_scale=scale)
        if n_dims and q >= n_dims:   # own fact rows, keys of the shared dimension
            own = W.config4_query(q, int(sz["fact"][q]), int(sz["dim"][dq]), int(sz["cutoff"][q]),
                                  int(sz["groups"][dq]), fact_scale=scale).fact
            own["fk"] = wl.dim["pk"][np.arange(own["fk"].size) * 7919 % wl.dim["pk"].size]
            wl = W.Workload(wl.name, own, wl.dim, wl.query)
        if dq not in dims:
            dims[dq] = eng.table_from_torch({k: torch.from_numpy(v).to(dev) for k, v in wl.dim.items()})
            tabs.append(dims[dq])
        if fact_pages:
            ft = eng.table_from_numpy(wl.fact, placement=T.TP_HOST_PAGES)
        else:
            ft = eng.table_from_torch({k: torch.from_numpy(v).to(dev) for k, v in wl.fact.items()})
        tabs.append(ft)
        rows += wl.n_fact
        alg += 34 * wl.n_fact + 8 * wl.dim["pk"].size
        plans.append(eng.plan(ft, dims[dq], wl.query))
    return tabs, plans, rows, alg


def batched_measure(T, W, torch, dev, stream, scale, peak, reps=3):
    import tempfile
    eng = T.Engine(compute_stream=stream.cuda_stream)
    tabs, plans, rows, alg = _mix_tables(eng, T, W, torch, dev, 256, scale)

    def best_of(b):
        best = 1e30
        for i in range(reps + 1):
            for r in b.execute():
                r.free()
            if i:
                best = min(best, b.last_ms)
        return best

    b = T.Batch(eng, plans)
    best_b = best_of(b)
    # the autotuner over the same plans, then the batch built from its table
    tune = {}
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "tune.txt")
        t0 = time.perf_counter()
        T.autotune(eng, plans, path)
        tune["tuning_s"] = time.perf_counter() - t0
        lines = [l.split() for l in open(path) if not l.startswith("#")]
        bt = T.Batch(eng, plans, tuning_path=path)
        tune["tuned_ms"] = best_of(bt)
        bt.destroy()
    tune["classes"] = len(lines)
    tune["changed"] = {
        "rows_per_warp": sum(1 for l in lines if int(l[2]) != 1024),
        "device_memory_agg": sum(1 for l in lines if int(l[3]) == 2),
        "load_factor_0.7": sum(1 for l in lines if float(l[1]) > 0.6)}
    tune["choices"] = {l[0]: {"load_factor": float(l[1]), "rows_per_warp": int(l[2]), "agg": int(l[3])}
                       for l in lines}
    torch.cuda.synchronize()
    best_p = 1e30
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for p in plans:
            p.execute().free()
        e1.record(stream)
        torch.cuda.synchronize()
        best_p = min(best_p, e0.elapsed_time(e1))
    b.destroy()
    for p in plans:
        p.destroy()
    for t in tabs:
        t.destroy()
    eng.close()
    gbs = alg / (best_b / 1e3) / 1e9
    gbs_t = alg / (tune["tuned_ms"] / 1e3) / 1e9
    return {"queries": 256, "fact_rows": rows, "fact_scale": scale, "batched_ms": best_b, "plain_ms": best_p,
            "speedup": best_p / best_b, "batched_rows_per_s": rows / (best_b / 1e3),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "alg_bytes": alg},
            "autotuned": dict(tune, roofline={"bound": "hbm", "achieved": gbs_t, "peak": peak, "unit": "GB/s",
                                              "frac": gbs_t / peak, "alg_bytes": alg},
                              speedup_vs_default=best_b / tune["tuned_ms"]),
            "how": "one persistent graph-captured launch vs 256 tp_execute calls on one stream"}


def host_ram_bytes() -> int:
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        return 0


def outofcore_measure(T, W, torch, dev, n_fact, n_dim, budgets_gb, steps, link, lip_budget=0.0, with_cpu=True):
    """The out-of-core star query: fact and build tables in 64 MiB pinned pages,
    streamed through the device; the join runs radix-partitioned 64 ways and
    spills the partitions the budget cannot hold.  Rows are scaled down (and
    the line says so) when host memory cannot hold the pages."""
    page = 64 << 20
    fact_b, dim_b = 38, 12                       # bytes per fact row (native widths) and build row
    ram = host_ram_bytes()
    scale = 1.0
    # the tables (each batch rounded up to whole pages) plus room to spill all
    # of them, plus one partly filled page per spilled partition and table
    need = lambda s: 2.5 * (n_fact * fact_b + n_dim * dim_b) * s + 128 * page
    while ram and need(scale) > 0.6 * ram and scale > 0.05:
        scale /= 2
    nf, nd = int(n_fact * scale), int(n_dim * scale)
    n_pages = int(need(scale) // page) + 1
    t0 = time.perf_counter()
    eng = T.Engine(page_bytes=page, n_pages=n_pages, batch_rows=6_000_000, prefetch_depth=2,
                   cuda_device=dev.index or 0)
    chunk = 25_000_000
    dt = eng.table_from_chunks(W.config3_dim(nd, row0=r, n=min(chunk, nd - r)) for r in range(0, nd, chunk))
    passing = [0]   # fact rows the filter keeps: every fk has a partner, so the total count must match

    def fact_chunks():
        for r in range(0, nf, chunk):
            c = W.config3_fact(r, min(chunk, nf - r), n_dim=nd)
            passing[0] += int((c["date"] <= W.CUTOFF_98).sum())
            yield c

    ft = eng.table_from_chunks(fact_chunks())
    setup_s = time.perf_counter() - t0
    out = {"fact_rows": nf, "dim_rows": nd, "scale": scale, "pages": n_pages, "setup_s": round(setup_s, 1),
           "host_ram_gb": round(ram / 2**30, 1), "link_peak_gbs": link}
    alg = nf * fact_b + nd * dim_b
    for b in budgets_gb:
        eng.set_budget(int(b * 2**30))
        p = eng.plan(ft, dt, W.q_lowcard(), join_partitions=64)
        p.execute().free()
        s0 = eng.stats()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        groups, total = 0, 0
        for _ in range(steps):
            with p.execute() as r:
                groups = r.n_groups
                total = int(r.counts().sum())
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t1) / steps
        s1 = eng.stats()
        h2d = (s1["h2d_bytes"] - s0["h2d_bytes"]) / steps
        d2h = (s1["d2h_bytes"] - s0["d2h_bytes"]) / steps
        out[f"budget_{b:g}GB"] = {
            "ms_per_step": sec * 1e3, "fact_rows_per_s": nf / sec, "groups": groups,
            "count_check": total == passing[0],
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "alg_gbs": alg / sec / 1e9, "link_frac_alg": alg / sec / 1e9 / link,
            "link_frac_moved": (h2d + d2h) / sec / 1e9 / link,
            "phase_ms": {k: (s1[f"part_{k}_ms"] - s0[f"part_{k}_ms"]) / steps for k in ("build", "stream", "spilled")},
            "roofline": roofline_obj(alg, sec * 1e3, link, bound="link", peak_kind="measured in this run",
                                     note="fact (38 B/row) and build (12 B/row) bytes at native width over "
                                          "the host-to-device link peak")}
        p.destroy()
    # ablations at the largest budget (every partition resident): no
    # prefetch (Section 3.3.3), and per-batch pinned buffers instead of the
    # page pool (Section 3.4)
    b = max(budgets_gb)
    eng.set_budget(int(b * 2**30))
    for name, depth, pinned in (("prefetch_0", 0, False), ("pinned_per_batch", 2, True)):
        eng.set_copy_options(depth, pinned)
        p = eng.plan(ft, dt, W.q_lowcard(), join_partitions=64)
        p.execute().free()
        s0 = eng.stats()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(steps):
            with p.execute() as r:
                total = int(r.counts().sum())
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t1) / steps
        s1 = eng.stats()
        out.setdefault("ablations", {})[name] = {
            "budget_gb": b, "ms_per_step": sec * 1e3, "count_check": total == passing[0],
            "h2d_bytes_per_step": int((s1["h2d_bytes"] - s0["h2d_bytes"]) / steps),
            "slowdown_vs_default": sec * 1e3 / out[f"budget_{b:g}GB"]["ms_per_step"]}
        p.destroy()
    eng.set_copy_options(2, False)
    out["ablations"]["managed_memory"] = ("measured on the headline query (e2e.managed_memory: fact columns in "
                                          "managed memory, demand-paged or read in place, against the page pool); "
                                          "a join table oversubscribing the GPU's memory is not created here")
    if lip_budget > 0:
        out["lookahead"] = lookahead_measure(T, W, torch, eng, ft, dt, nf, lip_budget, steps)
    ft.destroy()
    dt.destroy()
    eng.close()
    if with_cpu:
        # the oracle on the same query at 1/100 of the rows (fact and build
        # side in the same ratio), regenerated from the counter-based generator
        sf, sd = max(1, n_fact // 100), max(1, n_dim // 100)
        cb = cpu_baseline_obj(W.config3_fact(0, sf, n_dim=sd), W.config3_dim(sd), W.q_lowcard(), sf)
        cb["sample"] = f"scaled workload: {sf} fact rows over a {sd}-row build side; " + cb["sample"]
        out["cpu_baseline"] = cb
    return out


def lookahead_measure(T, W, torch, eng, ft, dt, nf, budget_gb, steps):
    """The out-of-core star query with a predicate admitting 5 of the 25
    dimension attribute values (20% of the build rows), lookahead filter off
    and on: the filter keeps fact rows that cannot join out of the probes and
    out of the partition spill.  Both runs must give the same groups."""
    eng.set_budget(int(budget_gb * 2**30))
    q = dict(W.q_lowcard(), dim_filter=dict(col="attr", lo=0, hi=4))
    out = {"budget_gb": budget_gb, "dim_filter": "attr in [0, 4]: 20% of the build rows"}
    seen = {}
    for name, mode in (("off", T.TP_LIP_OFF), ("on", T.TP_LIP_AUTO)):
        p = eng.plan(ft, dt, q, join_partitions=64, lip=mode)
        p.execute().free()
        s0 = eng.stats()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(steps):
            with p.execute() as r:
                seen[name] = (r.keys().copy(), r.counts().copy())
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t1) / steps
        s1 = eng.stats()
        out[name] = {"ms_per_step": sec * 1e3, "fact_rows_per_s": nf / sec,
                     "h2d_bytes_per_step": int((s1["h2d_bytes"] - s0["h2d_bytes"]) / steps),
                     "d2h_bytes_per_step": int((s1["d2h_bytes"] - s0["d2h_bytes"]) / steps),
                     "filters_built": int(s1["lip_filters"] - s0["lip_filters"])}
        p.destroy()
    out["speedup"] = out["off"]["ms_per_step"] / out["on"]["ms_per_step"]
    out["results_equal"] = bool(np.array_equal(seen["off"][0], seen["on"][0]) and
                                np.array_equal(seen["off"][1], seen["on"][1]))
    return out


def star_measure(T, W, torch, dev, stream, eng, fact, dt, n_fact, peak, n_xdim=32_000_000, reps=5):
    """The 60M-row star query joined to a second dimension of n_xdim rows with
    unique sparse int64 keys (a hashed table of 1 GB, far over L2), whose
    predicate admits 3 of 25 attribute values (12%); grouped by the two fact
    flags, the first dimension's attribute and the second's band.  Lookahead
    filter off and on (same groups required), and the same join without the
    predicate."""
    seed = W.SEEDS[2] + 100
    xd = W.star_dim(n_xdim, seed)
    cols = {k: torch.from_numpy(v).to(dev) for k, v in fact.items()}
    cols["fk2"] = torch.from_numpy(W.star_fk(n_fact, n_xdim, seed)).to(dev)
    ft = eng.table_from_torch(cols)
    xt = eng.table_from_torch({k: torch.from_numpy(v).to(dev) for k, v in xd.items()})
    torch.cuda.synchronize()
    xj = dict(fact_col="fk2", dim_col="pk", dim_filter=dict(col="attr", lo=0, hi=2))
    group = [("fact", "flag", 2), ("fact", "status", 1), ("dim", "attr", 5), ("dim1", "band", 2)]
    out = {"fact_rows": n_fact, "second_dim_rows": n_xdim, "second_dim_filter": "attr in [0, 2]: 12%"}
    seen = {}
    for name, lip, xjoin in (("lookahead_off", T.TP_LIP_OFF, xj), ("lookahead_on", T.TP_LIP_AUTO, xj),
                             ("no_predicate", T.TP_LIP_AUTO, dict(xj, dim_filter=None))):
        q = dict(W.q_lowcard(), extra_joins=[xjoin], group=group)
        p = eng.plan(ft, dt, q, extra_dims=[xt], lip=lip)
        for _ in range(2):
            p.execute().free()
        s0 = eng.stats()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            with p.execute() as r:
                seen[name] = (r.keys().copy(), r.counts().copy())
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        s1 = eng.stats()
        # fact: the star query's 34 B plus fk2 (8 B); first dimension 8 B per
        # row; second dimension pk, attr, band (13 B per row) for its build
        alg = n_fact * (BYTES_PER_FACT_ROW + 8) + int(dt.rows) * BYTES_PER_DIM_ROW + n_xdim * 13
        out[name] = {"ms_per_step": ms, "fact_rows_per_s": n_fact / (ms / 1e3), "groups": int(seen[name][0].size),
                     "compiled_kernel": s1["jit_launches"] > s0["jit_launches"],
                     "filters_built": int(s1["lip_filters"] - s0["lip_filters"]) // reps,
                     "roofline": roofline_obj(alg, ms, peak, note="whole query, both builds included")}
        p.destroy()
    out["lookahead_speedup"] = out["lookahead_off"]["ms_per_step"] / out["lookahead_on"]["ms_per_step"]
    out["results_equal"] = bool(np.array_equal(seen["lookahead_off"][0], seen["lookahead_on"][0]) and
                                np.array_equal(seen["lookahead_off"][1], seen["lookahead_on"][1]))
    ft.destroy()
    xt.destroy()
    return out


def _open_loop(srv, plans, rate, n, rng):
    """Poisson arrivals at `rate` for n requests; latency = scheduled arrival
    -> result on the host.  Returns (latencies ms, wall s)."""
    import threading
    import time as _t
    gaps = rng.exponential(1.0 / rate, n)
    order = rng.integers(0, len(plans), n)
    sched, tickets, lat = [], [], []

    def collect():
        for i in range(n):
            while len(tickets) <= i:
                _t.sleep(0.0001)
            res, times = srv.wait(tickets[i], timeout_s=600)
            res.free()
            lat.append((times[2] - sched[i]) / 1e6)
    th = threading.Thread(target=collect)
    th.start()
    t0 = _t.monotonic_ns()
    at = t0
    for i in range(n):
        at += int(gaps[i] * 1e9)
        while _t.monotonic_ns() < at:
            pass
        sched.append(at)
        tickets.append(srv.submit(plans[order[i]]))
    th.join()
    return lat, (_t.monotonic_ns() - t0) / 1e9


def _closed_loop(srv, plans, n, rng):
    """n requests submitted back to back (at most 512 outstanding): the
    server's maximum throughput in queries/s."""
    import time as _t
    order = rng.integers(0, len(plans), n)
    pending = []
    t0 = _t.monotonic()
    for i in range(n):
        if len(pending) >= 512:
            srv.wait(pending.pop(0), timeout_s=600)[0].free()
        pending.append(srv.submit(plans[order[i]]))
    for t in pending:
        srv.wait(t, timeout_s=600)[0].free()
    return n / (_t.monotonic() - t0)


def served_measure(T, W, torch, dev, rates, seconds, max_requests, scale, fact_pages=False, closed_n=0):
    """The served pattern against plain per-query execution on the same
    arrival traces.  served: continuous batching (every request a batched
    launch can run joins the next launch; the rest run on 8 lanes with cached
    join tables); plain: one request at a time, no cache.  Open-loop Poisson
    arrivals per rate for `seconds` or `max_requests`; then a closed loop of
    closed_n requests for the maximum throughput.  fact_pages: every request
    streams its fact table from pinned pages (lanes only)."""
    page = 16 << 20
    n_pages = 0
    if fact_pages:
        sz = W.config4_sizes(n_queries=256)
        n_pages = int(sum(int(f * scale) * 34 * 1.1 + page for f in sz["fact"]) // page) + 64
    eng = T.Engine(page_bytes=page, n_pages=n_pages, batch_rows=4 << 20)
    tabs, plans, _, _ = _mix_tables(eng, T, W, torch, dev, 256, scale, n_dims=64, fact_pages=fact_pages)
    for p in plans:     # warm: plan history, selectivity samples
        p.execute().free()
    out = {"requests_per_rate": f"min({max_requests}, {seconds:g} s x rate)"}
    for mode in ("served", "plain"):
        srv = T.Server(eng, workers=8, cache_dims=True, batch=True) if mode == "served" else \
            T.Server(eng, workers=1, max_inflight=1, cache_dims=False)
        for p in plans:   # warm: run-time compiled shapes, cached join tables
            srv.wait(srv.submit(p), timeout_s=600)[0].free()
        for t in [srv.submit(p) for p in plans]:   # and one batched launch of every shape together
            srv.wait(t, timeout_s=600)[0].free()
        rng = np.random.default_rng(0x7E5E0005)
        for rate in rates:
            st0 = srv.stats()
            n = max(8, min(max_requests, int(rate * seconds)))
            lat, wall = _open_loop(srv, plans, rate, n, rng)
            st1 = srv.stats()
            lat.sort()
            launches = st1["batches"] - st0["batches"]
            out[f"{mode}@{rate}"] = {
                "requests": n, "p50_ms": lat[len(lat) // 2], "p99_ms": lat[max(0, int(len(lat) * 0.99) - 1)],
                "qps": n / wall, "failed": st1["failed"] - st0["failed"],
                "batched_launches": launches,
                "requests_per_launch": (n / launches) if launches else None}
        if closed_n:
            out[f"{mode}@max"] = {"requests": closed_n, "qps": _closed_loop(srv, plans, closed_n, rng)}
        srv.stop()
    for p in plans:
        p.destroy()
    for t in tabs:
        t.destroy()
    eng.close()
    return out


def e2e_measure(T, W, torch, dev, stream, local, world, fact, dim, n_fact, n_dim, steps, link, flags):
    """The headline query through tp_execute from 64 MiB pinned host pages,
    every host-to-device copy and the read-back of every result array inside
    the timed region.  flags = TP_FLAG_RAW_PAGES keeps every column at full
    width in the pages (no frame-of-reference narrowing)."""
    page = 64 << 20
    need = (n_fact * (BYTES_PER_FACT_ROW + 8) + n_dim * BYTES_PER_DIM_ROW) * 1.1
    n_pages = int(need // page) + 16
    eng2 = T.Engine(page_bytes=page, n_pages=n_pages, batch_rows=4 << 20, prefetch_depth=2,
                    compute_stream=stream.cuda_stream, cuda_device=local, flags=flags)
    ft2 = eng2.table_from_numpy(fact, placement=T.TP_HOST_PAGES)
    dt2 = eng2.table_from_numpy(dim, placement=T.TP_HOST_PAGES)
    p3 = eng2.plan(ft2, dt2, W.q_lowcard())

    def e2e_step():
        with p3.execute() as r:
            r.keys(), r.counts()
            for a in range(4):
                if a != 2:
                    r.sum_words(a)
            r.avg(3)

    for _ in range(2):
        e2e_step()
    s0 = eng2.stats()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        e2e_step()
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, world)
    s1 = eng2.stats()
    h2d_gbs = (s1["h2d_bytes"] - s0["h2d_bytes"]) / t_e2e / 1e9
    out = {"value": world * n_fact * steps / t_e2e, "unit": "fact rows/s",
           "link_peak_gbs": link, "link_frac": h2d_gbs / link,
           "h2d_bytes_per_step": (s1["h2d_bytes"] - s0["h2d_bytes"]) // steps,
           "d2h_bytes_per_step": (s1["d2h_bytes"] - s0["d2h_bytes"]) // steps,
           "h2d_gbs": h2d_gbs,
           "source": "pinned page pool, 64 MiB pages, prefetch depth 2" +
                     (", full-width columns" if flags & T.TP_FLAG_RAW_PAGES else ", bit-packed frame-of-reference columns")}
    p3.destroy()
    ft2.destroy()
    dt2.destroy()
    eng2.close()
    return out


def _cudart():
    """The CUDA runtime library, for the managed-memory ablation only (the
    library under test links its own runtime statically)."""
    import ctypes
    for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so.13"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            pass
    return None


def managed_measure(T, W, torch, dev, stream, local, fact, dim, n_fact, steps, link):
    """Ablation of explicit staging against managed (UVM) memory (the paper's
    Section 5 finds the latter far slower): the headline query over fact
    columns in managed memory, (a) on the device (prefetched there first),
    (b) moved back to the host before each step (outside the timed region)
    and migrated by demand paging as the kernel reads them, (c) kept on the
    host (preferred location the host, mapped for the device) and read in
    place over the link.  Plain-load kernels throughout (TP_FLAG_NO_STAGED):
    page faults are taken by ordinary loads.  The GPU's memory is not
    oversubscribed: that would take filling a shared GPU's memory."""
    import ctypes
    rt = _cudart()
    if rt is None:
        return "unavailable: no CUDA runtime library to allocate managed memory"

    class Loc(ctypes.Structure):
        _fields_ = [("type", ctypes.c_int), ("id", ctypes.c_int)]

    rt.cudaMallocManaged.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t, ctypes.c_uint]
    rt.cudaMemPrefetchAsync.argtypes = [ctypes.c_void_p, ctypes.c_size_t, Loc, ctypes.c_uint, ctypes.c_void_p]
    rt.cudaMemAdvise.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, Loc]
    rt.cudaFree.argtypes = [ctypes.c_void_p]
    LOC_DEVICE, LOC_HOST = 1, 2
    ADVISE_PREFERRED, ADVISE_ACCESSED_BY = 3, 5

    def ok(rc, what):
        if rc != 0:
            raise RuntimeError(f"{what} returned CUDA error {rc}")

    ok(rt.cudaSetDevice(local), "cudaSetDevice")
    host, on_dev = Loc(LOC_HOST, 0), Loc(LOC_DEVICE, local)
    allocs, cols = [], {}
    eng = ft = dt = plan = None
    try:
        for name, arr in fact.items():
            p = ctypes.c_void_p()
            ok(rt.cudaMallocManaged(ctypes.byref(p), max(arr.nbytes, 16), 1), "cudaMallocManaged")
            allocs.append((p.value, arr.nbytes))
            ctypes.memmove(p.value, arr.ctypes.data, arr.nbytes)   # first touch on the host
            cols[name] = (p.value, arr.dtype)
        eng = T.Engine(compute_stream=stream.cuda_stream, flags=T.TP_FLAG_NO_STAGED, cuda_device=local)
        dt = eng.table_from_torch({k: torch.from_numpy(v).to(dev) for k, v in dim.items()})
        ft = eng.table_from_pointers(cols, n_fact)
        plan = eng.plan(ft, dt, W.q_lowcard())
        fact_bytes = BYTES_PER_FACT_ROW * n_fact   # the columns the query reads

        def move(loc):
            for a, nb in allocs:
                ok(rt.cudaMemPrefetchAsync(a, nb, loc, 0, ctypes.c_void_p(stream.cuda_stream)), "cudaMemPrefetchAsync")
            torch.cuda.synchronize()

        def run():
            with plan.execute() as r:
                return r.keys().copy(), r.counts().copy()

        def timed(before):
            times, res = [], None
            for _ in range(steps):
                before()
                t0 = time.perf_counter()
                res = run()
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            sec = statistics.median(times)
            return {"ms_per_step": sec * 1e3, "fact_rows_per_s": n_fact / sec,
                    "fact_gbs": fact_bytes / sec / 1e9}, res

        move(on_dev)
        run()
        out = {"fact_bytes_read": fact_bytes, "managed_bytes": sum(nb for _, nb in allocs),
               "kernels": "plain loads (TP_FLAG_NO_STAGED)", "link_peak_gbs": link}
        out["device_resident"], ref = timed(lambda: None)
        out["demand_paging"], res = timed(lambda: move(host))
        same = all(np.array_equal(a, b) for a, b in zip(ref, res))
        for a, nb in allocs:
            ok(rt.cudaMemAdvise(a, nb, ADVISE_PREFERRED, host), "cudaMemAdvise")
            ok(rt.cudaMemAdvise(a, nb, ADVISE_ACCESSED_BY, on_dev), "cudaMemAdvise")
        move(host)
        out["host_resident_mapped"], res = timed(lambda: None)
        same = same and all(np.array_equal(a, b) for a, b in zip(ref, res))
        out["results_match"] = bool(same)
        for k in ("demand_paging", "host_resident_mapped"):
            out[k]["link_frac"] = out[k]["fact_gbs"] / link
            out[k]["slowdown_vs_device"] = out[k]["ms_per_step"] / out["device_resident"]["ms_per_step"]
        return out
    finally:
        for h in (plan, ft, dt):
            if h is not None:
                h.destroy()
        if eng is not None:
            eng.close()
        torch.cuda.synchronize()
        for a, _ in allocs:
            rt.cudaFree(ctypes.c_void_p(a))


def config1_measure(T, W, torch, dev, stream, peak, with_cpu=True, reps=50):
    """Config 1: 1M fact rows, 10k-row dimension, device-resident, one batch.
    At 34 MB of input (about 5 us of HBM traffic) the query is bound by
    launch and synchronisation latency, not by bandwidth; the roofline
    fraction is reported all the same."""
    wl = W.config1()
    eng1 = T.Engine(compute_stream=stream.cuda_stream, flags=T.TP_FLAG_TIME_KERNELS)
    ft = eng1.table_from_torch({k: torch.from_numpy(v).to(dev) for k, v in wl.fact.items()})
    dt = eng1.table_from_torch({k: torch.from_numpy(v).to(dev) for k, v in wl.dim.items()})
    torch.cuda.synchronize()
    p = eng1.plan(ft, dt, wl.query)
    ms, kms, groups, _ = time_plan(torch, stream, eng1, p, reps=reps, warm=5)
    n = wl.n_fact
    alg = BYTES_PER_FACT_ROW * n + BYTES_PER_DIM_ROW * wl.n_dim
    out = {"fact_rows": n, "dim_rows": wl.n_dim, "groups": groups, "ms_per_step": ms,
           "fact_rows_per_s": n / (ms / 1e3), "kernel_ms": kms,
           "roofline": roofline_obj(BYTES_PER_FACT_ROW * n, kms, peak, note="latency-bound: launch and "
                                    "synchronisation dominate a 34 MB input"),
           "query_roofline": roofline_obj(alg, ms, peak)}
    if with_cpu:
        out["cpu_baseline"] = cpu_baseline_obj(wl.fact, wl.dim, wl.query, n)
    p.destroy()
    ft.destroy()
    dt.destroy()
    eng1.close()
    return out


def highcard_measure(T, W, torch, dev, stream, eng, ft, dt, fact, dim, n_fact, peak, only_hashed=False):
    """Config 2b (1%-selective date range, group by order key: about 600k
    groups), 2b' (the same at ~98%: 15M groups) with the direct-addressed
    table the dense order keys allow, and 2b' with the hashed table (sparse
    keys' general case, TP_FLAG_NO_DIRECT_AGG).  Algorithmic bytes: the filter
    column for every row, fk/orderkey/price/disc (28 B) for every passing row,
    and 32 B per output group (key, count, 128-bit sum)."""
    lo = W.config2_range_lo()
    engh = T.Engine(compute_stream=stream.cuda_stream, flags=T.TP_FLAG_TIME_KERNELS | T.TP_FLAG_NO_DIRECT_AGG)
    fth = engh.table_from_torch({k: torch.from_numpy(v).to(dev) for k, v in fact.items()})
    dth = engh.table_from_torch({k: torch.from_numpy(v).to(dev) for k, v in dim.items()})
    torch.cuda.synchronize()
    out = {}
    for name, q, e, f_t, d_t in (
            ("star-60M-highcard-1pct", W.q_highcard(lo, lo + W.RANGE_1PCT), eng, ft, dt),
            ("star-60M-highcard-98pct", W.q_highcard(0, W.CUTOFF_98), eng, ft, dt),
            ("star-60M-highcard-98pct-hashed", W.q_highcard(0, W.CUTOFF_98), engh, fth, dth)):
        if only_hashed and e is not engh:
            continue
        p = e.plan(f_t, d_t, q)
        ms, kms, groups, joined = time_plan(torch, stream, e, p, reps=5)
        alg = 4 * n_fact + 28 * joined + 32 * groups
        out[name] = {"ms_per_step": ms, "fact_rows_per_s": n_fact / (ms / 1e3), "groups": groups,
                     "passing_rows": joined, "kernel_ms": kms,
                     "table": "hashed" if e is engh else "auto (direct-addressed when the key range is dense)",
                     "roofline": roofline_obj(alg, kms, peak, note="aggregate kernels (selection and gather, "
                                              "or the staged scan) per query"),
                     "query_roofline": roofline_obj(alg, ms, peak)}
        p.destroy()
    fth.destroy()
    dth.destroy()
    engh.close()
    return out


def hashed_join_measure(T, W, torch, dev, stream, n_fact, n_dim, peak, reps=10):
    """Config 2a with unique sparse int64 dimension keys: the join needs the
    open-addressing table (2M keys at load factor 0.5: 4M 16-byte slots) and
    the foreign key is int64, so 38 B per fact row and 12 B per dimension
    row."""
    fact, dim = W.config2_tables(n_fact=n_fact, n_dim=n_dim, sparse_keys=True)
    fact.pop("okey")
    e = T.Engine(compute_stream=stream.cuda_stream, flags=T.TP_FLAG_TIME_KERNELS)
    ft = e.table_from_torch({k: torch.from_numpy(v).to(dev) for k, v in fact.items()})
    dt = e.table_from_torch({k: torch.from_numpy(v).to(dev) for k, v in dim.items()})
    torch.cuda.synchronize()
    p = e.plan(ft, dt, W.q_lowcard())
    s0 = e.stats()
    ms, kms, groups, _ = time_plan(torch, stream, e, p, reps=reps, warm=3)
    s1 = e.stats()
    per_row = BYTES_PER_FACT_ROW + 4
    out = {"fact_rows": n_fact, "dim_rows": n_dim, "groups": groups, "ms_per_step": ms,
           "fact_rows_per_s": n_fact / (ms / 1e3), "kernel_ms": kms,
           "compiled_kernel": s1["jit_launches"] > s0["jit_launches"],
           "roofline": roofline_obj(per_row * n_fact, kms, peak, note="fused filter/probe/aggregate kernel"),
           "query_roofline": roofline_obj(per_row * n_fact + 12 * n_dim, ms, peak)}
    p.destroy()
    ft.destroy()
    dt.destroy()
    e.close()
    return out


# ------------------------------------------------------------------ GPU arm
def main():
    args = parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    import torch
    from datagen import workloads as W
    from paper_2508_05029_gb300 import build
    from paper_2508_05029_gb300 import theseus as T

    if rank == 0 or not build.up_to_date():
        if local == 0:
            build.build()
    barrier(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n_fact, n_dim = args.n_fact, args.n_dim
    # weak scaling: every rank runs its own replica of the workload (own seed)
    fact, dim = W.config2_tables(n_fact=n_fact, n_dim=n_dim, seed=W.SEEDS[2] + rank)
    stream = torch.cuda.Stream(device=dev)
    eng = T.Engine(compute_stream=stream.cuda_stream, flags=T.TP_FLAG_TIME_KERNELS, cuda_device=local)
    ft = eng.table_from_torch({k: torch.from_numpy(v).to(dev) for k, v in fact.items()})
    dt = eng.table_from_torch({k: torch.from_numpy(v).to(dev) for k, v in dim.items()})
    torch.cuda.synchronize()
    plan = eng.plan(ft, dt, W.q_lowcard())

    def step():
        plan.execute().free()

    for _ in range(max(3, args.warmup)):
        step()
    st0 = eng.stats()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    st1 = eng.stats()
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world)
    ms_step = ms_total / args.steps
    value = weak_value(world, n_fact, args.steps, ms_total)
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    k_ms = (st1["agg_kernel_ms"] - st0["agg_kernel_ms"]) / max(1, st1["agg_kernel_launches"] - st0["agg_kernel_launches"])
    peak, peak_kind = measured_peaks()
    alg_bytes = BYTES_PER_FACT_ROW * n_fact
    achieved = alg_bytes / (k_ms / 1e3) / 1e9
    step_gbs = (alg_bytes + BYTES_PER_DIM_ROW * n_dim) / (ms_step / 1e3) / 1e9

    extra = {}
    if not args.no_extra:
        legs = set(args.legs.split(","))
        if "config1" in legs:
            extra["star-1M-lowcard"] = config1_measure(T, W, torch, dev, stream, peak, args.cpu_sample_rows > 0)
        if "highcard" in legs or "highcard-hashed" in legs:
            extra.update(highcard_measure(T, W, torch, dev, stream, eng, ft, dt, fact, dim, n_fact, peak,
                                          only_hashed="highcard" not in legs))
        if "star" in legs:
            extra["star-60M-two-dims"] = star_measure(T, W, torch, dev, stream, eng, fact, dt, n_fact, peak)
        if "hashed" in legs:
            extra["star-60M-lowcard-hashed"] = hashed_join_measure(T, W, torch, dev, stream, n_fact, n_dim, peak)
    plan.destroy()
    ft.destroy()
    dt.destroy()
    eng.close()
    del ft, dt

    # ---- end to end: host pages -> device -> result arrays on the host
    e2e = None
    if args.e2e_steps > 0:
        link = link_peak_gbs(dev)
        e2e = e2e_measure(T, W, torch, dev, stream, local, world, fact, dim, n_fact, n_dim, args.e2e_steps, link, 0)
        raw = e2e_measure(T, W, torch, dev, stream, local, world, fact, dim, n_fact, n_dim, args.e2e_steps, link,
                          T.TP_FLAG_RAW_PAGES)
        e2e["raw_pages"] = {k: raw[k] for k in ("value", "unit", "link_frac", "h2d_bytes_per_step", "h2d_gbs")}
        if rank == 0 and world == 1:
            e2e["managed_memory"] = managed_measure(T, W, torch, dev, stream, local, fact, dim, n_fact, 3, link)

    if not args.no_outofcore and rank == 0:
        link_ooc = e2e["link_peak_gbs"] if e2e else link_peak_gbs(dev)
        extra["star-600M-outofcore"] = outofcore_measure(
            T, W, torch, dev, args.ooc_fact, args.ooc_dim, [float(x) for x in args.ooc_budgets.split(",")],
            args.ooc_steps, link_ooc, args.ooc_lip_budget)

    patterns = None
    if not args.no_patterns:
        peak_hbm, _ = measured_peaks()
        patterns = {"batched": batched_measure(T, W, torch, dev, stream, args.batch_scale, peak_hbm),
                    "served": served_measure(T, W, torch, dev, (200, 500, 1000, 2000, 5000), args.serve_seconds,
                                             args.serve_requests, args.batch_scale, closed_n=args.serve_requests),
                    "served_streamed": served_measure(T, W, torch, dev, (200, 1000, 2000),
                                                      args.serve_seconds, args.serve_requests // 4,
                                                      args.batch_scale, fact_pages=True)}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_sample_rows > 0:
        cpu = cpu_baseline_obj(fact, dim, W.q_lowcard(), min(args.cpu_sample_rows, n_fact))

    if rank == 0:
        kernel = "tpj_dense" if st1["jit_launches"] > st0["jit_launches"] else "k_agg_shared_staged"
        traffic = profiled_traffic(kernel, n_fact)
        line = {
            "metric": METRIC, "value": value, "unit": "fact rows/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "fact_rows": n_fact, "dim_rows": n_dim, "zipf_s": 0.8,
                       "groups": 150, "parallelism": f"replicas{world}",
                       "l2": "inputs (2.3 GB) larger than L2 (129 MB); no flush"},
            "hbm_gbs": step_gbs,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": kernel, "kernel_ms": k_ms,
                         "alg_bytes_per_launch": alg_bytes},
            "e2e": e2e, "gpu_launches": launches, "clocks": clk, "cpu_baseline": cpu, "extra": extra,
            "patterns": patterns,
        }
        print(json.dumps(line), flush=True)
    barrier(world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
