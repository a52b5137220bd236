#!/usr/bin/env python
"""Isochrone query throughput on one or more GB300s.

One step = one batch of k isochrone queries through the whole hot path
(upward CH search, persistent level sweep, isochrone-edge emission, per-query
sort) on the synthetic 4,243 x 4,243 road-like grid (18,003,049 vertices).
Default workload: 64 sources per sweep with limits drawn uniformly from
[3,600, 72,000], CUDA-graph replay.  Prints one JSON line (rank 0).

  python bench.py [--gpus N --steps K --warmup W] [--workload NAME] [--impl ours|reference]

With N > 1 (torchrun) every rank holds a replica of the graph and answers its
own batches; value = queries answered by all ranks / slowest rank's time.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # 18M-vertex graph, 64 sources per sweep, uneven limits
    "grid18m_k64": dict(graph="grid18m", k=64, tau=("uniform", 3600, 72000)),
    # 18M-vertex graph, 16 sources per sweep, shared limit
    "grid18m_k16": dict(graph="grid18m", k=16, tau=("fixed", 36000)),
    # 18M-vertex graph, one source per launch
    "grid18m_k1": dict(graph="grid18m", k=1, tau=("uniform", 3600, 72000)),
    # 18M-vertex graph, one source per launch, limit 3,600 (a small range: restricted sweeps)
    "grid18m_k1_tau3600": dict(graph="grid18m", k=1, tau=("fixed", 3600)),
    # 18M-vertex graph, uneven limits, queries per sweep chosen by the autotuner among 16, 32, 64
    "grid18m_kauto": dict(graph="grid18m", k=64, lanes=(16, 32, 64), tau=("uniform", 3600, 72000)),
    "grid4m_k64": dict(graph="grid4m", k=64, tau=("uniform", 3600, 72000)),
    "grid4m_k16": dict(graph="grid4m", k=16, tau=("fixed", 36000)),
    "grid1k_k1": dict(graph="grid1k", k=1, tau=("choice", (2000, 10000, 50000))),
    # 64 x 64 grid (4,096 vertices), one query with limit 1,500
    "grid64_k1": dict(graph="grid64", k=1, tau=("fixed", 1500)),
    "grid1k_k16": dict(graph="grid1k", k=16, tau=("choice", (2000, 10000, 50000))),
    "grid1k_k64": dict(graph="grid1k", k=64, tau=("uniform", 2000, 50000)),
}
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one sweep launch
# from one ncu capture per workload, with the hash of the sweep's sources and
# the sweep options that capture ran; reported as the roofline's traffic only
# while both match the run (else null).
SWEEP_TRAFFIC = {
    # k_sweep_tma<64, 8> on the 18M graph, one launch (ncu, --clock-control none, one pass):
    # 14,094,586,368 bytes read + 3,376,537,088 written
    "grid18m_k64": ("b2ee130f3957ab02", {"core_vertices": 20000}, 17471123456),
}
SWEEP_SOURCES = ("k_sweep_tma.cu", "iso_device.cuh", "schedule.cpp")
# sweep options that change the kernel's memory traffic, with their defaults
# (0 = the library's automatic choice)
TRAFFIC_OPTS = ("threads_per_vertex", "schedule_delay", "chunk_span", "solo_width", "fuse_width", "ctas_per_sm",
                "sweep_kernel", "core_vertices", "restrict_sweep", "fused_emission")


def lanes_class(k):
    """Lanes of the sweep that serves k queries (the library rounds k up to 1, 4, 8, 16, 32 or 64)."""
    for K in (1, 4, 8, 16, 32, 64):
        if k <= K:
            return K
    return 64


def max_over_ranks(x, dist=None, device="cpu"):
    """Largest x over all ranks (the job's time is its slowest rank's); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def first_on_rank0(fn, dist=None, rank=0):
    """Run fn() on rank 0 first and on the other ranks after it: an expensive
    step whose result rank 0 leaves in a shared cache (the contraction
    hierarchy) is then done once per node instead of once per rank."""
    if dist is None:
        return fn()
    if rank == 0:
        out = fn()
        dist.barrier()
        return out
    dist.barrier()
    return fn()


def job_throughput(world, queries_per_step, steps, seconds):
    """Whole-job queries/s: every rank answers its own queries (replicas, weak scaling)."""
    return world * queries_per_step * steps / seconds


def sweep_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1512_09090_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_key(opts):
    """The options of a run that decide the sweep's traffic (absent = 0 = automatic)."""
    return {k: int(opts.get(k, 0)) for k in TRAFFIC_OPTS}


def sweep_traffic(workload, opts):
    """DRAM bytes of one sweep launch from the recorded ncu capture, or None
    unless that capture ran the same sweep sources with the same options."""
    rec = SWEEP_TRAFFIC.get(workload)
    if not rec or rec[0] != sweep_source_hash() or traffic_key(rec[1]) != traffic_key(opts):
        return None
    return rec[2]


METRIC = "isochrone queries/s on 18M-vertex graph (1 GB300); sweep HBM GB/s vs peak; p99 ms"
CACHE = os.path.join(ROOT, "paper_1512_09090_gb300", "_cache")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def draw_taus(spec, k, seed):
    from paper_1512_09090_gb300 import synth
    kind = spec[0]
    if kind == "fixed":
        return np.full(k, spec[1], np.int32)
    if kind == "uniform":
        return synth.draw_taus_uniform(k, spec[1], spec[2], seed)
    rng = np.random.default_rng(seed)
    return np.asarray(spec[1], np.int32)[rng.integers(0, len(spec[1]), size=k)]


def load_graph_and_ch(name):
    """Generate the graph and build (or load a cached) contraction hierarchy."""
    from paper_1512_09090_gb300 import chcache
    return chcache.workload_graph_and_ch(name, log=log)


def sweep_bytes_scope(A, k):
    """Algorithmic bytes of one sweep of k lanes as the measurement scope counts
    them: B = 4(n+1) offsets + 8 m_down arcs + 4kn label writes + 4kn label
    reads + 4(L+1) level table."""
    n = A["perm"].shape[0]
    m_down = int(A["down_src"].shape[0])
    levels = int(A["level_off"].shape[0])  # L + 1
    return dict(offsets=4 * (n + 1), arcs=8 * m_down, d_write=4 * k * n, d_read=4 * k * n, levels=4 * levels)


def sweep_bytes(A, k, write_all=False):
    """Algorithmic bytes of this design's sweep of k lanes (a tighter count than
    sweep_bytes_scope): the CSR offsets and every downward arc once, every
    stored label row written once (the lowest level's rows are not stored),
    every row that is the source of a downward arc read once, the in-range
    masks written, the upward-label flags read and the level table."""
    n = A["perm"].shape[0]
    lo = A["level_off"]
    n_low = int(lo[-1] - lo[-2])                 # lowest level: rows not stored
    n_hi = n if write_all else n - n_low
    n_src = int(np.unique(A["down_src"]).shape[0])  # rows read at least once
    m_down = int(A["down_src"].shape[0])
    mask_b = 1 if k <= 8 else k // 8
    return dict(offsets=4 * (n + 1), arcs=8 * m_down, d_write=4 * k * n_hi, d_read=4 * k * n_src,
                mask_write=mask_b * n, upflag_read=n, levels=4 * (lo.shape[0]))


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"iso_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(g, spec, k_hint, budget_s=15.0):
    """The CPU oracle (Dijkstra stopped at tau + full arc scan) on a bounded
    sample of the same workload, all host cores."""
    import oracle
    from paper_1512_09090_gb300 import synth
    cores = os.cpu_count() or 1
    srcs = synth.draw_sources(g, 1, 9001)
    taus = draw_taus(spec["tau"], 1, 9002)
    t0 = time.perf_counter()
    oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs, taus, threads=1)
    t1 = max(time.perf_counter() - t0, 1e-3)
    q = int(max(cores, min(4 * cores * max(1, int(budget_s / (t1 * 2))), 4096)))
    q = max(cores, min(q, int(cores * budget_s / t1)))
    srcs = synth.draw_sources(g, q, 9003)
    taus = draw_taus(spec["tau"], q, 9004)
    t0 = time.perf_counter()
    oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs, taus, threads=cores)
    el = time.perf_counter() - t0
    return {"value": q / el, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"{q} queries of the same workload (one-query latency {t1 * 1e3:.0f} ms single-threaded), "
                      f"{el:.1f}s wall"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def run_reference(args, spec, budget_s=150.0):
    """The oracle as the reference arm: same workload, metric and unit, on host
    cores (one query per core per step, OpenMP over queries).  One oracle query
    on the 18M graph takes seconds, so the run is bounded: it times as many of
    the requested steps as fit in budget_s (at least one), after at most one
    warm-up step, and reports the steps it timed."""
    from paper_1512_09090_gb300 import synth
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    g = synth.workload_graph(spec["graph"])
    cores = os.cpu_count() or 1
    oracle.build()
    per_step = max(1, min(spec["k"], cores))
    warm = min(args.warmup, 1)
    t_step = None
    for w in range(warm):
        s = synth.draw_sources(g, per_step, 500 + w)
        t0 = time.perf_counter()
        oracle.query_batch(g.n, g.tail, g.head, g.weight, s, draw_taus(spec["tau"], per_step, 600 + w), threads=cores)
        t_step = time.perf_counter() - t0
    steps = args.steps if t_step is None else max(1, min(args.steps, int(budget_s / max(t_step, 1e-3))))
    times = []
    for i in range(steps):
        s = synth.draw_sources(g, per_step, 700 + i)
        t = draw_taus(spec["tau"], per_step, 800 + i)
        t0 = time.perf_counter()
        oracle.query_batch(g.n, g.tail, g.head, g.weight, s, t, threads=cores)
        times.append(time.perf_counter() - t0)
        if t_step is None and sum(times) > budget_s:
            break
    steps = len(times)
    total = sum(times)
    value = per_step * steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * total / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": args.workload, "graph": spec["graph"], "n": g.n, "m": int(g.tail.shape[0]),
                       "queries_per_sweep": spec["k"], "tau": list(spec["tau"]), "parallelism": "host cores",
                       "queries_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} queries per step x {steps} steps "
                                       f"({args.steps} requested; capped at {budget_s:.0f} s of timed work)"},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="grid18m_k64", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tpv", type=int, default=0)
    ap.add_argument("--fuse", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--sweep-kernel", type=int, default=0)
    ap.add_argument("--delay", type=int, default=0, help="schedule delay (TMA sweep)")
    ap.add_argument("--solo", type=int, default=0, help="top levels swept by CTA 0 alone: size limit (-1 = none)")
    ap.add_argument("--span", type=int, default=0, help="largest BFS-rank span of a sweep chunk (0 = no limit)")
    ap.add_argument("--core", type=int, default=0, help="vertices of the per-lane core (0 = automatic, -1 = none)")
    ap.add_argument("--landmarks", type=int, default=8, help="landmarks for restricted sweeps (0 = none)")
    ap.add_argument("--restrict", type=int, default=-1, help="restricted sweep: 1 on, 0 off, -1 autotuned")
    ap.add_argument("--fused", type=int, default=-1, help="fused emission: 1 on, 0 off, -1 autotuned")
    ap.add_argument("--pipeline", type=int, default=2, help="batches in flight (workspaces, one stream each)")
    ap.add_argument("--no-chain", dest="chain", action="store_false",
                    help="let batches in flight contend freely instead of starting each after the previous sweep")
    ap.add_argument("--trace", action="store_true", help="print per-step sweep times to stderr")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=5000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    spec = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, spec)

    import torch
    import paper_1512_09090_gb300 as P
    from paper_1512_09090_gb300 import _build, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    first_on_rank0(_build.build, dist, local)   # in-tree library: one writer
    g, ch = first_on_rank0(lambda: load_graph_and_ch(spec["graph"]), dist, local)
    A = ch.arrays()
    dg = P.iso_upload_graph(ch)
    if args.landmarks:
        t_lm = time.perf_counter()
        dg.add_landmarks(ch, args.landmarks)   # lower bounds for restricted sweeps
        log(f"[bench] {args.landmarks} landmarks in {time.perf_counter() - t_lm:.1f}s")
    k = spec["k"]
    opts = dict(use_cuda_graph=1)
    tuned = None
    if not args.no_autotune and not (args.tpv or args.delay or args.sweep_kernel):
        from paper_1512_09090_gb300 import autotune
        # the configurations fix the queries per sweep (k) except where the
        # workload lists lane choices; every other axis is tuned
        lanes_choices = tuple(spec.get("lanes", (k,)))
        ts = synth.draw_sources(g, 8 * max(lanes_choices), 777)
        tt = draw_taus(spec["tau"], 8 * max(lanes_choices), 778)
        tuned = autotune.tune(dg, ts, tt, lanes_choices=lanes_choices, reps=8, budget_s=150.0,
                              cache_path=os.path.join(CACHE, "autotune.json"), log=log)
        k = int(tuned["lanes"])
        for key in autotune.TUNED_KEYS:
            if key in tuned:
                opts[key] = tuned[key]
    for flag, key in ((args.tpv, "threads_per_vertex"), (args.delay, "schedule_delay"),
                      (args.sweep_kernel, "sweep_kernel"), (args.fuse, "fuse_width"),
                      (args.ctas_per_sm, "ctas_per_sm"), (args.solo, "solo_width"), (args.span, "chunk_span"),
                      (args.core, "core_vertices")):
        if flag:
            opts[key] = flag
    if args.restrict >= 0:
        opts["restrict_sweep"] = args.restrict
    if args.fused >= 0:
        opts["fused_emission"] = args.fused
    if not args.landmarks:
        opts.pop("restrict_sweep", None)
    if args.trace:
        opts["record_trace"] = 1
    # batches in flight: each workspace has its own stream, so one batch's
    # emission and sort overlap the next batch's upward search
    wss = [P.Workspace(dg, k, stream=torch.cuda.Stream(), **opts) for _ in range(max(1, args.pipeline))]
    ws = wss[0]
    nb = 16
    batches = []
    for b in range(nb):
        s = synth.draw_sources(g, k, 10_000 * (rank + 1) + b)
        t = draw_taus(spec["tau"], k, 20_000 * (rank + 1) + b)
        batches.append((torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda(), s, t))
    outs = [(torch.zeros(k + 1, dtype=torch.int64, device="cuda"),
             torch.zeros(64 * 65536, dtype=torch.int32, device="cuda")) for _ in wss]
    sweep_ms, lat_ms, phases = [], [], []

    def run(count, record, wss):
        # batch i goes to workspace i mod len(wss); a workspace's previous
        # batch is collected before it takes the next one
        inflight = [None] * len(wss)

        def finish(j):
            i0, t0 = inflight[j]
            o_off, o_arcs = outs[j]
            wss[j].collect(out_arcs=o_arcs, out_offsets=o_off)
            if record:
                lat_ms.append((time.perf_counter() - t0) * 1e3)
                ph = wss[j].timings()
                phases.append(ph)
                sweep_ms.append(ph["sweep"])
            inflight[j] = None

        prev = None
        for i in range(count):
            j = i % len(wss)
            if inflight[j] is not None:
                finish(j)
            s, t, _, _ = batches[i % nb]
            inflight[j] = (i, time.perf_counter())
            # chained: this batch starts after the previous batch's sweep, so
            # its upward search and core overlap that batch's emission and sort
            wss[j].submit(s, t, after=prev if args.chain else None)
            prev = wss[j]
        for j in range(len(wss)):
            if inflight[j] is not None:
                finish(j)

    run(max(args.warmup, len(wss)), False, wss)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        main = torch.cuda.current_stream()
        ev0.record(main)
        for w in wss:
            w.stream.wait_event(ev0)
        run(args.steps, True, wss)
        for w in wss:
            e = torch.cuda.Event()
            e.record(w.stream)
            main.wait_event(e)
        ev1.record(main)
        torch.cuda.synchronize()
    el_ms = ev0.elapsed_time(ev1)
    # Kernel durations for the roofline and the phase split: with batches in
    # flight, a phase's events also span waits for the other streams' kernels,
    # so these come from batches run one at a time on one workspace, after the
    # throughput region (same kernels, same inputs).
    pipelined = {"latency_ms": lat_ms[:], "sweep_ms": sweep_ms[:]}
    lat_ms.clear(); sweep_ms.clear(); phases.clear()
    run(min(args.steps, 30), True, wss[:1])
    if args.trace:
        steps, ns = ws.trace()
        lo = A["level_off"]
        prev = 0
        log("[trace] kind levels vertices us")
        for st, t in zip(steps, ns):
            if st[0] == 2:
                log(f"[trace] prologue {t / 1e3:.1f}")
                continue
            nv = int(lo[st[2]] - lo[st[1]])
            log(f"[trace] {st[0]} {st[1]}-{st[2]} {nv} {(t - prev) / 1e3:.1f}")
            prev = max(prev, t)
    if dist:
        el_ms = max_over_ranks(el_ms, dist, "cuda")
        dist.barrier()
    value = job_throughput(world, k, args.steps, el_ms / 1e3)

    # end to end through the public call with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        pin_s = torch.empty(k, dtype=torch.int32, pin_memory=True)
        pin_t = torch.empty(k, dtype=torch.int32, pin_memory=True)
        pin_off = torch.empty(k + 1, dtype=torch.int64, pin_memory=True)
        pin_arcs = torch.empty(64 * 65536, dtype=torch.int32, pin_memory=True)
        hs, ht, ho, ha = pin_s.numpy(), pin_t.numpy(), pin_off.numpy(), pin_arcs.numpy()
        d2h = 0
        for i in range(args.warmup):
            hs[:] = batches[i % nb][2]; ht[:] = batches[i % nb][3]
            P.iso_query(dg, hs, ht, out_offsets=ho, out_arcs=ha, cap=ha.shape[0], **opts)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            hs[:] = batches[i % nb][2]; ht[:] = batches[i % nb][3]
            P.iso_query(dg, hs, ht, out_offsets=ho, out_arcs=ha, cap=ha.shape[0], **opts)
            d2h += int(ho[-1]) * 4 + (k + 1) * 8
        e2e_s = time.perf_counter() - t0
        if dist:
            e2e_s = max_over_ranks(e2e_s, dist, "cuda")
        e2e = {"value": job_throughput(world, k, args.steps, e2e_s), "unit": "queries/s",
               "h2d_bytes_per_step": 2 * 4 * k,
               "d2h_bytes_per_step": d2h // args.steps}

    serving_stats = None
    if not args.no_serving:
        from paper_1512_09090_gb300 import serving
        nreq = args.serve_requests
        s_src = synth.draw_sources(g, nreq, 4000 + rank)
        s_tau = synth.draw_taus_loguniform(nreq, 600, 72000, 5000 + rank)
        sopts = {kk: v for kk, v in opts.items() if kk != "record_trace"}
        with serving.IsoServer(dg, lanes=k, workspaces=2, memory_fraction=0.5, max_workspaces=4, **sopts) as srv:
            # a burst first: the pool grows while requests wait and memory allows
            serving.run_poisson(srv, s_src[: nreq // 2], s_tau[: nreq // 2], np.zeros(nreq // 2))
            # the server's own capacity: every request queued at once
            _, wall0 = serving.run_poisson(srv, s_src, s_tau, np.zeros(nreq))
            capacity = nreq / wall0
            rate = 0.8 * capacity                               # 80% of the measured capacity
            s_arr = synth.poisson_arrivals(nreq, rate, 6000 + rank)
            res, wall = serving.run_poisson(srv, s_src, s_tau, s_arr)
            nws, grown, refused = len(srv.workspaces), srv.grown, srv.refused_growth
        serving_stats = {"requests": nreq, "capacity_qps": round(capacity, 1), "offered_qps": round(rate, 1),
                         "achieved_qps": round(nreq / wall, 1), "workspaces": nws, "workspaces_grown": grown,
                         "growth_refused_by_memory": refused,
                         "tau": "log-uniform [600, 72000]", "arrivals": "Poisson", **serving.latency_summary(res)}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    K = lanes_class(k)
    alg = sum(sweep_bytes_scope(A, K).values())
    alg_design = sum(sweep_bytes(A, K).values())
    sw = statistics.mean(sweep_ms)
    peak, src = peaks()
    achieved = alg / (sw / 1e3) / 1e9
    traffic = sweep_traffic(args.workload, opts)
    info = ws.sweep_info()
    kern = f"k_sweep_tma<{K}>" if not info["core_levels"] else f"k_core + k_sweep_tma<{K}>"
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": kern,
            "alg_bytes_per_launch": alg, "alg_bytes_design": alg_design,
            "traffic_over_alg": None if traffic is None else round(traffic / alg, 3),
            "traffic_kernel": None if traffic is None else f"k_sweep_tma<{K}> (k_core's own bytes not counted)",
            "peak_source": src, "sweep_ms": round(sw, 4), "lanes_per_launch": K}
    lat = sorted(pipelined["latency_ms"])
    line = {"metric": METRIC, "value": round(value, 2), "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(el_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "graph": spec["graph"], "n": g.n, "m": g.m,
                       "m_down": int(A["down_src"].shape[0]), "levels": int(A["level_off"].shape[0] - 1),
                       "queries_per_sweep": k, "tau": list(spec["tau"]), "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (distance rows " + f"{4 * k * g.n / 1e9:.2f} GB)",
                       "opts": opts, "batches_in_flight": len(wss), "chained": bool(args.chain)},
            "roofline": roof,
            "latency_ms": {"p50": round(lat[len(lat) // 2], 3), "p99": round(lat[min(len(lat) - 1,
                                                                                     int(0.99 * len(lat)))], 3)},
            "phases_ms": {key: round(statistics.mean(p[key] for p in phases), 4) for key in phases[0]},
            "serving": serving_stats,
            "autotune": None if tuned is None else {kk: v for kk, v in tuned.items() if kk != "tried"},
            "gpu_launches": (4 + (1 if info["core_levels"] else 0) + (1 if opts.get("restrict_sweep") else 0)
                             - (1 if opts.get("fused_emission") else 0))
            * args.steps, "e2e": e2e,
            "sweep_shape": {**info, "skipped_chunks_last_batch": ws.skipped_chunks()}}
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, spec, k)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
