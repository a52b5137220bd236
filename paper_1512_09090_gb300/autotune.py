"""Autotuner for batched isochrone queries.

For a device graph it times batches of real queries on the real path and
picks, by query throughput:
  - lanes per sweep k (when the caller allows more than one choice),
  - threads per vertex of the TMA-staged sweep (per lane class),
  - the schedule delay (in rounds of one chunk per CTA),
  - the per-lane core's size (core_vertices),
  - the narrow-level threshold (fuse_width: leading levels below it run
    grid-synchronously, later narrow ones with a warp per vertex),
  - the CTA-0-alone width of the top levels (solo_width, used without core),
  - the chunk span limit (chunk_span, 0 among the candidates),
  - restricted sweeps on or off (restrict_sweep), where the graph has landmarks,
  - emission fused into the sweep or as a separate pass (fused_emission).
The search is coordinate descent from the library's defaults: one axis at a
time, keeping the best value before moving on, for as many passes as the time
budget allows.  Results are cached in a JSON file keyed by the graph's shape,
the device and a hash of the kernel sources, so a process that uploads the
same graph again skips the search.

Every candidate computes the same labels and lists (the options change only
how the work is scheduled), so the tuner chooses among results that are
identical by construction.
"""

from __future__ import annotations

import hashlib
import json
import os
import time

from . import _lib

# threads per vertex supported by the TMA-staged sweep, per lane class
TPV_CHOICES = {1: (1,), 4: (1,), 8: (1,), 16: (2, 4), 32: (4, 8), 64: (8, 16)}
DELAY_ROUNDS = (2, 3, 4, 6)
CORE_CHOICES = (0, 20000, -1)
FUSE_CHOICES = (0, -1)
SOLO_CHOICES = (0, -1)
SPAN_CHOICES = (0, 10000)
COMBO_SPANS = (4096, 16384)  # chunk spans tried together with restricted sweeps
_CSRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")


def source_hash() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(_CSRC)):
        if f.endswith((".cu", ".cuh", ".cpp", ".h")):
            with open(os.path.join(_CSRC, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:12]


def graph_key(g: _lib.DeviceGraph) -> str:
    import torch
    dev = torch.cuda.get_device_name(g.device)
    return f"n{g.n}-m{g.m}-down{g.m_down}-L{g.levels}-lm{getattr(g, 'landmarks', 0)}-{dev}-src{source_hash()}"


def _time_config(g, lanes, sources, taus, opts, reps):
    import torch
    ws = _lib.Workspace(g, lanes, use_cuda_graph=1, **opts)
    try:
        ws.submit(sources[:lanes], taus[:lanes])
        ws.collect()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in range(reps):
            s = sources[(r * lanes) % len(sources):][:lanes]
            t = taus[(r * lanes) % len(taus):][:lanes]
            if len(s) < lanes:
                s, t = sources[:lanes], taus[:lanes]
            ws.submit(s, t)
            ws.collect()
        el = time.perf_counter() - t0
    finally:
        ws.free()
    return lanes * reps / el


def axes_for(lanes: int, sms: int, landmarks: bool = False) -> list[tuple[str, tuple]]:
    """The tuned options and their candidate values for a lane count (0 = the library's default);
    restricted sweeps are a candidate where the graph has landmarks."""
    axes = [("fused_emission", (0, 1)),
            ("threads_per_vertex", TPV_CHOICES.get(lanes, (1,))),
            ("schedule_delay", tuple(r * sms for r in DELAY_ROUNDS)),
            ("core_vertices", CORE_CHOICES),
            ("fuse_width", FUSE_CHOICES),
            ("solo_width", SOLO_CHOICES),
            ("chunk_span", SPAN_CHOICES)]
    if landmarks:
        axes.insert(0, ("restrict_sweep", (0, 1)))
    return axes


def tune(g: _lib.DeviceGraph, sources, taus, lanes_choices=(64,), reps: int = 5, cache_path: str | None = None,
         budget_s: float = 120.0, log=None, passes: int = 2) -> dict:
    """Best {"lanes", **iso_query_opts} for g on this kind of query mix.  The
    result also lists every configuration tried ("tried") and the axes."""
    key = graph_key(g)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    ck = f"{key}-lanes{'_'.join(map(str, lanes_choices))}"
    if ck in cache:
        return cache[ck]
    import torch
    sms = torch.cuda.get_device_properties(g.device).multi_processor_count
    start = time.perf_counter()
    tried = []
    seen = {}

    def score(lanes, opts):
        k = (lanes, tuple(sorted(opts.items())))
        if k in seen:
            return seen[k]
        try:
            qps = _time_config(g, lanes, sources, taus, opts, reps)
        except _lib.IsoError:
            qps = -1.0
        seen[k] = qps
        tried.append({"lanes": lanes, **opts, "qps": round(qps, 1)})
        if log:
            log(f"[autotune] lanes={lanes} {opts} -> {qps:.0f} q/s")
        return qps

    best_lanes, best_opts, best_qps = None, {}, -1.0
    for lanes in lanes_choices:
        opts = {}
        cur = score(lanes, opts)
        for _ in range(passes):
            improved = False
            for name, values in axes_for(lanes, sms, getattr(g, "landmarks", 0) > 0):
                for v in values:
                    if time.perf_counter() - start > budget_s:
                        break
                    cand = {**opts, name: v}
                    cand = {kk: vv for kk, vv in cand.items() if vv != 0}  # 0 = default: leave it out
                    q = score(lanes, cand)
                    if q > cur * 1.005:  # keep a change only if it is clearly better
                        opts, cur, improved = cand, q, True
            if not improved:
                break
        # restricted sweeps skip more with spatially compact chunks: try the pair
        if getattr(g, "landmarks", 0) > 0:
            for span in COMBO_SPANS:
                if time.perf_counter() - start > budget_s:
                    break
                cand = {**opts, "restrict_sweep": 1, "chunk_span": span}
                q = score(lanes, cand)
                if q > cur * 1.005:
                    opts, cur = cand, q
        if cur > best_qps:
            best_lanes, best_opts, best_qps = lanes, opts, cur
    result = {"lanes": best_lanes if best_lanes is not None else lanes_choices[0], **best_opts,
              "qps": round(best_qps, 1),
              "axes": [a for a, _ in axes_for(best_lanes or lanes_choices[0], sms, getattr(g, "landmarks", 0) > 0)],
              "tried": tried}
    if cache_path:
        cache[ck] = result
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return result


TUNED_KEYS = ("threads_per_vertex", "schedule_delay", "core_vertices", "fuse_width", "solo_width", "chunk_span",
              "restrict_sweep", "fused_emission")
