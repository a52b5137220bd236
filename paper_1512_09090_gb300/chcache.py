"""On-disk cache of contraction hierarchies for the synthetic workloads, so the
benchmark and the full-size tests build an 18M-vertex hierarchy once per
machine.  Files live in the package's _cache directory (not versioned); the
key covers the generator's parameters and the CH builder's source."""

from __future__ import annotations

import hashlib
import json
import os
import sys
import time

from . import _lib, synth

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_cache")


def _log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload_graph_and_ch(name: str, log=_log):
    t0 = time.time()
    g = synth.workload_graph(name)
    log(f"[chcache] graph {name}: n={g.n} m={g.m} ({time.time() - t0:.1f}s)")
    h = hashlib.sha1(json.dumps(synth.WORKLOADS[name], sort_keys=True).encode())
    for src in ("ch.cpp", "ch_io.cpp"):
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", src), "rb") as f:
            h.update(f.read())
    path = os.path.join(CACHE, f"{name}-{h.hexdigest()[:12]}.ch")
    if os.path.exists(path):
        try:
            ch = _lib.iso_load_ch(path)
            log(f"[chcache] CH loaded from {os.path.basename(path)}")
            return g, ch
        except _lib.IsoError as e:
            log(f"[chcache] cache unreadable ({e}); rebuilding")
    t0 = time.time()
    ch = _lib.iso_build_ch(g.n, g.tail, g.head, g.weight)
    log(f"[chcache] CH built in {time.time() - t0:.1f}s: {ch.stats()}")
    try:
        os.makedirs(CACHE, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        ch.save(tmp)
        os.replace(tmp, path)
    except OSError as e:
        log(f"[chcache] could not cache the CH: {e}")
    return g, ch
