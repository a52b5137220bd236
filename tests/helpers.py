"""Shared test helpers: cached CH builds and a plain CPU PHAST used to check a
hierarchy's structure before any kernel runs."""

import heapq
import os

import numpy as np

import paper_1512_09090_gb300 as P
from paper_1512_09090_gb300 import synth

INF = 0x7FFFFFFF
_CH = {}


def arcs_of(case):
    a = np.array(case["arcs"], dtype=np.int64).reshape(-1, 3)
    return case["n"], a[:, 0].astype(np.int32), a[:, 1].astype(np.int32), a[:, 2].astype(np.int32)


def workload(name):
    key = ("w", name)
    if key not in _CH:
        g = synth.workload_graph(name)
        _CH[key] = (g, P.iso_build_ch(g.n, g.tail, g.head, g.weight))
    return _CH[key]


def cpu_phast(A, s, tau):
    """PHAST over the CH arrays A (sweep order): Dijkstra in the upward graph
    from s, then one pass over the levels top-down; labels > tau become INF.
    Returns labels indexed by original vertex id."""
    pos, perm, lo = A["pos"], A["perm"], A["level_off"]
    n = pos.shape[0]
    d = np.full(n, np.iinfo(np.int64).max, dtype=np.int64)
    s0 = int(pos[s])
    d[s0] = 0
    heap = [(0, s0)]
    done = set()
    while heap:
        du, u = heapq.heappop(heap)
        if u in done or du != d[u]:
            continue
        done.add(u)
        for j in range(A["up_off"][u], A["up_off"][u + 1]):
            x, nd = int(A["up_dst"][j]), du + int(A["up_w"][j])
            if nd <= tau and nd < d[x]:
                d[x] = nd
                heapq.heappush(heap, (nd, x))
    do, src, w = A["down_off"], A["down_src"].astype(np.int64), A["down_w"].astype(np.int64)
    for j in range(lo.shape[0] - 1):
        a, b = lo[j], lo[j + 1]
        if a == b:
            continue
        e0, e1 = do[a], do[b]
        heads = np.repeat(np.arange(a, b), np.diff(do[a:b + 1]))
        cand = np.where(d[src[e0:e1]] <= tau, d[src[e0:e1]] + w[e0:e1], np.iinfo(np.int64).max)
        np.minimum.at(d, heads, cand)
        seg = d[a:b]
        seg[seg > tau] = np.iinfo(np.int64).max
    out = np.where(d <= tau, d, INF).astype(np.int64)
    res = np.empty(n, dtype=np.int64)
    res[perm] = out
    return res
