"""Seeded synthetic road-like graphs and isochrone queries.

This module only draws inputs: a perturbed grid graph G = (V, E) with integer
travel times len: E -> Z>=0 (Section 2 of Baum et al., "Fast Computation of
Isochrones in Road Networks") and query batches (source s, time limit tau;
Section 3).  It contains none of the query method's arithmetic, so both the
CUDA path and the CPU oracle can consume its output.

Graph recipe (the stand-in for the paper's road network, Section 6):
  * an R x C grid; each of the 2RC-R-C grid edges is kept with probability
    ``p_keep`` and becomes two directed arcs with independent lengths;
  * each of the two diagonals of every grid cell is kept independently with
    probability ``p_diag`` and likewise becomes two arcs;
  * lengths are uniform integers in [wmin, wmax];
  * highway tiers ``(period, factor)``: an arc lying along a row or column whose
    index is a multiple of ``period`` gets len' = max(1, len // factor); where
    tiers overlap the largest factor applies (diagonals are never highways);
  * vertex ids are randomly permuted and arcs shuffled, so the input is in no
    particular order.
"""

from __future__ import annotations

import dataclasses

import numpy as np

INF = 0x7FFFFFFF


@dataclasses.dataclass
class RoadGraph:
    n: int
    tail: np.ndarray   # int32[m]
    head: np.ndarray   # int32[m]
    weight: np.ndarray  # int32[m]
    rows: int = 0
    cols: int = 0
    grid_of: np.ndarray | None = None  # int64[n]: grid index r*C+c of each vertex id

    @property
    def m(self) -> int:
        return int(self.tail.shape[0])


def grid_road_graph(rows: int, cols: int, *, p_keep: float = 0.9, p_diag: float = 0.05,
                    wmin: int = 10, wmax: int = 100, highways=(), seed: int = 1,
                    permute: bool = True) -> RoadGraph:
    """Draw the perturbed grid road graph described in the module docstring."""
    rng = np.random.default_rng(seed)
    R, C = int(rows), int(cols)
    n = R * C
    gid = np.arange(n, dtype=np.int64).reshape(R, C)

    def tier_factor(index: np.ndarray) -> np.ndarray:
        f = np.ones(index.shape, dtype=np.int64)
        for period, factor in highways:
            f = np.where(index % int(period) == 0, np.maximum(f, int(factor)), f)
        return f

    ends_a, ends_b, facs = [], [], []
    # horizontal grid edges (r, c) - (r, c+1): lie along row r
    a = gid[:, :-1].ravel(); b = gid[:, 1:].ravel()
    r_idx = np.repeat(np.arange(R, dtype=np.int64), C - 1)
    ends_a.append(a); ends_b.append(b); facs.append(tier_factor(r_idx))
    # vertical grid edges (r, c) - (r+1, c): lie along column c
    a = gid[:-1, :].ravel(); b = gid[1:, :].ravel()
    c_idx = np.tile(np.arange(C, dtype=np.int64), R - 1)
    ends_a.append(a); ends_b.append(b); facs.append(tier_factor(c_idx))
    ea = np.concatenate(ends_a); eb = np.concatenate(ends_b); ef = np.concatenate(facs)
    keep = rng.random(ea.shape[0]) < p_keep
    ea, eb, ef = ea[keep], eb[keep], ef[keep]
    # diagonals of each cell: (r,c)-(r+1,c+1) and (r,c+1)-(r+1,c)
    d1a = gid[:-1, :-1].ravel(); d1b = gid[1:, 1:].ravel()
    d2a = gid[:-1, 1:].ravel(); d2b = gid[1:, :-1].ravel()
    da = np.concatenate([d1a, d2a]); db = np.concatenate([d1b, d2b])
    dkeep = rng.random(da.shape[0]) < p_diag
    da, db = da[dkeep], db[dkeep]
    ea = np.concatenate([ea, da]); eb = np.concatenate([eb, db])
    ef = np.concatenate([ef, np.ones(da.shape[0], dtype=np.int64)])
    # two directed arcs per kept edge, independent lengths
    tail = np.concatenate([ea, eb]); head = np.concatenate([eb, ea])
    fac = np.concatenate([ef, ef])
    w = rng.integers(wmin, wmax + 1, size=tail.shape[0], dtype=np.int64)
    w = np.maximum(1, w // fac) if highways else w
    if permute:
        perm = rng.permutation(n).astype(np.int64)      # grid index -> vertex id
        tail = perm[tail]; head = perm[head]
        order = rng.permutation(tail.shape[0])
        tail, head, w = tail[order], head[order], w[order]
        grid_of = np.empty(n, dtype=np.int64); grid_of[perm] = np.arange(n, dtype=np.int64)
    else:
        grid_of = np.arange(n, dtype=np.int64)
    return RoadGraph(n=n, tail=tail.astype(np.int32), head=head.astype(np.int32),
                     weight=w.astype(np.int32), rows=R, cols=C, grid_of=grid_of)


def random_graph(n: int, m: int, *, wmin: int = 0, wmax: int = 20, seed: int = 1,
                 self_loops: bool = True) -> RoadGraph:
    """Small arbitrary digraph (parallel arcs and self-loops allowed) for brute-force checks."""
    rng = np.random.default_rng(seed)
    tail = rng.integers(0, n, size=m, dtype=np.int64)
    head = rng.integers(0, n, size=m, dtype=np.int64)
    if not self_loops:
        bad = tail == head
        head[bad] = (head[bad] + 1) % max(n, 1)
    w = rng.integers(wmin, wmax + 1, size=m, dtype=np.int64)
    return RoadGraph(n=n, tail=tail.astype(np.int32), head=head.astype(np.int32),
                     weight=w.astype(np.int32))


def draw_sources(g: RoadGraph, k: int, seed: int) -> np.ndarray:
    """k sources drawn uniformly (with replacement) among vertices with out-degree > 0."""
    rng = np.random.default_rng(seed)
    outdeg = np.bincount(g.tail, minlength=g.n)
    cand = np.flatnonzero(outdeg > 0)
    if cand.size == 0:
        cand = np.arange(g.n)
    return cand[rng.integers(0, cand.size, size=k)].astype(np.int32)


def draw_taus_uniform(k: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=k, dtype=np.int64).astype(np.int32)


def draw_taus_loguniform(k: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), size=k))
    return np.clip(np.rint(x), lo, hi).astype(np.int32)


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


# The five workloads: an R x C grid and its highway tiers, plus the query recipe.
WORKLOADS = {
    "grid64": dict(rows=64, cols=64, highways=(), seed=1),
    "grid1k": dict(rows=1000, cols=1000, highways=((32, 4),), seed=2),
    "grid18m": dict(rows=4243, cols=4243, highways=((16, 2), (128, 4), (1024, 8)), seed=3),
    # a 4M-vertex graph with the same tiers, for profiling runs that must stay a few GB
    "grid4m": dict(rows=2000, cols=2000, highways=((16, 2), (128, 4), (1024, 8)), seed=4),
}


def workload_graph(name: str) -> RoadGraph:
    spec = dict(WORKLOADS[name])
    return grid_road_graph(spec.pop("rows"), spec.pop("cols"), **spec)
