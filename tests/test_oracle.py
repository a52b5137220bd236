"""Pins for the CPU oracle (Section 3's definition and isoDijkstra).

Every check compares the oracle with something other than itself: hand-worked
examples (tests/golden), brute-force distances (Floyd-Warshall and exhaustive
path enumeration written here), scipy's shortest-path routine, and invariants
that any correct isochrone must satisfy.  A final test compiles variants of the
oracle with a planted mistake and shows that these pins reject each one.
"""

import itertools

import numpy as np
import pytest

import oracle
from paper_1512_09090_gb300 import synth

INF = oracle.INF


def _arrays(case):
    a = np.array(case["arcs"], dtype=np.int64).reshape(-1, 3)
    return case["n"], a[:, 0].astype(np.int32), a[:, 1].astype(np.int32), a[:, 2].astype(np.int32)


def test_golden_hand_cases(golden_cases):
    for case in golden_cases:
        n, t, h, w = _arrays(case)
        for q in case["queries"]:
            arcs, dist = oracle.isochrone(n, t, h, w, q["s"], q["tau"])
            assert arcs.tolist() == q["expected"], (case["name"], q)
            assert oracle.iso_dijkstra(n, t, h, w, q["s"], q["tau"]).tolist() == q["expected"], (case["name"], q)
            if "dist" in q:
                want = [d if d <= q["tau"] else INF for d in q["dist"]]
                assert dist.tolist() == want, (case["name"], q)


def floyd_warshall(n, t, h, w):
    """All-pairs distances, plain triple loop (Python ints, inf = None)."""
    D = [[None] * n for _ in range(n)]
    for v in range(n):
        D[v][v] = 0
    for a, b, c in zip(t.tolist(), h.tolist(), w.tolist()):
        if D[a][b] is None or c < D[a][b]:
            D[a][b] = c
    for x in range(n):
        for i in range(n):
            if D[i][x] is None:
                continue
            for j in range(n):
                if D[x][j] is None:
                    continue
                c = D[i][x] + D[x][j]
                if D[i][j] is None or c < D[i][j]:
                    D[i][j] = c
    return D


def path_enumeration(n, t, h, w, s):
    """Shortest distances from s by trying every simple path (tiny graphs only)."""
    adj = {v: [] for v in range(n)}
    for a, b, c in zip(t.tolist(), h.tolist(), w.tolist()):
        adj[a].append((b, c))
    best = [None] * n
    def go(v, d, seen):
        if best[v] is None or d < best[v]:
            best[v] = d
        for b, c in adj[v]:
            if b not in seen:
                go(b, d + c, seen | {b})
    go(s, 0, {s})
    return best


def definition_isochrone(t, h, dist, tau):
    inr = [d is not None and d <= tau for d in dist]
    return [e for e, (a, b) in enumerate(zip(t.tolist(), h.tolist())) if inr[a] != inr[b]]


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 9))
    m = int(rng.integers(0, 3 * n + 1))
    g = synth.random_graph(n, m, wmin=0, wmax=20, seed=seed)
    D = floyd_warshall(n, g.tail, g.head, g.weight)
    for s in range(n):
        P = path_enumeration(n, g.tail, g.head, g.weight, s)
        assert P == D[s]
        finite = [d for d in D[s] if d is not None]
        taus = sorted({0, max(finite), max(finite) + 1, *[d for d in finite], *[d - 1 for d in finite if d > 0]})
        for tau in taus:
            want = definition_isochrone(g.tail, g.head, D[s], tau)
            arcs, dist = oracle.isochrone(n, g.tail, g.head, g.weight, s, tau)
            assert arcs.tolist() == want
            assert dist.tolist() == [d if d is not None and d <= tau else INF for d in D[s]]
            assert oracle.iso_dijkstra(n, g.tail, g.head, g.weight, s, tau).tolist() == want


@pytest.mark.parametrize("seed", range(6))
def test_against_scipy_dijkstra(seed):
    scipy_sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g = synth.grid_road_graph(30, 40, highways=((8, 3),), seed=seed)
    # positive lengths, parallel arcs collapse to the minimum in a sparse matrix
    A = scipy_sp.coo_matrix((g.weight.astype(np.float64), (g.tail, g.head)), shape=(g.n, g.n)).tocsr()
    A.sum_duplicates()  # no duplicates in this generator; kept explicit
    srcs = synth.draw_sources(g, 5, seed)
    D = csgraph.dijkstra(A, directed=True, indices=srcs)
    for i, s in enumerate(srcs):
        for tau in (0, 300, 1500, 5000):
            arcs, dist = oracle.isochrone(g.n, g.tail, g.head, g.weight, s, tau)
            want_d = np.where(D[i] <= tau, D[i], INF).astype(np.int64)
            assert np.array_equal(dist.astype(np.int64), want_d)
            inr = D[i] <= tau
            want = np.flatnonzero(inr[g.tail] != inr[g.head])
            assert np.array_equal(arcs, want)


def check_invariants(g, s, tau, arcs, dist):
    """Properties every correct answer has (Section 3), independent of how it was found."""
    inr = dist != INF
    assert inr[s]
    assert np.all(dist[inr] <= tau) and np.all(dist[inr] >= 0)
    # soundness and completeness of the reported set
    cross = inr[g.tail] != inr[g.head]
    assert np.array_equal(np.flatnonzero(cross), arcs)
    assert np.all(np.diff(arcs) > 0)
    # closure: an arc from an in-range vertex that stays within tau ends in range
    du = dist[g.tail].astype(np.int64) + g.weight
    stay = inr[g.tail] & (du <= tau)
    assert np.all(inr[g.head[stay]])
    # labels are no larger than any relaxation along an arc from the range
    assert np.all(dist[g.head[stay]].astype(np.int64) <= du[stay])
    # every in-range v != s has a tight in-arc from the range
    tight = stay & (dist[g.head].astype(np.int64) == du)
    has_tight = np.zeros(g.n, dtype=bool)
    has_tight[g.head[tight]] = True
    need = inr.copy(); need[s] = False
    assert np.all(has_tight[need])


@pytest.mark.parametrize("name", ["grid64"])
def test_invariants_and_monotonicity(name):
    g = synth.workload_graph(name)
    srcs = synth.draw_sources(g, 6, 11)
    for s in srcs:
        prev = None
        for tau in (0, 100, 700, 1500, 4000, 20000):
            arcs, dist = oracle.isochrone(g.n, g.tail, g.head, g.weight, s, tau)
            check_invariants(g, s, tau, arcs, dist)
            assert np.array_equal(arcs, oracle.iso_dijkstra(g.n, g.tail, g.head, g.weight, s, tau))
            inr = dist != INF
            if prev is not None:
                assert np.all(inr[prev])            # range grows with tau
            prev = inr


def test_batch_equals_single():
    g = synth.workload_graph("grid64")
    srcs = synth.draw_sources(g, 7, 3)
    taus = synth.draw_taus_uniform(7, 0, 3000, 4)
    off, arcs, dist = oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs, taus, want_dist=True, threads=3)
    for i in range(7):
        a, d = oracle.isochrone(g.n, g.tail, g.head, g.weight, srcs[i], taus[i])
        assert np.array_equal(arcs[off[i]:off[i + 1]], a)
        assert np.array_equal(dist[i], d)


def test_bad_input_rejected():
    with pytest.raises(ValueError):
        oracle.tau_dijkstra(3, [0], [1], [1], 5, 10)
    with pytest.raises(ValueError):
        oracle.tau_dijkstra(3, [0], [1], [1], 0, -1)


MUTANTS = {1: "strict < tau", 2: "relaxes toward the tail", 3: "drops the arc length",
           4: "OR instead of XOR", 5: "no infinity-key insertion in isoDijkstra"}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_reject_planted_mistakes(mutant, golden_cases):
    """Each variant with a planted mistake fails at least one hand-worked case."""
    failed = False
    for case in golden_cases:
        n, t, h, w = _arrays(case)
        for q in case["queries"]:
            a, _ = oracle.isochrone(n, t, h, w, q["s"], q["tau"], mutant=mutant)
            b = oracle.iso_dijkstra(n, t, h, w, q["s"], q["tau"], mutant=mutant)
            if a.tolist() != q["expected"] or b.tolist() != q["expected"]:
                failed = True
    assert failed, MUTANTS[mutant]
