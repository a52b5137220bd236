"""Landmark distances for restricted sweeps (iso_ch_landmarks), on the host:
forward and backward distances equal the oracle's Dijkstra on the input graph
and on its reverse, and the lower bounds they give never exceed a true
distance (the property the restricted sweep relies on to skip chunks)."""

import numpy as np

import oracle
from paper_1512_09090_gb300 import synth

from helpers import workload

INF = 0x7FFFFFFF
UNREACH = 0xFFFFFFFF


def _oracle_dist(g, sources, reverse=False):
    tail, head = (g.head, g.tail) if reverse else (g.tail, g.head)
    taus = np.full(len(sources), 1 << 30, np.int32)
    _, _, d = oracle.query_batch(g.n, tail, head, g.weight, np.asarray(sources, np.int32), taus, want_dist=True,
                                 threads=8)
    return np.where(d == INF, UNREACH, d.astype(np.int64)).astype(np.uint64)


def test_landmark_distances_equal_dijkstra():
    g, ch = workload("grid64")
    v, f, b = ch.landmarks(4)
    assert len(set(v.tolist())) == 4
    assert np.array_equal(f.astype(np.uint64), _oracle_dist(g, v))
    assert np.array_equal(b.astype(np.uint64), _oracle_dist(g, v, reverse=True))


def test_landmark_distances_on_a_graph_with_unreachable_parts():
    g = synth.random_graph(300, 700, wmin=0, wmax=20, seed=7)
    import paper_1512_09090_gb300 as P
    ch = P.iso_build_ch(g.n, g.tail, g.head, g.weight)
    v, f, b = ch.landmarks(3)
    assert np.array_equal(f.astype(np.uint64), _oracle_dist(g, v))
    assert np.array_equal(b.astype(np.uint64), _oracle_dist(g, v, reverse=True))


def test_bounds_never_exceed_true_distances():
    g, ch = workload("grid1k")
    v, f, b = ch.landmarks(8)
    f = f.astype(np.int64)
    b = b.astype(np.int64)
    rng = np.random.default_rng(3)
    srcs = synth.draw_sources(g, 6, 11)
    d = _oracle_dist(g, srcs).astype(np.int64)
    for i, s in enumerate(srcs):
        t = rng.integers(0, g.n, size=5000)
        fin = (f[:, t] < UNREACH - 1) & (f[:, [s]] < UNREACH - 1)
        lb1 = np.where(fin, f[:, t] - f[:, [s]], 0).max(axis=0)
        fin2 = (b[:, t] < UNREACH - 1) & (b[:, [s]] < UNREACH - 1)
        lb2 = np.where(fin2, b[:, [s]] - b[:, t], 0).max(axis=0)
        true = d[i, t]
        assert np.all(np.maximum(lb1, lb2) <= true)
        # and the bounds are informative somewhere
        assert np.any(np.maximum(lb1, lb2) > 0)
