"""Host test of the seeded input generator (paper_1512_09090_gb300/synth.py)
against the recipe it states: grid and diagonal arcs only, both directions of
every kept edge with independent lengths, lengths in [wmin, wmax] divided by
the largest highway factor of the row or column an arc lies on, keep rates
near p_keep and p_diag, a vertex permutation that preserves the graph, and
query draws inside their ranges."""

import numpy as np

from paper_1512_09090_gb300 import synth


def _grid_coords(g, v):
    gi = g.grid_of[v]
    return gi // g.cols, gi % g.cols


def test_grid_arcs_follow_the_recipe():
    R, C = 60, 70
    tiers = ((8, 2), (32, 4))
    g = synth.grid_road_graph(R, C, highways=tiers, seed=11)
    assert g.n == R * C and g.tail.dtype == np.int32 and g.weight.dtype == np.int32
    rt, ct = _grid_coords(g, g.tail)
    rh, ch = _grid_coords(g, g.head)
    dr, dc = rh - rt, ch - ct
    straight = (np.abs(dr) + np.abs(dc)) == 1
    diagonal = (np.abs(dr) == 1) & (np.abs(dc) == 1)
    assert np.all(straight | diagonal)                     # grid and cell-diagonal arcs only
    # every kept edge is two arcs, one each way
    fwd = set(zip(g.tail.tolist(), g.head.tolist()))
    assert all((h, t) in fwd for t, h in fwd)
    assert len(fwd) == g.m                                 # no parallel arcs
    # lengths: [10, 100] // factor, at least 1; factor from the row (horizontal
    # arcs) or column (vertical arcs) index, diagonals never highways
    line = np.where(dr == 0, rt, ct)
    fac = np.ones(g.m, np.int64)
    for period, factor in tiers:
        fac = np.where(straight & (line % period == 0), np.maximum(fac, factor), fac)
    lo = np.maximum(1, 10 // fac)
    hi = 100 // fac
    assert np.all(g.weight >= lo) and np.all(g.weight <= hi)
    assert np.all(g.weight[fac == 1] >= 10)
    # keep rates (binomial, 5 sigma)
    n_edges, n_diag = 2 * R * C - R - C, 2 * (R - 1) * (C - 1)
    kept, kept_d = straight.sum() // 2, diagonal.sum() // 2
    assert abs(kept - 0.9 * n_edges) < 5 * np.sqrt(n_edges * 0.9 * 0.1)
    assert abs(kept_d - 0.05 * n_diag) < 5 * np.sqrt(n_diag * 0.05 * 0.95)


def test_permutation_preserves_the_graph():
    a = synth.grid_road_graph(30, 40, seed=5, permute=False)
    b = synth.grid_road_graph(30, 40, seed=5, permute=True)
    assert np.array_equal(a.grid_of, np.arange(a.n))
    ea = sorted(zip(a.tail.tolist(), a.head.tolist(), a.weight.tolist()))
    eb = sorted(zip(b.grid_of[b.tail].tolist(), b.grid_of[b.head].tolist(), b.weight.tolist()))
    assert ea == eb                                        # same arcs and lengths in grid coordinates
    assert sorted(b.grid_of.tolist()) == list(range(b.n))  # a permutation


def test_query_draws_stay_in_range():
    g = synth.grid_road_graph(20, 20, seed=3, p_keep=0.5)
    s = synth.draw_sources(g, 500, 7)
    outdeg = np.bincount(g.tail, minlength=g.n)
    assert np.all(outdeg[s] > 0)
    t = synth.draw_taus_uniform(500, 3600, 72000, 8)
    assert t.min() >= 3600 and t.max() <= 72000
    t = synth.draw_taus_loguniform(500, 600, 72000, 9)
    assert t.min() >= 600 and t.max() <= 72000
    # log-uniform: about half of the draws below the geometric mean
    assert 0.4 < np.mean(t < np.sqrt(600 * 72000)) < 0.6
    a = synth.poisson_arrivals(2000, 100.0, 1)
    assert np.all(np.diff(a) > 0) and abs(a[-1] / 2000 - 0.01) < 0.002
    # seeded: the same draws again
    assert np.array_equal(s, synth.draw_sources(g, 500, 7))
