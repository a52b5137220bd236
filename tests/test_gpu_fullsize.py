"""Parity at the benchmark's full size: the 4,243 x 4,243 grid (18,003,049
vertices, 68,396,596 arcs), 64 queries per sweep with limits drawn uniformly
from [3,600, 72,000], in the launch configuration bench.py times (TMA-staged
sweep, CUDA-graph replay), and 16 sources with a shared limit of 36,000.  The
oracle computes every lane one by one (Dijkstra stopped at tau + full arc
scan, on all host cores); lists and labels must be identical."""

import os

import numpy as np
import pytest

import oracle
import paper_1512_09090_gb300 as P
from paper_1512_09090_gb300 import chcache, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module")
def big():
    g, ch = chcache.workload_graph_and_ch("grid18m")
    return g, P.iso_upload_graph(ch)


def _batch(dg, srcs, taus, **opts):
    ws = P.Workspace(dg, len(srcs), use_cuda_graph=1, **opts)
    ws.submit(srcs, taus)
    off, arcs, _ = ws.collect()
    # a second batch on the same workspace (CUDA-graph replay) gives the same answer
    ws.submit(srcs, taus)
    off2, arcs2, _ = ws.collect()
    info = ws.sweep_info()
    ws.free()
    assert np.array_equal(off, off2) and np.array_equal(arcs, arcs2)
    return off, arcs, info


def _against_oracle(g, srcs, taus, off, arcs, lanes):
    o_off, o_arcs, _ = oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs[lanes], taus[lanes],
                                          threads=os.cpu_count() or 1)
    for j, i in enumerate(lanes):
        assert np.array_equal(arcs[off[i]:off[i + 1]], o_arcs[o_off[j]:o_off[j + 1]]), i


def test_fullsize_batch_of_64_against_oracle(big):
    # the benchmark's workload: 64 sources, limits uniform in [3,600, 72,000];
    # every lane is checked
    g, dg = big
    k = 64
    srcs = synth.draw_sources(g, k, 10_001)
    taus = synth.draw_taus_uniform(k, 3600, 72000, 20_001)
    off, arcs, info = _batch(dg, srcs, taus)
    assert info["core_levels"] > 0 and info["chunks"] > 0
    _against_oracle(g, srcs, taus, off, arcs, list(range(k)))


def test_fullsize_vertices_in_range(big):
    g, dg = big
    k = 64
    srcs = synth.draw_sources(g, k, 10_004)
    taus = synth.draw_taus_uniform(k, 3600, 72000, 20_004)
    ws = P.Workspace(dg, k, use_cuda_graph=1)
    ws.submit(srcs, taus)
    ws.collect()
    bits = ws.collect_range()
    ws.free()
    lanes = [0, 31, 63, int(np.argmax(taus))]
    _, _, o_dist = oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs[lanes], taus[lanes], want_dist=True,
                                      threads=os.cpu_count() or 1)
    got = np.unpackbits(bits[lanes].view(np.uint8), axis=1, bitorder="little")[:, :g.n].astype(bool)
    assert np.array_equal(got, o_dist != 0x7FFFFFFF)


def test_fullsize_fused_emission(big):
    # the sweep emits the isochrone edges itself, 64 lanes, every lane checked
    g, dg = big
    k = 64
    srcs = synth.draw_sources(g, k, 10_007)
    taus = synth.draw_taus_uniform(k, 3600, 72000, 20_007)
    off, arcs, _ = _batch(dg, srcs, taus, fused_emission=1)
    _against_oracle(g, srcs, taus, off, arcs, list(range(k)))


def test_fullsize_16_sources_shared_limit_against_oracle(big):
    # 16 sources batched in one sweep with a shared limit of 36,000
    g, dg = big
    k = 16
    srcs = synth.draw_sources(g, k, 10_002)
    taus = np.full(k, 36000, np.int32)
    off, arcs, _ = _batch(dg, srcs, taus)
    _against_oracle(g, srcs, taus, off, arcs, list(range(k)))


def test_fullsize_global_memory_staging_paths(big):
    # lowered staging limits send many chunks of the 18M sweep through the
    # paths that read arcs and dependency lists from global memory
    g, dg = big
    k = 64
    srcs = synth.draw_sources(g, k, 10_003)
    taus = synth.draw_taus_uniform(k, 3600, 72000, 20_003)
    off, arcs, info = _batch(dg, srcs, taus, debug_stage_arcs=1024, debug_stage_deps=4)
    assert info["chunks_over_arc_cap"] > 0 and info["chunks_over_dep_cap"] > 0
    _against_oracle(g, srcs, taus, off, arcs, [0, 21, 42, 63, int(np.argmax(taus)), int(np.argmin(taus))])


def test_fullsize_labels_sampled_against_oracle(big):
    g, dg = big
    srcs = synth.draw_sources(g, 2, 30_001)
    taus = np.array([36000, 72000], np.int32)
    off, arcs, dist = P.iso_query(dg, srcs, taus, want_dist=True)
    _, _, o_dist = oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs, taus, want_dist=True, threads=2)
    assert np.array_equal(dist, o_dist)


def test_fullsize_restricted_sweep(big):
    # one source per launch with small limits, and a 64-lane batch, with chunks
    # skipped by landmark bounds
    g, dg = big
    ch = chcache.workload_graph_and_ch("grid18m")[1]
    dg.add_landmarks(ch, 8)
    srcs = synth.draw_sources(g, 4, 10_005)
    taus = np.array([3600, 5000, 9000, 20000], np.int32)
    for i in range(4):
        ws = P.Workspace(dg, 1, use_cuda_graph=1, restrict_sweep=1)
        ws.submit(srcs[i:i + 1], taus[i:i + 1])
        off, arcs, _ = ws.collect()
        assert ws.skipped_chunks() > 0
        ws.free()
        _against_oracle(g, srcs[i:i + 1], taus[i:i + 1], off, arcs, [0])
    k = 64
    srcs = synth.draw_sources(g, k, 10_006)
    taus = synth.draw_taus_uniform(k, 3600, 72000, 20_006)
    off, arcs, _ = _batch(dg, srcs, taus, restrict_sweep=1)
    _against_oracle(g, srcs, taus, off, arcs, [0, 17, 38, 63, int(np.argmin(taus))])
