"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Distances (clamped to INF beyond tau) and sorted isochrone-edge lists must be
bit-exact: lengths and labels are int32 and no approximate arithmetic is
involved.  Covers every lane class (k = 1..64), every threads-per-vertex
variant, level fusion on and off, CUDA graphs on and off, host and device
buffers, uneven limits, duplicate sources, degenerate graphs, overflow,
argument errors and the barrier timeout."""

import numpy as np
import pytest

import oracle
import paper_1512_09090_gb300 as P
from paper_1512_09090_gb300 import synth

from helpers import INF, arcs_of, workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

_DEV = {}


def dev_graph(name):
    if name not in _DEV:
        g, ch = workload(name)
        _DEV[name] = (g, P.iso_upload_graph(ch))
    return _DEV[name]


def check_batch(g, dg, srcs, taus, want_dist=True, **opts):
    off, arcs, dist = P.iso_query(dg, srcs, taus, want_dist=want_dist, **opts)
    o_off, o_arcs, o_dist = oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs, taus, want_dist=want_dist,
                                               threads=8)
    assert np.array_equal(off, o_off)
    assert np.array_equal(arcs, o_arcs)
    if want_dist:
        assert np.array_equal(dist, o_dist)
    return off, arcs


@pytest.mark.parametrize("fused", [0, 1])
def test_golden_hand_cases(golden_cases, fused):
    for case in golden_cases:
        n, t, h, w = arcs_of(case)
        ch = P.iso_build_ch(n, t, h, w)
        dg = P.iso_upload_graph(ch)
        srcs = np.array([q["s"] for q in case["queries"]], np.int32)
        taus = np.array([q["tau"] for q in case["queries"]], np.int32)
        off, arcs, dist = P.iso_query(dg, srcs, taus, want_dist=True, fused_emission=fused)
        for i, q in enumerate(case["queries"]):
            assert arcs[off[i]:off[i + 1]].tolist() == q["expected"], (case["name"], q)
            if "dist" in q:
                want = [x if x <= q["tau"] else INF for x in q["dist"]]
                assert dist[i].tolist() == want, (case["name"], q)


@pytest.mark.parametrize("seed", range(12))
def test_random_small_graphs(seed):
    # random multigraphs: one-way arcs (dummy downward arcs for fused emission),
    # zero lengths, self-loops, parallel arcs
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 60))
    g = synth.random_graph(n, int(rng.integers(0, 5 * n)), wmin=0, wmax=40, seed=seed)
    dg = P.iso_upload_graph(P.iso_build_ch(g.n, g.tail, g.head, g.weight))
    k = int(rng.integers(1, 65))
    srcs = rng.integers(0, n, size=k).astype(np.int32)
    taus = rng.integers(0, 200, size=k).astype(np.int32)
    check_batch(g, dg, srcs, taus)
    check_batch(g, dg, srcs, taus, fused_emission=1)


@pytest.mark.parametrize("seed", range(3))
def test_fused_emission_one_way_grid(seed):
    # a 300 x 300 grid with 30% of its arcs dropped: many one-way arcs, so
    # dummy downward arcs order their endpoints, through the chunk schedule as
    # well as the core
    rng = np.random.default_rng(300 + seed)
    base = synth.grid_road_graph(300, 300, seed=40 + seed)
    keep = rng.random(base.m) > 0.3
    g = synth.RoadGraph(n=base.n, tail=base.tail[keep], head=base.head[keep], weight=base.weight[keep])
    dg = P.iso_upload_graph(P.iso_build_ch(g.n, g.tail, g.head, g.weight))
    srcs = synth.draw_sources(g, 16, 50 + seed)
    taus = synth.draw_taus_uniform(16, 0, 20000, 60 + seed)
    for core in (0, -1):
        check_batch(g, dg, srcs, taus, fused_emission=1, core_vertices=core)


@pytest.mark.parametrize("k", [1, 5, 16, 64])
@pytest.mark.parametrize("opts", [{}, {"core_vertices": -1}, {"fuse_width": -1}, {"threads_per_vertex": 0}])
def test_fused_emission_grid1k(k, opts):
    g, dg = dev_graph("grid1k")
    srcs = synth.draw_sources(g, k, 180 + k)
    taus = synth.draw_taus_uniform(k, 0, 60000, 181 + k)
    check_batch(g, dg, srcs, taus, want_dist=False, fused_emission=1, use_cuda_graph=1, **opts)


def test_fused_emission_with_restricted_sweep_and_overflow():
    g, dg = lm_graph("grid1k")
    srcs = synth.draw_sources(g, 3, 191)
    taus = np.array([2000, 5000, 40000], np.int32)
    check_batch(g, dg, srcs, taus, fused_emission=1, restrict_sweep=1)
    # 64 lanes with a large limit
    srcs = synth.draw_sources(g, 64, 192)
    taus = np.full(64, 60000, np.int32)
    check_batch(g, dg, srcs, taus, want_dist=False, fused_emission=1)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 16, 17, 32, 64, 65, 130])
def test_grid64_lane_counts(k):
    g, dg = dev_graph("grid64")
    srcs = synth.draw_sources(g, k, 1000 + k)
    taus = synth.draw_taus_uniform(k, 0, 4000, 2000 + k)
    check_batch(g, dg, srcs, taus)


PLAIN_VARIANTS = [(8, 2), (16, 1), (16, 2), (16, 4), (32, 1), (32, 2), (32, 4), (32, 8),
                  (64, 1), (64, 2), (64, 4), (64, 8), (64, 16)]
TMA_VARIANTS = [(1, 1), (4, 1), (8, 1), (16, 2), (16, 4), (32, 4), (32, 8), (64, 8), (64, 16)]


@pytest.mark.parametrize("kernel,k,tpv", [(2, k, t) for k, t in PLAIN_VARIANTS] + [(1, k, t) for k, t in TMA_VARIANTS])
def test_threads_per_vertex_variants(kernel, k, tpv):
    g, dg = dev_graph("grid64")
    srcs = synth.draw_sources(g, k, 7)
    taus = synth.draw_taus_uniform(k, 300, 3000, 8)
    check_batch(g, dg, srcs, taus, threads_per_vertex=tpv, sweep_kernel=kernel)


@pytest.mark.parametrize("kernel", [1, 2])
def test_both_sweep_kernels_on_grid1k(kernel):
    g, dg = dev_graph("grid1k")
    srcs = synth.draw_sources(g, 64, 31)
    taus = synth.draw_taus_uniform(64, 0, 60000, 32)
    check_batch(g, dg, srcs, taus, want_dist=True, sweep_kernel=kernel)


def test_trace_reports_every_step():
    g, dg = dev_graph("grid1k")
    ws = P.Workspace(dg, 16, record_trace=1)
    ws.submit(synth.draw_sources(g, 16, 3), np.full(16, 20000, np.int32))
    ws.collect()
    steps, ns = ws.trace()
    L = g_levels(dg)
    assert steps.shape[0] == ns.shape[0] == L + 1
    assert np.array_equal(steps[:L, 1], np.arange(L)) and steps[L, 0] == 2
    assert np.all(ns[:L] > 0) and ns[L] >= 0


def g_levels(dg):
    return dg.levels


@pytest.mark.parametrize("fuse", [-1, 1, 64, 100000])
@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("kernel", [1, 2])
def test_fusion_and_cuda_graph(fuse, graph, kernel):
    g, dg = dev_graph("grid64")
    srcs = synth.draw_sources(g, 16, 5)
    taus = synth.draw_taus_uniform(16, 0, 3000, 6)
    check_batch(g, dg, srcs, taus, fuse_width=fuse, use_cuda_graph=graph, sweep_kernel=kernel)


@pytest.mark.parametrize("solo", [-1, 1, 124, 1 << 30])
@pytest.mark.parametrize("graph", [0, 1])
def test_top_block_sizes(solo, graph):
    # -1: no levels in CTA 0 alone; 1 << 30: CTA 0 sweeps the whole hierarchy
    g, dg = dev_graph("grid64")
    srcs = synth.draw_sources(g, 16, 15)
    taus = synth.draw_taus_uniform(16, 0, 3000, 16)
    check_batch(g, dg, srcs, taus, solo_width=solo, use_cuda_graph=graph, sweep_kernel=1, core_vertices=-1)


@pytest.mark.parametrize("solo,fuse", [(-1, -1), (124, -1), (-1, 0), (1 << 30, 0), (124, 1 << 20), (-1, 1 << 20)])
def test_leading_level_phases(solo, fuse):
    # fuse -1: no level-synchronous phase (every level in the chunk schedule);
    # solo -1 with the default fuse width: all narrow levels under grid barriers;
    # fuse 1 << 20: every level grid-synchronous, the widest ones in several
    # passes over the grid's thread groups
    g, dg = dev_graph("grid1k")
    srcs = synth.draw_sources(g, 16, 61)
    taus = synth.draw_taus_uniform(16, 0, 60000, 62)
    check_batch(g, dg, srcs, taus, want_dist=True, solo_width=solo, fuse_width=fuse, sweep_kernel=1,
                core_vertices=-1)


@pytest.mark.parametrize("span", [512, 4096])
def test_chunk_span_limit(span):
    # chunks of sparse levels cut by BFS-rank span: many chunks smaller than
    # the thread groups of a CTA
    g, dg = dev_graph("grid1k")
    srcs = synth.draw_sources(g, 16, 71)
    taus = synth.draw_taus_uniform(16, 0, 60000, 72)
    check_batch(g, dg, srcs, taus, want_dist=True, chunk_span=span, sweep_kernel=1)


@pytest.mark.parametrize("solo", [-1, 124, 4000])
def test_top_block_grid1k(solo):
    g, dg = dev_graph("grid1k")
    srcs = synth.draw_sources(g, 64, 51)
    taus = synth.draw_taus_uniform(64, 0, 60000, 52)
    check_batch(g, dg, srcs, taus, want_dist=True, solo_width=solo, sweep_kernel=1, core_vertices=-1)


@pytest.mark.parametrize("core", [-1, 1, 200, 5000, 0])
@pytest.mark.parametrize("k", [1, 5, 16, 64])
def test_per_lane_core_grid1k(core, k):
    # core 1 / 200 / 5000: the top level blocks within that many vertices are
    # swept per lane in shared memory (1: just the top level), then grid
    # barriers, then chunks; 0: as many as fit; -1: none
    g, dg = dev_graph("grid1k")
    srcs = synth.draw_sources(g, k, 81 + k)
    taus = synth.draw_taus_uniform(k, 0, 60000, 82 + k)
    check_batch(g, dg, srcs, taus, want_dist=True, core_vertices=core, sweep_kernel=1)


@pytest.mark.parametrize("arcs,deps", [(64, 0), (0, 1), (16, 1), (1, 1)])
def test_global_memory_staging_paths(arcs, deps):
    # lower staging limits force the sweep's two global-memory paths: chunks
    # whose arc block exceeds the stage buffer read their arcs from global
    # memory, and dependency lists longer than the held list are checked there
    g, dg = dev_graph("grid1k")
    opts = dict(debug_stage_arcs=arcs, debug_stage_deps=deps, sweep_kernel=1)
    ws = P.Workspace(dg, 16, **opts)
    info = ws.sweep_info()
    ws.free()
    assert info["arc_cap"] == (arcs or 3072) and info["dep_cap"] == (deps or 128)
    if arcs:
        assert info["chunks_over_arc_cap"] > 0
    if deps:
        assert info["chunks_over_dep_cap"] > 0
    srcs = synth.draw_sources(g, 16, 97)
    taus = synth.draw_taus_uniform(16, 0, 60000, 98)
    check_batch(g, dg, srcs, taus, want_dist=True, **opts)


def test_sweep_info_describes_the_phases():
    g, dg = dev_graph("grid1k")
    ws = P.Workspace(dg, 64)
    info = ws.sweep_info()
    ws.free()
    assert info["levels"] == dg.levels
    assert 0 < info["core_levels"] <= info["solo_levels"] <= info["sync_levels"] <= info["levels"]
    assert 0 < info["core_vertices"] <= 53248 and info["chunks"] > 0
    assert info["max_chunk_arcs"] > 0 and info["max_chunk_deps"] > 0


@pytest.mark.parametrize("graph", [0, 1])
def test_per_lane_core_sources_inside_the_core(graph):
    # sources at the top of the hierarchy (their upward labels are all core
    # labels) mixed with ordinary ones, fused and unfused narrow levels
    g, ch = workload("grid1k")
    _, dg = dev_graph("grid1k")
    perm = ch.arrays()["perm"]
    srcs = np.concatenate([perm[[0, 1, 7, 100, 3000, 40000]], synth.draw_sources(g, 10, 91)]).astype(np.int32)
    taus = synth.draw_taus_uniform(len(srcs), 0, 60000, 92)
    for fuse in (0, -1):
        check_batch(g, dg, srcs, taus, want_dist=True, sweep_kernel=1, fuse_width=fuse, use_cuda_graph=graph)


@pytest.mark.parametrize("k", [1, 3, 64])
def test_per_lane_core_covers_the_whole_graph(k):
    # grid64 (4,096 vertices) fits the core: every level is swept per lane and
    # the chunk schedule is empty
    g, dg = dev_graph("grid64")
    srcs = synth.draw_sources(g, k, 95)
    taus = synth.draw_taus_uniform(k, 0, 3000, 96)
    check_batch(g, dg, srcs, taus, want_dist=True, sweep_kernel=1)
    check_batch(g, dg, srcs, taus, want_dist=False, sweep_kernel=1, use_cuda_graph=1)


def test_duplicate_sources_and_extreme_limits():
    g, dg = dev_graph("grid64")
    s = synth.draw_sources(g, 1, 3)[0]
    tmax = 0x7FFFFFFE - int(g.weight.max())
    srcs = np.array([s, s, s, s, s, 0, 0, 17], np.int32)
    taus = np.array([0, 1500, 1500, 10 ** 6, tmax, 0, tmax, 1], np.int32)
    check_batch(g, dg, srcs, taus)


def test_grid1k_single_and_batched():
    g, dg = dev_graph("grid1k")
    srcs = synth.draw_sources(g, 6, 77)
    for tau in (2000, 10000, 50000):
        for s in srcs[:3]:
            check_batch(g, dg, np.array([s], np.int32), np.array([tau], np.int32), want_dist=False)
    taus = synth.draw_taus_uniform(16, 2000, 50000, 78)
    check_batch(g, dg, synth.draw_sources(g, 16, 79), taus, want_dist=True)


def test_device_buffers_and_workspaces():
    g, dg = dev_graph("grid64")
    k = 16
    srcs = synth.draw_sources(g, k, 41)
    taus = synth.draw_taus_uniform(k, 100, 3000, 42)
    want_off, want_arcs, _ = oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs, taus)
    ds = torch.from_numpy(srcs).cuda()
    dt = torch.from_numpy(taus).cuda()
    o_off = torch.zeros(k + 1, dtype=torch.int64, device="cuda")
    o_arcs = torch.zeros(int(want_off[-1]) + 5, dtype=torch.int32, device="cuda")
    P.iso_query(dg, ds, dt, out_offsets=o_off, out_arcs=o_arcs)
    assert np.array_equal(o_off.cpu().numpy(), want_off)
    assert np.array_equal(o_arcs.cpu().numpy()[:want_off[-1]], want_arcs)
    # two workspaces on two streams, interleaved
    w1 = P.Workspace(dg, 16)
    w2 = P.Workspace(dg, 64, use_cuda_graph=1)
    srcs2 = synth.draw_sources(g, 40, 43)
    taus2 = synth.draw_taus_uniform(40, 0, 5000, 44)
    w1.submit(ds, dt)
    w2.submit(srcs2, taus2)
    off1, arcs1, _ = w1.collect()
    off2, arcs2, _ = w2.collect()
    assert np.array_equal(off1, want_off) and np.array_equal(arcs1, want_arcs)
    e_off, e_arcs, _ = oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs2, taus2)
    assert np.array_equal(off2, e_off) and np.array_equal(arcs2, e_arcs)
    t = w2.timings()
    assert t["sweep"] > 0


def test_overflow_reports_needed_offsets():
    g, dg = dev_graph("grid64")
    srcs = synth.draw_sources(g, 4, 1)
    taus = np.full(4, 1500, np.int32)
    want_off, _, _ = oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs, taus)
    off = np.zeros(5, np.int64)
    small = np.zeros(3, np.int32)
    with pytest.raises(P.IsoError) as e:
        P.iso_query(dg, srcs, taus, out_offsets=off, out_arcs=small, cap=3)
    assert e.value.code == P.ISO_E_OVERFLOW
    assert np.array_equal(off, want_off)


@pytest.mark.parametrize("k", [1, 8, 64])
def test_failed_batch_leaves_workspace_clean(k):
    # one invalid source in device memory: the batch fails on the device after
    # the other lanes' upward searches ran; the next batch on the same
    # workspace must not see anything of it
    g, dg = dev_graph("grid1k")
    ws = P.Workspace(dg, k, use_cuda_graph=1)
    srcs = synth.draw_sources(g, k, 91)
    bad = srcs.copy()
    bad[k // 2] = g.n + 3
    taus = synth.draw_taus_uniform(k, 2000, 60000, 92)
    ws.submit(torch.from_numpy(bad).cuda(), torch.from_numpy(taus).cuda())
    with pytest.raises(P.IsoError) as e:
        ws.collect()
    assert e.value.code == P.ISO_E_INVAL
    for seed in (93, 94):
        s2 = synth.draw_sources(g, k, seed)
        ws.submit(s2, taus)
        off, arcs, _ = ws.collect()
        o_off, o_arcs, _ = oracle.query_batch(g.n, g.tail, g.head, g.weight, s2, taus, threads=8)
        assert np.array_equal(off, o_off) and np.array_equal(arcs, o_arcs)
    ws.free()


def test_argument_errors_and_recovery():
    g, dg = dev_graph("grid64")
    for s, t in [(-1, 10), (g.n, 10), (0, -1), (0, 0x7FFFFFFF)]:
        with pytest.raises(P.IsoError) as e:
            P.iso_query(dg, np.array([s], np.int32), np.array([t], np.int32))
        assert e.value.code == P.ISO_E_INVAL
    # invalid values in device memory are caught by the first kernel
    with pytest.raises(P.IsoError) as e:
        P.iso_query(dg, torch.tensor([g.n + 5], dtype=torch.int32, device="cuda"),
                    torch.tensor([10], dtype=torch.int32, device="cuda"))
    assert e.value.code == P.ISO_E_INVAL
    check_batch(g, dg, synth.draw_sources(g, 4, 9), np.full(4, 900, np.int32))


@pytest.mark.parametrize("kernel,core,graph", [(1, 0, "grid64"), (1, -1, "grid64"), (1, 0, "grid1k"),
                                                (1, -1, "grid1k"), (2, 0, "grid64")])
def test_barrier_timeout_is_reported_and_context_survives(kernel, core, graph):
    # every device-side wait of the sweep gives up after the timeout: the grid
    # barrier after the per-lane core (core 0; on grid64 the core is the whole
    # graph), the leading levels' barriers and the chunks' dependency waits
    g, dg = dev_graph(graph)
    srcs = synth.draw_sources(g, 4, 2)
    taus = np.full(4, 1000, np.int32)
    with pytest.raises(P.IsoError) as e:
        P.iso_query(dg, srcs, taus, debug_barrier_extra=1, barrier_timeout_ns=20_000_000, sweep_kernel=kernel,
                    core_vertices=core)
    assert e.value.code == P.ISO_E_TIMEOUT
    torch.cuda.synchronize()
    check_batch(g, dg, srcs, taus, core_vertices=core, sweep_kernel=kernel)


def _unpack(bits, n):
    return np.unpackbits(np.ascontiguousarray(bits).view(np.uint8), axis=1, bitorder="little")[:, :n].astype(bool)


@pytest.mark.parametrize("k", [1, 13, 64])
def test_vertices_in_range_bitsets(k):
    # the other output Section 3 names: per query, the set of vertices in range
    g, dg = dev_graph("grid1k")
    srcs = synth.draw_sources(g, k, 101 + k)
    taus = synth.draw_taus_uniform(k, 0, 60000, 102 + k)
    ws = P.Workspace(dg, k)
    with pytest.raises(P.IsoError):
        ws.collect_range()                       # nothing collected yet
    ws.submit(srcs, taus)
    ws.collect()
    bits = ws.collect_range()
    _, _, o_dist = oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs, taus, want_dist=True, threads=8)
    assert np.array_equal(_unpack(bits, g.n), o_dist != INF)
    # into a device buffer with a longer row pitch (the extra words stay untouched)
    words = (g.n + 31) // 32
    dbuf = torch.full((k, words + 5), -1, dtype=torch.int32, device="cuda")
    ws.collect_range(dbuf)
    got = dbuf.cpu().numpy()
    assert np.all(got[:, words:] == -1)
    assert np.array_equal(got[:, :words].view(np.uint32), bits)
    ws.free()


def test_chained_batches_on_two_workspaces():
    # iso_submit_after: each batch starts after the previous batch's sweep on
    # the other workspace; results equal those of independent queries
    g, dg = dev_graph("grid1k")
    wss = [P.Workspace(dg, 16, use_cuda_graph=1, stream=torch.cuda.Stream()) for _ in range(2)]
    batches = [(synth.draw_sources(g, 16, 120 + b), synth.draw_taus_uniform(16, 0, 60000, 140 + b)) for b in range(6)]
    got, prev = {}, None
    for b, (s, t) in enumerate(batches):
        ws = wss[b % 2]
        if b >= 2:
            got[b - 2] = ws.collect()
        ws.submit(s, t, after=prev)
        prev = ws
    got[4] = wss[0].collect()
    got[5] = wss[1].collect()
    for b, (s, t) in enumerate(batches):
        off, arcs, _ = P.iso_query(dg, s, t)
        assert np.array_equal(got[b][0], off) and np.array_equal(got[b][1], arcs), b
    for ws in wss:
        ws.free()


_LM = {}


def lm_graph(name):
    """A device graph of the workload with landmarks for restricted sweeps."""
    if name not in _LM:
        g, ch = workload(name)
        dg = P.iso_upload_graph(ch)
        dg.add_landmarks(ch, 8)
        _LM[name] = (g, dg)
    return _LM[name]


def test_landmarks_replaced_only_without_restricted_workspaces():
    # a workspace with restricted sweeps keeps using the landmarks it was made
    # with (its chunk bounds, its captured CUDA graph): replacing them is refused
    # while it lives and allowed once it is freed; iso_query's own restricted
    # workspace is dropped and made again
    g, ch = workload("grid1k")
    dg = P.iso_upload_graph(ch)
    dg.add_landmarks(ch, 4)
    srcs = synth.draw_sources(g, 3, 195)
    taus = np.array([2000, 5000, 9000], np.int32)
    check_batch(g, dg, srcs, taus, restrict_sweep=1)
    ws = P.Workspace(dg, 3, restrict_sweep=1, use_cuda_graph=1)
    with pytest.raises(P.IsoError) as e:
        dg.add_landmarks(ch, 8)
    assert e.value.code == P.ISO_E_INVAL
    ws.submit(srcs, taus)
    off, arcs, _ = ws.collect()
    o_off, o_arcs, _ = oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs, taus, threads=8)
    assert np.array_equal(off, o_off) and np.array_equal(arcs, o_arcs)
    ws.free()
    dg.add_landmarks(ch, 8)
    check_batch(g, dg, srcs, taus, restrict_sweep=1)
    dg.free()


@pytest.mark.parametrize("k,tmax", [(1, 3000), (1, 20000), (3, 8000), (16, 5000), (64, 60000)])
def test_restricted_sweep(k, tmax):
    # chunks that landmark bounds show out of range for every lane are skipped;
    # the answers stay exact (lists and distances)
    g, dg = lm_graph("grid1k")
    srcs = synth.draw_sources(g, k, 150 + k)
    taus = synth.draw_taus_uniform(k, 0, tmax, 160 + k)
    ws = P.Workspace(dg, k, restrict_sweep=1, use_cuda_graph=1)
    ws.submit(srcs, taus, want_dist=True)
    off, arcs, dist = ws.collect(want_dist=True)
    skipped = ws.skipped_chunks()
    chunks = ws.sweep_info()["chunks"]
    ws.free()
    o_off, o_arcs, o_dist = oracle.query_batch(g.n, g.tail, g.head, g.weight, srcs, taus, want_dist=True, threads=8)
    assert np.array_equal(off, o_off) and np.array_equal(arcs, o_arcs) and np.array_equal(dist, o_dist)
    if k <= 3 and tmax <= 8000:
        assert skipped > chunks // 4        # few sources, small limits: much of the map is skipped
    assert 0 <= skipped <= chunks


def test_restricted_sweep_errors_and_reuse():
    g, dg = dev_graph("grid64")               # no landmarks on this graph
    with pytest.raises(P.IsoError):
        P.Workspace(dg, 4, restrict_sweep=1)
    g, dg = lm_graph("grid1k")
    srcs = synth.draw_sources(g, 16, 171)
    taus = synth.draw_taus_uniform(16, 0, 6000, 172)
    # two batches in a row on one workspace, then without restriction: all equal
    ws = P.Workspace(dg, 16, restrict_sweep=1)
    for _ in range(2):
        ws.submit(srcs, taus)
        off, arcs, _ = ws.collect()
    ws.free()
    o2, a2, _ = P.iso_query(dg, srcs, taus)
    assert np.array_equal(off, o2) and np.array_equal(arcs, a2)


def test_large_isochrone_edge_lists():
    # 70,000 parallel arcs cross the isochrone of one query: more than the
    # sort's four shared-memory parts hold, so the lane is sorted in global
    # memory by one CTA
    rng = np.random.default_rng(5)
    par = 70_000
    tail = np.concatenate([[0, 2, 3], np.ones(par, np.int64)]).astype(np.int32)
    head = np.concatenate([[1, 3, 2], np.full(par, 2, np.int64)]).astype(np.int32)
    w = np.concatenate([[1, 1, 1], rng.integers(10, 20, size=par)]).astype(np.int32)
    order = rng.permutation(tail.shape[0])
    tail, head, w = tail[order], head[order], w[order]
    n = 4
    dg = P.iso_upload_graph(P.iso_build_ch(n, tail, head, w))
    srcs = np.array([0, 0, 3], np.int32)
    taus = np.array([5, 12, 30], np.int32)
    off, arcs, _ = P.iso_query(dg, srcs, taus)
    o_off, o_arcs, _ = oracle.query_batch(n, tail, head, w, srcs, taus)
    assert np.array_equal(off, o_off) and np.array_equal(arcs, o_arcs)
    assert off[1] - off[0] == par


def test_clustered_isochrone_edge_ids():
    # the crossing arcs have consecutive ids among 2^18 arcs, so the sort's
    # buckets get hundreds of ids each and are ranked by the whole CTA
    leaves = 1000
    pad = 1 << 18
    star = np.arange(1, leaves + 1, dtype=np.int32)
    sink = 2 * leaves + 1
    tail = np.concatenate([np.zeros(leaves, np.int32), star, np.full(pad, sink, np.int32)])
    head = np.concatenate([star, star + leaves, np.full(pad, sink, np.int32)])
    w = np.concatenate([np.ones(leaves, np.int32), np.full(leaves, 10, np.int32), np.ones(pad, np.int32)])
    n = sink + 1
    ch = P.iso_build_ch(n, tail, head, w)
    dg = P.iso_upload_graph(ch)
    srcs = np.array([0, 0], np.int32)
    taus = np.array([5, 12], np.int32)
    off, arcs, _ = P.iso_query(dg, srcs, taus)
    o_off, o_arcs, _ = oracle.query_batch(n, tail, head, w, srcs, taus)
    assert np.array_equal(off, o_off) and np.array_equal(arcs, o_arcs)
    assert off[1] == leaves and np.array_equal(arcs[:leaves], np.arange(leaves, 2 * leaves))
