"""Host-side checks of the C ABI (no GPU): exported symbols, the contraction
hierarchy (structure, and a CPU PHAST over it against the oracle), the CH file
format, and argument validation."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1512_09090_gb300 as P
from paper_1512_09090_gb300 import synth
from paper_1512_09090_gb300._lib import lib, IsoError

from helpers import INF, arcs_of, cpu_phast, workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "iso.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"\b(iso_[a-z_0-9]+)\s*\(", hdr))
    assert {"iso_build_ch", "iso_upload_graph", "iso_query"} <= declared
    L = lib()
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert L.iso_version().decode().startswith("iso-gb300")


def check_structure(ch, n):
    A = ch.arrays()
    st = ch.stats()
    L = st["levels"]
    lo = A["level_off"]
    assert lo[0] == 0 and lo[-1] == n and np.all(np.diff(lo) >= 0)
    level_of = np.empty(n, dtype=np.int64)
    for j in range(L):
        level_of[lo[j]:lo[j + 1]] = L - 1 - j
    assert np.array_equal(np.sort(A["perm"]), np.arange(n))
    assert np.array_equal(A["pos"][A["perm"]], np.arange(n))
    heads = np.repeat(np.arange(n), np.diff(A["down_off"]))
    # every downward arc comes from a strictly higher level, earlier in the sweep
    assert np.all(level_of[A["down_src"]] > level_of[heads])
    assert np.all(A["down_src"] < heads)
    tails = np.repeat(np.arange(n), np.diff(A["up_off"]))
    assert np.all(level_of[A["up_dst"]] > level_of[tails])
    assert np.all(A["down_w"] >= 0) and np.all(A["up_w"] >= 0)
    assert np.array_equal(np.sort(A["orig_id"]), np.arange(st["m"]))
    assert np.array_equal(np.sort(A["bfs"]), np.arange(n))
    # within a level, sweep order follows the BFS rank
    for j in range(L):
        assert np.all(np.diff(A["bfs"][lo[j]:lo[j + 1]]) > 0)
    return A


def test_ch_golden_cases(golden_cases):
    for case in golden_cases:
        n, t, h, w = arcs_of(case)
        ch = P.iso_build_ch(n, t, h, w)
        A = check_structure(ch, n)
        for q in case["queries"]:
            d = cpu_phast(A, q["s"], q["tau"])
            want = oracle.tau_dijkstra(n, t, h, w, q["s"], q["tau"])
            assert np.array_equal(d, want.astype(np.int64)), (case["name"], q)


@pytest.mark.parametrize("seed", range(25))
def test_ch_random_small(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 40))
    g = synth.random_graph(n, int(rng.integers(0, 4 * n)), wmin=0, wmax=30, seed=seed)
    ch = P.iso_build_ch(g.n, g.tail, g.head, g.weight, threads=int(rng.integers(1, 4)))
    A = check_structure(ch, n)
    for s in range(0, n, max(1, n // 5)):
        for tau in (0, 15, 60, 10 ** 6):
            want = oracle.tau_dijkstra(n, g.tail, g.head, g.weight, s, tau)
            assert np.array_equal(cpu_phast(A, s, tau), want.astype(np.int64))


def test_ch_grid64_phast_matches_oracle():
    g, ch = workload("grid64")
    A = check_structure(ch, g.n)
    for s in synth.draw_sources(g, 8, 21):
        for tau in (0, 400, 1500, 6000):
            want = oracle.tau_dijkstra(g.n, g.tail, g.head, g.weight, s, tau)
            assert np.array_equal(cpu_phast(A, s, tau), want.astype(np.int64))


def test_ch_parallel_builds_agree_on_distances():
    g = synth.grid_road_graph(50, 60, highways=((8, 4),), seed=9)
    A1 = P.iso_build_ch(g.n, g.tail, g.head, g.weight, threads=1).arrays()
    A4 = P.iso_build_ch(g.n, g.tail, g.head, g.weight, threads=4).arrays()
    for s in synth.draw_sources(g, 4, 2):
        assert np.array_equal(cpu_phast(A1, s, 3000), cpu_phast(A4, s, 3000))


def test_ch_save_load_roundtrip(tmp_path):
    g, ch = workload("grid64")
    path = str(tmp_path / "g.ch")
    ch.save(path)
    ch2 = P.iso_load_ch(path)
    A, B = ch.arrays(), ch2.arrays()
    assert ch.stats()["levels"] == ch2.stats()["levels"]
    for k in A:
        assert np.array_equal(A[k], B[k]), k
    # a truncated or foreign file is rejected
    raw = open(path, "rb").read()
    open(path, "wb").write(raw[:len(raw) // 2])
    with pytest.raises(IsoError) as e:
        P.iso_load_ch(path)
    assert e.value.code == P.ISO_E_IO
    open(path, "wb").write(b"not a ch file at all" * 10)
    with pytest.raises(IsoError):
        P.iso_load_ch(path)


def _corrupt_and_load(path, raw, offset, value):
    b = bytearray(raw)
    b[offset:offset + 4] = np.array([value], np.int32).tobytes()
    open(path, "wb").write(bytes(b))
    with pytest.raises(IsoError) as e:
        P.iso_load_ch(path)
    return e.value.code


def test_load_rejects_well_formed_but_inconsistent_files(tmp_path):
    # file layout: 8-byte magic, 4 int32 + 4 int64 header, perm[n], bfs[n],
    # level_off[L+1] (int32), down_off[n+1] (int64), down_src[m_down], ...
    g, ch = workload("grid64")
    path = str(tmp_path / "g.ch")
    ch.save(path)
    raw = open(path, "rb").read()
    A = ch.arrays()
    n, L = g.n, len(A["level_off"]) - 1
    bfs_at = 56 + 4 * n
    # BFS ranks that are not a permutation
    assert _corrupt_and_load(path, raw, bfs_at + 4, int(A["bfs"][0])) == P.ISO_E_IO
    # a downward arc from a vertex of the lowest level
    src_at = bfs_at + 4 * n + 4 * (L + 1) + 8 * (n + 1)
    assert _corrupt_and_load(path, raw, src_at, n - 1) == P.ISO_E_IO
    # the unmodified file still loads
    open(path, "wb").write(raw)
    assert P.iso_load_ch(path).stats()["n"] == n


def test_build_rejects_bad_input():
    t = np.array([0, 1], np.int32); h = np.array([1, 2], np.int32); w = np.array([1, 1], np.int32)
    for args in [(0, t, h, w), (2, t, h, w), (3, t, h, np.array([1, -1], np.int32)),
                 (3, t, h, np.array([1, 1 << 30], np.int32)), (3, np.array([-1, 0], np.int32), h, w)]:
        with pytest.raises(IsoError) as e:
            P.iso_build_ch(*args)
        assert e.value.code == P.ISO_E_INVAL
    assert "outside" in lib().iso_last_error().decode() or lib().iso_last_error()


def test_query_without_device_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g, ch = workload("grid64")
    out = ctypes.c_void_p()
    rc = lib().iso_upload_graph(ch.handle, None, None, ctypes.byref(out))
    assert rc == P.ISO_E_NODEV
    assert not out.value


def test_every_entry_point_rejects_null_handles():
    # no device needed: each call with NULL handles returns its error (or -1)
    # and sets its own message; the free calls accept NULL
    N = None
    calls = {
        "iso_build_ch": ((3, 0, N, N, N, N, N), P.ISO_E_INVAL),
        "iso_ch_info": ((N, N), P.ISO_E_INVAL),
        "iso_ch_view_arrays": ((N, N), P.ISO_E_INVAL),
        "iso_ch_sweep_position": ((N, 0), -1),
        "iso_save_ch": ((N, b"unused.ch"), P.ISO_E_INVAL),
        "iso_load_ch": ((N, N), P.ISO_E_INVAL),
        "iso_ch_landmarks": ((N, 8, N, N, N), P.ISO_E_INVAL),
        "iso_upload_graph": ((N, N, N, N), P.ISO_E_INVAL),
        "iso_graph_add_landmarks": ((N, N, 8), P.ISO_E_INVAL),
        "iso_query": ((N, 1, N, N, N, N, 0, N, N, N), P.ISO_E_INVAL),
        "iso_query_noalloc": ((N, 1, N, N, N, N, 0, N), P.ISO_E_INVAL),
        "iso_workspace_create": ((N, 64, N, N, N), P.ISO_E_INVAL),
        "iso_submit": ((N, 1, N, N, 0, N), P.ISO_E_INVAL),
        "iso_submit_after": ((N, N, 1, N, N, 0, N), P.ISO_E_INVAL),
        "iso_collect": ((N, N, N, 0, N), P.ISO_E_INVAL),
        "iso_collect_range": ((N, N, 0), P.ISO_E_INVAL),
        "iso_workspace_trace": ((N, N, N, 0), -1),
        "iso_workspace_timings": ((N, N), P.ISO_E_INVAL),
        "iso_workspace_sweep_info": ((N, N), P.ISO_E_INVAL),
        "iso_workspace_skipped_chunks": ((N, N), P.ISO_E_INVAL),
    }
    L = lib()
    for name, (args, want) in calls.items():
        assert getattr(L, name)(*args) == want, name
        msg = L.iso_last_error().decode()
        assert msg.startswith(name), (name, msg)
    for name in ("iso_free_ch", "iso_free_graph", "iso_free_workspace"):
        getattr(L, name)(None)
