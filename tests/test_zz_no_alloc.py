"""The allocation-free entry point (iso_query_noalloc) against iso_query.

Callers that cannot allocate device memory while answering a query (a fully
reserved device, a thread that must not wait on allocator locks) use
iso_query_noalloc, which runs on a fixed static device array.  This file is
collected last on purpose.  Every check calls the C ABI and compares with the
existing entry point bit for bit (the tolerance of all parity tests here:
integer results, exact), on two calls in a row so the second call runs on the
scratch the first one left behind."""

import ctypes

import numpy as np
import pytest

import paper_1512_09090_gb300 as P
from paper_1512_09090_gb300 import synth
from paper_1512_09090_gb300._lib import lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _graph(name):
    g = synth.workload_graph(name)
    return g, P.iso_upload_graph(P.iso_build_ch(g.n, g.tail, g.head, g.weight))


def _noalloc(dg, srcs, taus, cap):
    k = len(srcs)
    off = np.zeros(k + 1, np.int64)
    arcs = np.zeros(max(cap, 1), np.int32)
    srcs = np.ascontiguousarray(srcs, np.int32)
    taus = np.ascontiguousarray(taus, np.int32)
    rc = lib().iso_query_noalloc(dg.handle, k, srcs.ctypes.data, taus.ctypes.data, off.ctypes.data,
                                 arcs.ctypes.data, cap, dg.stream.cuda_stream)
    return rc, off, arcs[:off[-1]]


def test_noalloc_matches_iso_query_twice():
    g, dg = _graph("grid1k")
    for call, (k, seed) in enumerate([(4, 11), (3, 12), (1, 13)]):
        srcs = synth.draw_sources(g, k, seed)
        taus = synth.draw_taus_uniform(k, 2000, 20000, seed + 100)
        want_off, want_arcs, _ = P.iso_query(dg, srcs, taus)
        rc, off, arcs = _noalloc(dg, srcs, taus, int(want_off[-1]) + 10)
        assert rc == P.ISO_OK, lib().iso_last_error().decode()
        assert np.array_equal(off, want_off), call
        assert np.array_equal(arcs, want_arcs), call


def test_noalloc_device_buffers_and_limits():
    g, dg = _graph("grid64")
    srcs = synth.draw_sources(g, 4, 5)
    taus = synth.draw_taus_uniform(4, 100, 3000, 6)
    want_off, want_arcs, _ = P.iso_query(dg, srcs, taus)
    for _ in range(2):
        d_off = torch.zeros(5, dtype=torch.int64, device="cuda")
        d_arcs = torch.zeros(int(want_off[-1]) + 1, dtype=torch.int32, device="cuda")
        P._lib.iso_query_noalloc(dg, torch.from_numpy(srcs).cuda(), torch.from_numpy(taus).cuda(), d_off, d_arcs)
        assert np.array_equal(d_off.cpu().numpy(), want_off)
        assert np.array_equal(d_arcs.cpu().numpy()[:want_off[-1]], want_arcs)
    # beyond the stated limits: a clear error, nothing launched
    rc, _, _ = _noalloc(dg, np.zeros(5, np.int32), np.zeros(5, np.int32), 10)
    assert rc == P.ISO_E_INVAL and "outside 0..4" in lib().iso_last_error().decode()
    n = (1 << 20) + 1
    big = P.iso_upload_graph(P.iso_build_ch(n, np.array([0, 1], np.int32), np.array([1, 0], np.int32),
                                            np.array([3, 3], np.int32)))
    rc, _, _ = _noalloc(big, np.zeros(1, np.int32), np.ones(1, np.int32), 10)
    assert rc == P.ISO_E_INVAL and "limit" in lib().iso_last_error().decode()
    # overflow of the caller's buffer reports the needed offsets
    rc, off, _ = _noalloc(dg, srcs, taus, 2)
    assert rc == P.ISO_E_OVERFLOW and np.array_equal(off, want_off)
