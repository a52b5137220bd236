"""Continuous batching: every request's isochrone inside a mixed batch equals
the isochrone of that request alone (integer results, compared exactly), and
requests that arrive while batches are on the device are admitted into later
batches of several concurrently used workspaces."""

import numpy as np
import pytest

import oracle
import paper_1512_09090_gb300 as P
from paper_1512_09090_gb300 import serving, synth

from helpers import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def test_results_alone_equal_results_in_the_mix():
    g, ch = workload("grid1k")
    dg = P.iso_upload_graph(ch)
    count = 300
    srcs = synth.draw_sources(g, count, 71)
    taus = synth.draw_taus_loguniform(count, 600, 72000, 72)
    arrivals = synth.poisson_arrivals(count, 20000.0, 73)
    with serving.IsoServer(dg, lanes=16, workspaces=3) as srv:
        res, wall = serving.run_poisson(srv, srcs, taus, arrivals)
    batches = {}
    for r in res:
        batches[r.batch] = batches.get(r.batch, 0) + 1
    assert len(batches) > 1 and max(batches.values()) > 1        # several batches, mixed ones
    alone_off, alone_arcs, _ = P.iso_query(dg, srcs, taus)        # the same requests, batched differently
    for i, r in enumerate(res):
        assert np.array_equal(r.arcs, alone_arcs[alone_off[i]:alone_off[i + 1]])
    for i in range(0, count, 37):                                 # and a few truly alone, plus the oracle
        o, a, _ = P.iso_query(dg, srcs[i:i + 1], taus[i:i + 1])
        assert np.array_equal(res[i].arcs, a)
        want, _ = oracle.isochrone(g.n, g.tail, g.head, g.weight, int(srcs[i]), int(taus[i]))
        assert np.array_equal(res[i].arcs, want)
    s = serving.latency_summary(res)
    assert s["p99_ms"] >= s["p50_ms"] > 0
