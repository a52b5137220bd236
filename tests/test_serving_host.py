"""Host logic of the continuous-batching server (serving.py) on CPU, with fake
workspaces in place of device ones: requests are answered by batches of at
most `lanes`, every request receives its own answer, a failing batch fails
exactly its requests, close() ends the workers, and the pool grows only
while (fake) device memory has room for another workspace."""

import threading
import time

import numpy as np
import pytest

from paper_1512_09090_gb300 import serving


class FakeWorkspace:
    """Answers request (s, tau) with the arc list [s, s + tau] after a short delay."""

    def __init__(self, fail_on=None, delay_s=0.002):
        self.fail_on = fail_on
        self.delay_s = delay_s
        self.batches = []
        self._pending = None

    def submit(self, sources, taus):
        assert self._pending is None, "submit twice without collect"
        self._pending = (np.asarray(sources).copy(), np.asarray(taus).copy())

    def collect(self):
        s, t = self._pending
        self._pending = None
        time.sleep(self.delay_s)
        self.batches.append(len(s))
        if self.fail_on is not None and self.fail_on in s:
            raise RuntimeError("device failure")
        off = np.zeros(len(s) + 1, np.int64)
        arcs = []
        for i in range(len(s)):
            arcs += [int(s[i]), int(s[i] + t[i])]
            off[i + 1] = len(arcs)
        return off, np.array(arcs, np.int32), None


def test_every_request_gets_its_own_answer_in_batches_of_at_most_lanes():
    wss = [FakeWorkspace(), FakeWorkspace()]
    lanes = 8
    with serving.IsoServer.over_workspaces(wss, lanes) as srv:
        futs = [srv.submit(s, 10 * s) for s in range(200)]
        res = [f.result(timeout=30) for f in futs]
    for s, r in enumerate(res):
        assert r.arcs.tolist() == [s, 11 * s]
        assert r.t_done >= r.t_arrival
    sizes = [b for ws in wss for b in ws.batches]
    assert sum(sizes) == 200 and max(sizes) <= lanes
    assert len({r.batch for r in res}) == len(sizes)


def test_a_failing_batch_fails_exactly_its_requests():
    ws = FakeWorkspace(fail_on=13, delay_s=0.0)
    with serving.IsoServer.over_workspaces([ws], 4) as srv:
        f_bad = srv.submit(13, 1)
        with pytest.raises(RuntimeError):
            f_bad.result(timeout=30)
        f_ok = srv.submit(5, 1)
        assert f_ok.result(timeout=30).arcs.tolist() == [5, 6]


def test_poisson_replay_and_summary():
    ws = FakeWorkspace(delay_s=0.001)
    with serving.IsoServer.over_workspaces([ws], 16) as srv:
        arr = np.linspace(0.0, 0.05, 40)
        res, wall = serving.run_poisson(srv, np.arange(40), np.full(40, 3), arr)
    assert len(res) == 40 and wall >= 0.05
    summ = serving.latency_summary(res)
    assert 0 <= summ["p50_ms"] <= summ["p99_ms"] and summ["batches"] >= 1


def test_close_ends_the_workers():
    srv = serving.IsoServer.over_workspaces([FakeWorkspace(), FakeWorkspace(), FakeWorkspace()], 4)
    srv.close()
    assert all(not t.is_alive() for t in srv._threads)
    assert threading.active_count() >= 1


class FakeDevWorkspace(FakeWorkspace):
    """A fake workspace made the way the server makes device ones: it takes
    device memory from a fake pool, is warmed by a batch, and accepts `after`
    (batches chained to the previous batch's sweep)."""
    pool = None

    def __init__(self, g, lanes, **opts):
        super().__init__(delay_s=0.02)
        FakeDevWorkspace.pool["free"] -= FakeDevWorkspace.pool["size"]
        FakeDevWorkspace.pool["made"] += 1

    def submit(self, sources, taus, after=None):
        super().submit(sources, taus)

    def free(self):
        FakeDevWorkspace.pool["free"] += FakeDevWorkspace.pool["size"]


@pytest.fixture
def fake_device(monkeypatch):
    torch = pytest.importorskip("torch")
    pool = {"free": 0, "size": 1 << 30, "made": 0}
    FakeDevWorkspace.pool = pool
    monkeypatch.setattr(serving._lib, "Workspace", FakeDevWorkspace)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a: (pool["free"], 1 << 40))
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    return pool


def _flood(srv, n):
    reqs = [srv.submit(i, 5) for i in range(n)]
    for i, r in enumerate(reqs):
        assert r.result(timeout=60).arcs.tolist() == [i, i + 5]


def test_pool_grows_while_device_memory_allows(fake_device):
    # requests wait behind the one busy workspace: the pool grows (up to
    # max_workspaces), each new workspace warmed before it takes requests
    fake_device["free"] = 100 << 30
    with serving.IsoServer(object(), lanes=4, workspaces=1, max_workspaces=3) as srv:
        assert srv.bytes_per_workspace == 1 << 30      # measured from the first workspace
        _flood(srv, 200)
        assert srv.grown >= 1 and srv.refused_growth == 0
        assert len(srv.workspaces) == 1 + srv.grown <= 3
    assert fake_device["made"] == 1 + srv.grown


def test_growth_refused_when_device_memory_is_short(fake_device):
    # room for the first workspace only: after it, half of the free memory
    # (0.25 GB) does not cover another (1 GB), so every growth is refused and
    # the one workspace answers everything
    fake_device["free"] = (3 << 30) // 2
    with serving.IsoServer(object(), lanes=4, workspaces=1, max_workspaces=3, memory_fraction=0.5) as srv:
        _flood(srv, 120)
        assert srv.grown == 0 and srv.refused_growth >= 1
        assert len(srv.workspaces) == 1
    assert fake_device["made"] == 1
