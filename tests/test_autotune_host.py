"""Host test of the autotuner's search (paper_1512_09090_gb300/autotune.py).

The timing of a candidate is replaced by a score with a known best point, and
the device query by a fixed SM count, so the coordinate descent, the axes it
searches, the handling of failing candidates, the time budget and the cache
run without a GPU."""

import json
import types

import pytest

torch = pytest.importorskip("torch")

from paper_1512_09090_gb300 import _lib, autotune

SMS = 152


class FakeGraph:
    def __init__(self, landmarks=0):
        self.device = 0
        self.landmarks = landmarks


@pytest.fixture
def fake_device(monkeypatch):
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: types.SimpleNamespace(multi_processor_count=SMS))
    monkeypatch.setattr(autotune, "graph_key", lambda g: f"fake-lm{g.landmarks}")


def scorer(best, fail=()):
    """A _time_config stand-in: queries/s peaks at `best` (per axis, separable);
    options in `fail` raise IsoError as an unsupported candidate does."""
    calls = []

    def time_config(g, lanes, sources, taus, opts, reps):
        calls.append((lanes, dict(opts)))
        for k, v in fail:
            if opts.get(k) == v:
                raise _lib.IsoError(_lib.ISO_E_INVAL, "unsupported")
        q = 10000.0 + 100.0 * lanes
        for k, v in best.items():
            q += 500.0 if opts.get(k, 0) == v else 0.0
        return q
    return time_config, calls


def test_descent_finds_the_best_value_of_every_axis(fake_device, monkeypatch):
    best = {"threads_per_vertex": 16, "schedule_delay": 4 * SMS, "core_vertices": 20000, "chunk_span": 10000}
    tc, calls = scorer(best)
    monkeypatch.setattr(autotune, "_time_config", tc)
    r = autotune.tune(FakeGraph(), [0] * 512, [0] * 512, lanes_choices=(64,), budget_s=60.0)
    for k, v in best.items():
        assert r[k] == v, (k, r)
    assert r["lanes"] == 64
    # options left at the library's default are not listed
    assert "fuse_width" not in r and "solo_width" not in r and "fused_emission" not in r
    assert r["axes"] == [a for a, _ in autotune.axes_for(64, SMS)]
    assert "restrict_sweep" not in r["axes"]          # the graph has no landmarks
    assert len(r["tried"]) == len({(c[0], tuple(sorted(c[1].items()))) for c in calls})  # each candidate once


def test_lanes_choice_and_failing_candidates(fake_device, monkeypatch):
    tc, _ = scorer({"threads_per_vertex": 4}, fail=(("threads_per_vertex", 4),))
    monkeypatch.setattr(autotune, "_time_config", tc)
    r = autotune.tune(FakeGraph(), [0] * 512, [0] * 512, lanes_choices=(16, 32, 64), budget_s=60.0)
    assert r["lanes"] == 64                           # the scorer favours more lanes
    assert r.get("threads_per_vertex", 0) != 4        # a candidate that failed is never chosen
    assert any(t["qps"] == -1.0 for t in r["tried"])


def test_landmarks_add_the_restricted_sweep_axis_and_span_pairs(fake_device, monkeypatch):
    tc, calls = scorer({"restrict_sweep": 1, "chunk_span": 4096})
    monkeypatch.setattr(autotune, "_time_config", tc)
    r = autotune.tune(FakeGraph(landmarks=8), [0] * 512, [0] * 512, lanes_choices=(1,), budget_s=60.0)
    assert r["axes"][0] == "restrict_sweep"
    assert any(o.get("restrict_sweep") == 1 and o.get("chunk_span") in autotune.COMBO_SPANS for _, o in calls)
    assert r["restrict_sweep"] == 1 and r["chunk_span"] == 4096


def test_budget_and_cache(fake_device, monkeypatch, tmp_path):
    tc, calls = scorer({"threads_per_vertex": 16})
    monkeypatch.setattr(autotune, "_time_config", tc)
    r0 = autotune.tune(FakeGraph(), [0] * 512, [0] * 512, lanes_choices=(64,), budget_s=0.0)
    assert len(calls) == 1 and r0["tried"][0]["lanes"] == 64   # no budget: the defaults alone
    cache = tmp_path / "tune.json"
    calls.clear()
    r1 = autotune.tune(FakeGraph(), [0] * 512, [0] * 512, lanes_choices=(64,), budget_s=60.0, cache_path=str(cache))
    n1 = len(calls)
    assert n1 > 1 and r1["threads_per_vertex"] == 16
    saved = json.loads(cache.read_text())
    assert list(saved.values())[0]["threads_per_vertex"] == 16
    r2 = autotune.tune(FakeGraph(), [0] * 512, [0] * 512, lanes_choices=(64,), budget_s=60.0, cache_path=str(cache))
    assert len(calls) == n1 and r2 == r1                # answered from the cache
