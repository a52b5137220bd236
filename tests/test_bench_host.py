"""Host-side checks of bench.py: the reference arm (the oracle on host cores)
prints one JSON line with the fields the measurement contract asks for, and
the algorithmic byte count of a sweep follows its definition, and the clock
record (median and maximum SM clock, throttle reasons) is parsed as sampled."""

import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "grid1k_k16",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["unit"] == "queries/s" and j["higher_is_better"] is True
    assert j["value"] > 0 and j["steps"] >= 1 and j["config"]["workload"] == "grid1k_k16"
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == j["value"] and cb["sample"]
    assert j["e2e"] == {"value": j["value"], "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_sweep_bytes_definition():
    sys.path.insert(0, ROOT)
    import bench
    # a 6-vertex toy: three levels; downward arcs from sources 0, 0, 1, 2
    A = {"perm": np.arange(6), "level_off": np.array([0, 1, 3, 6]), "down_src": np.array([0, 0, 1, 2])}
    b = bench.sweep_bytes(A, 64)
    n, k = 6, 64
    assert b["offsets"] == 4 * (n + 1)
    assert b["arcs"] == 8 * 4
    assert b["d_write"] == 4 * k * (n - 3)       # the lowest level (3 vertices) stores no rows
    assert b["d_read"] == 4 * k * 3              # distinct sources 0, 1, 2
    assert b["mask_write"] == 8 * n and b["upflag_read"] == n
    assert bench.sweep_bytes(A, 64, write_all=True)["d_write"] == 4 * k * n


def test_sweep_bytes_scope_definition():
    """The roofline's numerator: 4(n+1) + 8 m_down + 4kn + 4kn + 4(L+1)."""
    sys.path.insert(0, ROOT)
    import bench
    A = {"perm": np.arange(6), "level_off": np.array([0, 1, 3, 6]), "down_src": np.array([0, 0, 1, 2])}
    n, k, L, m_down = 6, 64, 3, 4
    assert sum(bench.sweep_bytes_scope(A, k).values()) == 4 * (n + 1) + 8 * m_down + 8 * k * n + 4 * (L + 1)
    # 18M grid at 64 lanes: 9.990 GB
    n, m_down, L = 18_003_049, 87_496_783, 191
    big = {"perm": np.zeros(n, np.int8), "down_src": np.zeros(m_down, np.int8), "level_off": np.zeros(L + 1)}
    assert round(sum(bench.sweep_bytes_scope(big, 64).values()) / 1e9, 3) == 9.990
    assert [bench.lanes_class(k) for k in (1, 2, 5, 16, 17, 64)] == [1, 4, 8, 16, 32, 64]


def test_traffic_only_for_the_captured_sources_and_options():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.sweep_traffic("no-such-workload", {}) is None
    saved = dict(bench.SWEEP_TRAFFIC)
    try:
        h = bench.sweep_source_hash()
        bench.SWEEP_TRAFFIC["w"] = (h, {"schedule_delay": 608}, 123)
        assert bench.sweep_traffic("w", {"schedule_delay": 608, "use_cuda_graph": 1}) == 123
        assert bench.sweep_traffic("w", {"schedule_delay": 304}) is None     # other options
        assert bench.sweep_traffic("w", {"schedule_delay": 608, "chunk_span": 2500}) is None
        bench.SWEEP_TRAFFIC["w"] = ("0" * 16, {"schedule_delay": 608}, 123)
        assert bench.sweep_traffic("w", {"schedule_delay": 608}) is None     # other sources
    finally:
        bench.SWEEP_TRAFFIC.clear()
        bench.SWEEP_TRAFFIC.update(saved)


def test_clock_summary_parses_samples_and_throttle_reasons(tmp_path):
    # nvidia-smi --format=csv,noheader,nounits lines as the sampler records them:
    # index, clocks.sm, clocks.max.sm, power.draw, active reasons, then the four
    # reasons the bench reports (hw_slowdown, hw_thermal, sw_thermal, sw_power_cap)
    import bench
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join([
        "0, 2070, 2070, 880.10, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 901.55, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]) + "\n")
    cs = bench.ClockSampler(0)
    cs.path = str(path)
    cs.proc = object()          # as if nvidia-smi had been started
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    path.write_text("0, 1200, 2070, 500, 0x48, Active, Not Active, Active, Not Active\n")
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    cs.proc = None              # nvidia-smi missing: no record
    assert cs.summary() is None
