"""Host test of the chunk schedule of the TMA-staged sweep (csrc/schedule.cpp).

PHAST's scan (Section 2) is correct in any order in which every vertex comes
after the sources of its downward arcs.  The sweep runs chunks in the order
the schedule gives and starts a chunk once the positions in its dependency
list are complete, so the schedule must be a topological order of the chunk
dependency graph, and the dependency lists -- reduced by dropping lists that
another dependency already implies -- must still imply every real dependency.
A small C++ driver links schedule.cpp, builds schedules for random
level-structured DAGs and checks exactly that, plus the record layout the
kernel's bulk copies need (16-byte aligned, padded lists; even arc bases) and
the optional limit on a chunk's BFS-rank span."""

import os
import shutil
import subprocess
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1512_09090_gb300", "csrc")

DRIVER = textwrap.dedent(r"""
    #include <cstdio>
    #include <cstdlib>
    #include <random>
    #include <vector>
    #include "sweep_schedule.h"

    static int fail(const char* what, long a, long b) {
        std::printf("FAIL %s %ld %ld\n", what, a, b);
        return 1;
    }

    // one random hierarchy: level sizes, downward arcs from higher to lower levels
    static int check(unsigned seed, int vpb, int narrow_width, int sync_levels, int delay, int span) {
        std::mt19937 rng(seed);
        const int L = 2 + (int)(rng() % 12);
        std::vector<int32_t> level_off(L + 1, 0);
        for (int j = 0; j < L; ++j) level_off[j + 1] = level_off[j] + 1 + (int)(rng() % (j < 3 ? 4 : 300));
        const int n = level_off[L];
        std::vector<int> level_of(n);
        for (int j = 0; j < L; ++j)
            for (int v = level_off[j]; v < level_off[j + 1]; ++v) level_of[v] = j;
        std::vector<uint32_t> down_off(n + 5, 0);
        std::vector<int32_t> down_src;
        for (int v = 0; v < n; ++v) {
            down_off[v] = (uint32_t)down_src.size();
            const int j = level_of[v];
            if (j > 0) {
                const int deg = (int)(rng() % 6);
                for (int d = 0; d < deg; ++d) down_src.push_back((int32_t)(rng() % (uint32_t)level_off[j]));
            }
        }
        for (int i = n; i < n + 5; ++i) down_off[i] = (uint32_t)down_src.size();
        std::vector<int32_t> bfs(n);
        for (int v = 0; v < n; ++v) bfs[v] = v;
        for (int v = n - 1; v > 0; --v) std::swap(bfs[v], bfs[rng() % (uint32_t)(v + 1)]);
        if (sync_levels > L) sync_levels = L;

        SweepSchedule S;
        if (iso_make_schedule(n, L, level_off.data(), down_off.data(), down_src.data(), bfs.data(), vpb, 31,
                              narrow_width, sync_levels, delay, span, &S) != 0)
            return fail("build", seed, 0);
        const int Q = S.Q;
        // every vertex below the synchronous levels in exactly one chunk; chunks within one level
        std::vector<int> pos_of_v(n, -1);
        for (int q = 0; q < Q; ++q) {
            const SchedChunk& c = S.info[q];
            if (c.v0 >= c.v1) return fail("empty chunk", q, 0);
            if (c.v0 < level_off[c.level] || c.v1 > level_off[c.level + 1]) return fail("chunk crosses level", q, 0);
            if (c.level < sync_levels) return fail("synchronous level scheduled", q, c.level);
            const int cap = c.mode ? 31 : vpb;
            if (c.v1 - c.v0 > cap) return fail("chunk too large", q, c.v1 - c.v0);
            for (int v = c.v0; v < c.v1; ++v) {
                if (pos_of_v[v] != -1) return fail("vertex twice", v, q);
                pos_of_v[v] = q;
                if (span > 0 && bfs[v] - bfs[c.v0] >= span) return fail("chunk span", q, v);
            }
            if ((c.abase & 1) != 0 || (uint32_t)c.abase > down_off[c.v0]) return fail("arc base", q, c.abase);
            if ((uint32_t)(c.abase + c.na) != down_off[c.v1]) return fail("arc count", q, c.na);
            if ((c.pa & 3) != 0) return fail("list alignment", q, c.pa);
            const int padded = (c.np + 3) & ~3;
            if (c.pa + padded > (int)S.pred.size()) return fail("list bounds", q, c.pa);
            for (int i = 0; i < padded; ++i) {
                const int p = S.pred[c.pa + i];
                if (p < 0 || p >= q) return fail("dependency not earlier", q, p);
                if (i >= c.np && c.np > 0 && p != S.pred[c.pa]) return fail("padding", q, p);
            }
        }
        for (int v = level_off[sync_levels]; v < n; ++v)
            if (pos_of_v[v] < 0) return fail("vertex missing", v, 0);
        // transitive closure of the kept lists covers every arc dependency
        std::vector<std::vector<char>> reach(Q, std::vector<char>(Q, 0));
        for (int q = 0; q < Q; ++q) {
            const SchedChunk& c = S.info[q];
            for (int i = 0; i < c.np; ++i) {
                const int p = S.pred[c.pa + i];
                reach[q][p] = 1;
                for (int r = 0; r < Q; ++r)
                    if (reach[p][r]) reach[q][r] = 1;
            }
        }
        for (int v = level_off[sync_levels]; v < n; ++v)
            for (uint32_t a = down_off[v]; a < down_off[v + 1]; ++a) {
                const int u = down_src[a];
                if (level_of[u] < sync_levels) continue;  // swept before the schedule
                const int pu = pos_of_v[u], pv = pos_of_v[v];
                if (pu >= pv) return fail("not topological", pu, pv);
                if (!reach[pv][pu]) return fail("dependency lost", pv, pu);
            }
        return 0;
    }

    int main() {
        int bad = 0, runs = 0;
        for (unsigned seed = 1; seed <= 60; ++seed)
            for (int vpb : {1, 7, 64})
                for (int nw : {0, 50})
                    for (int sync : {0, 2})
                        for (int delay : {0, 3, 40})
                            for (int span : {0, 1, 100}) {
                                bad += check(seed, vpb, nw, sync, delay, span);
                                ++runs;
                            }
        std::printf("%d runs, %d failed\n", runs, bad);
        return bad ? 1 : 0;
    }
""")


def test_schedule_is_topological_and_lists_imply_all_dependencies(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "drv.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "drv"
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, str(src), os.path.join(CSRC, "schedule.cpp"),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:]
    assert "0 failed" in r.stdout
