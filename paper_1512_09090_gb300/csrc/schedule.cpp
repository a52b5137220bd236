// Chunk schedule of the TMA-staged sweep (host side).
//
// PHAST's scanning phase (Section 2) is correct in any order in which every
// vertex comes after the sources of its downward arcs; the level order is one
// such order.  The sweep cuts every level into chunks of consecutive vertices
// and runs them in the order built here: a topological order of the chunk
// dependency graph (chunk c depends on every chunk holding a source of a
// downward arc into c) chosen by greedy list scheduling that prefers the chunk
// with the smallest spatial key (the BFS rank of its first vertex in the input
// graph).  Chunks of all levels of one region then run close together in time,
// so a label row is still in L2 when the next levels read it, instead of being
// fetched from HBM once per level as a level-by-level sweep must.  A chunk only
// becomes eligible `delay` positions after its last dependency, so that the
// device rarely has to wait for one.
//
// The top levels of the hierarchy hold few vertices each but form a long chain
// of dependencies; run as separate chunks, every level would cost a round trip
// between CTAs.  The first `sync_levels` levels therefore get no chunks: the
// sweep runs them level by level before it starts on the schedule, and arcs
// from them are no dependencies.
//
// For position q the device receives its chunk's vertex and arc ranges and the
// list of positions q depends on; it starts chunk q once all of them are
// complete.
#include <algorithm>
#include <cstdint>
#include <queue>
#include <tuple>
#include <vector>

#include "sweep_schedule.h"

int iso_make_schedule(int n, int L, const int32_t* level_off, const uint32_t* down_off, const int32_t* down_src,
                      const int32_t* bfs, int vpb, int narrow_chunk, int narrow_width, int sync_levels, int delay,
                      int chunk_span, SweepSchedule* out) {
    if (n <= 0 || L <= 0 || vpb <= 0 || narrow_chunk <= 0 || sync_levels < 0 || sync_levels > L) return -1;
    // chunks in level order
    std::vector<int32_t> cv0, cv1, clev, cmode;
    std::vector<int32_t> chunk_of(n, -1);  // -1: swept before the schedule
    for (int j = sync_levels; j < L; ++j) {
        const int lo = level_off[j], hi = level_off[j + 1];
        const int mode = narrow_width > 0 && hi - lo < narrow_width ? 1 : 0;
        const int per = mode ? narrow_chunk : vpb;
        for (int b = lo; b < hi;) {
            // up to `per` vertices, and (chunk_span > 0) within chunk_span BFS
            // ranks of the first: a sparse level's chunk then covers a small
            // part of the map, so its rows are read again soon
            int e = b + 1;
            while (e < hi && e - b < per && (chunk_span <= 0 || (int64_t)bfs[e] - bfs[b] < chunk_span)) ++e;
            const int c = (int)cv0.size();
            cv0.push_back(b); cv1.push_back(e); clev.push_back(j); cmode.push_back(mode);
            for (int v = b; v < e; ++v) chunk_of[v] = c;
            b = e;
        }
    }
    const int Q = (int)cv0.size();
    // dependency edges pred -> c, each distinct pair once
    std::vector<int32_t> mark(Q, -1), indeg(Q, 0), soff(Q + 1, 0);
    for (int pass = 0; pass < 2; ++pass) {
        std::fill(mark.begin(), mark.end(), -1);
        std::vector<int32_t> fill;
        if (pass == 1) {
            for (int c = 0; c < Q; ++c) soff[c + 1] += soff[c];
            fill.assign(soff.begin(), soff.end() - 1);
            out->succ.assign(soff[Q], 0);
        }
        for (int c = 0; c < Q; ++c) {
            for (int v = cv0[c]; v < cv1[c]; ++v)
                for (uint32_t a = down_off[v]; a < down_off[v + 1]; ++a) {
                    const int pc = chunk_of[down_src[a]];
                    if (pc < 0 || mark[pc] == c) continue;  // done before the schedule, or seen
                    mark[pc] = c;
                    if (pass == 0) { soff[pc + 1]++; indeg[c]++; }
                    else out->succ[fill[pc]++] = c;
                }
        }
    }
    // greedy list scheduling: smallest spatial key among eligible chunks
    using Item = std::pair<int64_t, int32_t>;  // (key, chunk)
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> ready;
    std::priority_queue<std::tuple<int64_t, int64_t, int32_t>, std::vector<std::tuple<int64_t, int64_t, int32_t>>,
                        std::greater<std::tuple<int64_t, int64_t, int32_t>>>
        waiting;  // (eligible position, key, chunk)
    std::vector<int64_t> earliest(Q, 0);
    std::vector<int32_t> pos_of(Q, -1);
    // spatial key, then higher level first
    auto key = [&](int c) { return (int64_t)bfs[cv0[c]] * (L + 1) + clev[c]; };
    for (int c = 0; c < Q; ++c)
        if (indeg[c] == 0) ready.push({key(c), c});
    out->info.resize(Q);
    for (int q = 0; q < Q; ++q) {
        while (!waiting.empty() && std::get<0>(waiting.top()) <= q) {
            ready.push({std::get<1>(waiting.top()), std::get<2>(waiting.top())});
            waiting.pop();
        }
        if (ready.empty()) {  // nothing eligible yet: take the soonest one
            if (waiting.empty()) return -1;  // cycle: cannot happen for a valid hierarchy
            ready.push({std::get<1>(waiting.top()), std::get<2>(waiting.top())});
            waiting.pop();
        }
        const int c = ready.top().second;
        ready.pop();
        pos_of[c] = q;
        const uint32_t ab = down_off[cv0[c]] & ~1u;
        out->info[q] = {cv0[c], cv1[c], clev[c], cmode[c], (int32_t)ab, (int32_t)(down_off[cv1[c]] - ab), 0, 0};
        for (int32_t i = soff[c]; i < soff[c + 1]; ++i) {
            const int s = out->succ[i];
            earliest[s] = std::max<int64_t>(earliest[s], (int64_t)q + delay);
            if (--indeg[s] == 0) waiting.push({earliest[s], key(s), s});
        }
    }
    // Dependency lists by position, without the dependencies another
    // dependency already implies: if c depends on p and on p', and p' depends
    // on p, then p' completing implies p did (p' only started after p), so
    // only p' is checked.  (One hop of the transitive reduction.)
    std::vector<std::vector<int32_t>> preds(Q);
    for (int c = 0; c < Q; ++c)
        for (int32_t i = soff[c]; i < soff[c + 1]; ++i) preds[out->succ[i]].push_back(c);
    std::vector<int32_t> keep_mark(Q, -1), implied(Q, -1);
    std::vector<std::vector<int32_t>> kept(Q);
    for (int c = 0; c < Q; ++c) {
        for (int32_t p : preds[c]) keep_mark[p] = c;
        for (int32_t p1 : preds[c])
            for (int32_t p2 : preds[p1])
                if (keep_mark[p2] == c) implied[p2] = c;
        for (int32_t p : preds[c])
            if (implied[p] != c) kept[c].push_back(p);
    }
    std::vector<int32_t> pred_at(Q + 1, 0);  // padded list starts by position
    for (int c = 0; c < Q; ++c) pred_at[pos_of[c] + 1] = ((int32_t)kept[c].size() + 3) & ~3;
    for (int q = 0; q < Q; ++q) pred_at[q + 1] += pred_at[q];
    out->pred.assign(std::max<int32_t>(pred_at[Q], 4), 0);
    for (int c = 0; c < Q; ++c) {
        const int q = pos_of[c];
        const int32_t o = pred_at[q];
        const int32_t np = (int32_t)kept[c].size();
        for (int32_t i = 0; i < np; ++i) {
            const int32_t pq = pos_of[kept[c][i]];
            if (pq >= q) return -1;  // not topological: refuse
            out->pred[o + i] = pq;
        }
        for (int32_t i = np; i < pred_at[q + 1] - o; ++i) out->pred[o + i] = out->pred[o];
        out->info[q].pa = o;
        out->info[q].np = np;
    }
    out->succ.clear();
    out->succ.shrink_to_fit();
    out->Q = Q;
    return 0;
}
