// Contraction hierarchy construction on the host (Section 2, "In CH [19] ...").
//
// Vertices are contracted in rounds.  Each round picks an independent set I of
// vertices whose priority is a strict local minimum among their current
// neighbours, contracts all of I at once, and recomputes the priorities of the
// vertices around I.  Contracting v adds a shortcut a -> b for an in-neighbour a
// and an out-neighbour b whenever no witness path a ~> b of length at most
// len(a,v) + len(v,b) is found in the remaining graph without I.  Excluding all
// of I (not just v) keeps simultaneous contraction exact: every shortest path
// through a vertex of I is replaced either by its shortcut or by a witness that
// avoids I entirely.  A witness search that gives up only adds shortcuts, so the
// search limits trade size for speed and never correctness.
//
// Levels follow the paper's rule: when u is contracted, every neighbour v still
// present gets l(v) = max(l(v), l(u) + 1).  Hence every CH arc points from a
// lower to a strictly higher level, and sorting by descending level gives a
// valid PHAST sweep order.  Within a level, vertices are ordered by a BFS
// numbering of the input graph so that nearby vertices stay nearby in memory.
#include <omp.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <numeric>

#include "ch_internal.h"
#include "../../include/iso.h"

namespace {

constexpr int32_t kNoArc = INT32_MAX;              // absent direction in a Nbr entry
constexpr int64_t kKeyInf = INT64_MAX;
constexpr int32_t kClamp = 0x7FFFFFFE;             // shortcut lengths are clamped here

// One neighbour of a vertex in the remaining graph, both directions merged.
struct Nbr {
    int32_t v;     // neighbour
    int32_t wout;  // length of (this -> v), kNoArc if absent
    int32_t win;   // length of (v -> this), kNoArc if absent
};

struct Shortcut {
    int32_t a, b, w;  // a -> b
};

// Small open-addressing map vertex -> (tentative distance, flags) for witness searches.
struct DistMap {
    std::vector<int32_t> key;
    std::vector<int64_t> dist;
    std::vector<uint8_t> flag;  // bit0 settled, bit1 target
    std::vector<uint32_t> used;
    uint32_t mask = 0;

    void reset(uint32_t cap) {
        key.assign(cap, -1);
        dist.assign(cap, kKeyInf);
        flag.assign(cap, 0);
        used.clear();
        mask = cap - 1;
    }
    void clear() {
        for (uint32_t s : used) { key[s] = -1; dist[s] = kKeyInf; flag[s] = 0; }
        used.clear();
    }
    static uint32_t hash(int32_t k) { return (uint32_t)k * 0x9E3779B1u; }
    uint32_t slot(int32_t k) {
        if (used.size() * 2 >= key.size()) grow();
        uint32_t s = hash(k) & mask;
        while (key[s] != -1 && key[s] != k) s = (s + 1) & mask;
        if (key[s] == -1) { key[s] = k; used.push_back(s); }
        return s;
    }
    int64_t get(int32_t k) const {
        uint32_t s = hash(k) & mask;
        while (key[s] != -1) {
            if (key[s] == k) return dist[s];
            s = (s + 1) & mask;
        }
        return kKeyInf;
    }
    void grow() {
        std::vector<int32_t> ok = key;
        std::vector<int64_t> od = dist;
        std::vector<uint8_t> of = flag;
        std::vector<uint32_t> ou = used;
        reset((uint32_t)key.size() * 2);
        for (uint32_t s : ou) {
            uint32_t t = hash(ok[s]) & mask;
            while (key[t] != -1) t = (t + 1) & mask;
            key[t] = ok[s]; dist[t] = od[s]; flag[t] = of[s]; used.push_back(t);
        }
    }
};

struct HeapItem {
    int64_t key;
    int32_t v;
    bool operator>(const HeapItem& o) const { return key > o.key; }
};

struct Work {
    DistMap map;
    std::vector<HeapItem> heap;
    std::vector<int32_t> ins, outs;
    std::vector<int32_t> win, wout;
    Work() { map.reset(1024); }
};

struct Graph {
    int32_t n;
    std::vector<std::vector<Nbr>> adj;
    std::unique_ptr<std::atomic<uint8_t>[]> lock;
    void acquire(int32_t v) {
        uint8_t z = 0;
        while (!lock[v].compare_exchange_weak(z, 1, std::memory_order_acquire)) z = 0;
    }
    void release(int32_t v) { lock[v].store(0, std::memory_order_release); }
};

// Forward Dijkstra from src in the remaining graph, never entering `skip` or a
// vertex with excl[x] != 0.  Stops when the smallest key exceeds bound, after
// settle_limit settled vertices, or when every target is settled.
void witness_search(const Graph& g, int32_t src, int32_t skip, const uint8_t* excl, int64_t bound,
                    int settle_limit, int targets, Work& w) {
    DistMap& mp = w.map;
    auto& hp = w.heap;
    hp.clear();
    uint32_t s0 = mp.slot(src);
    mp.dist[s0] = 0;
    hp.push_back({0, src});
    int settled = 0;
    while (!hp.empty()) {
        std::pop_heap(hp.begin(), hp.end(), std::greater<HeapItem>());
        HeapItem it = hp.back();
        hp.pop_back();
        uint32_t s = mp.slot(it.v);
        if ((mp.flag[s] & 1) || it.key != mp.dist[s]) continue;
        if (it.key > bound) break;
        mp.flag[s] |= 1;
        if (mp.flag[s] & 2) {
            if (--targets == 0) break;
        }
        if (++settled >= settle_limit) break;
        for (const Nbr& e : g.adj[it.v]) {
            if (e.wout == kNoArc || e.v == skip || (excl && excl[e.v])) continue;
            int64_t nd = it.key + e.wout;
            if (nd > bound) continue;
            uint32_t t = mp.slot(e.v);
            if (nd < mp.dist[t]) {
                mp.dist[t] = nd;
                hp.push_back({nd, e.v});
                std::push_heap(hp.begin(), hp.end(), std::greater<HeapItem>());
            }
        }
    }
}

// Shortcuts needed to contract v.  Appends them to out (if non-null) and
// returns their number.
int contract_vertex(const Graph& g, int32_t v, const uint8_t* excl, int settle_limit, Work& w,
                    std::vector<Shortcut>* out) {
    w.ins.clear(); w.outs.clear(); w.win.clear(); w.wout.clear();
    for (const Nbr& e : g.adj[v]) {
        if (e.win != kNoArc) { w.ins.push_back(e.v); w.win.push_back(e.win); }
        if (e.wout != kNoArc) { w.outs.push_back(e.v); w.wout.push_back(e.wout); }
    }
    int added = 0;
    for (size_t i = 0; i < w.ins.size(); ++i) {
        int32_t a = w.ins[i];
        int64_t bound = -1;
        int ntarget = 0;
        w.map.clear();
        for (size_t j = 0; j < w.outs.size(); ++j) {
            if (w.outs[j] == a) continue;
            bound = std::max<int64_t>(bound, (int64_t)w.win[i] + w.wout[j]);
            uint32_t s = w.map.slot(w.outs[j]);
            if (!(w.map.flag[s] & 2)) { w.map.flag[s] |= 2; ++ntarget; }
        }
        if (ntarget == 0) continue;
        witness_search(g, a, v, excl, bound, settle_limit, ntarget, w);
        for (size_t j = 0; j < w.outs.size(); ++j) {
            int32_t b = w.outs[j];
            if (b == a) continue;
            int64_t via = (int64_t)w.win[i] + w.wout[j];
            if (w.map.get(b) > via) {
                ++added;
                if (out) out->push_back({a, b, (int32_t)std::min<int64_t>(via, kClamp)});
            }
        }
    }
    w.map.clear();
    return added;
}

// Shortcuts that contracting v would add if witnesses were limited to one or
// two arcs (a -> b, or a -> x -> b with x != v).  Only priorities use it: an
// over-count changes the contraction order, never the hierarchy's correctness.
int estimate_shortcuts(const Graph& g, int32_t v, Work& w) {
    w.ins.clear(); w.outs.clear(); w.win.clear(); w.wout.clear();
    for (const Nbr& e : g.adj[v]) {
        if (e.win != kNoArc) { w.ins.push_back(e.v); w.win.push_back(e.win); }
        if (e.wout != kNoArc) { w.outs.push_back(e.v); w.wout.push_back(e.wout); }
    }
    int added = 0;
    DistMap& mp = w.map;
    for (size_t i = 0; i < w.ins.size(); ++i) {
        int32_t a = w.ins[i];
        mp.clear();
        int ntarget = 0;
        for (size_t j = 0; j < w.outs.size(); ++j) {
            if (w.outs[j] == a) continue;
            uint32_t s = mp.slot(w.outs[j]);
            int64_t via = (int64_t)w.win[i] + w.wout[j];
            if (!(mp.flag[s] & 2)) { mp.flag[s] = 2; ++ntarget; mp.dist[s] = via; }
        }
        if (ntarget == 0) continue;
        int witnessed = 0;
        auto hit = [&](int32_t b, int64_t len) {
            uint32_t s = mp.hash(b) & mp.mask;
            while (mp.key[s] != -1) {
                if (mp.key[s] == b) {
                    if (mp.flag[s] == 2 && len <= mp.dist[s]) { mp.flag[s] = 3; ++witnessed; }
                    return;
                }
                s = (s + 1) & mp.mask;
            }
        };
        for (const Nbr& e : g.adj[a]) {
            if (e.wout == kNoArc || e.v == v) continue;
            hit(e.v, e.wout);
            for (const Nbr& f : g.adj[e.v]) {
                if (f.wout == kNoArc || f.v == v) continue;
                hit(f.v, (int64_t)e.wout + f.wout);
            }
            if (witnessed == ntarget) break;
        }
        added += ntarget - witnessed;
    }
    mp.clear();
    return added;
}

inline uint32_t mix(uint32_t x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    return x;
}

// Priority: weighted edge difference plus contracted neighbours and level
// (the terms of [19] with PHAST-friendly level weight, Section 6).
inline int64_t priority_of(int shortcuts, int arcs, int32_t contracted_nbrs, int32_t level) {
    return 4LL * (shortcuts - arcs) + 2LL * contracted_nbrs + 3LL * level;
}

int count_arcs(const Graph& g, int32_t v) {
    int c = 0;
    for (const Nbr& e : g.adj[v]) c += (e.win != kNoArc) + (e.wout != kNoArc);
    return c;
}

void insert_arc(std::vector<Nbr>& a, int32_t v, int32_t wout, int32_t win) {
    for (Nbr& e : a)
        if (e.v == v) {
            e.wout = std::min(e.wout, wout);
            e.win = std::min(e.win, win);
            return;
        }
    a.push_back({v, wout, win});
}

void erase_nbr(std::vector<Nbr>& a, int32_t v) {
    for (size_t i = 0; i < a.size(); ++i)
        if (a[i].v == v) {
            a[i] = a.back();
            a.pop_back();
            return;
        }
}

}  // namespace

extern "C" int iso_build_ch(int32_t n, int64_t m, const int32_t* tail, const int32_t* head,
                            const int32_t* weight, const iso_ch_opts* opts, iso_ch** out) {
    iso::clear_error();
    if (!out) { iso::set_error("iso_build_ch: out is NULL"); return ISO_E_INVAL; }
    *out = nullptr;
    if (n <= 0 || m < 0) { iso::set_error("iso_build_ch: n must be > 0 and m >= 0"); return ISO_E_INVAL; }
    if (m > 0 && (!tail || !head || !weight)) {
        iso::set_error("iso_build_ch: arc arrays are NULL");
        return ISO_E_INVAL;
    }
    if (m > INT32_MAX) { iso::set_error("iso_build_ch: more than 2^31-1 arcs"); return ISO_E_INVAL; }
    if (opts) {
        for (int r : opts->reserved)
            if (r) { iso::set_error("iso_build_ch: reserved option fields must be zero"); return ISO_E_INVAL; }
    }
    int32_t max_w = 0;
    for (int64_t e = 0; e < m; ++e) {
        if (tail[e] < 0 || tail[e] >= n || head[e] < 0 || head[e] >= n) {
            iso::set_error("iso_build_ch: arc %lld has an endpoint outside [0,%d)", (long long)e, n);
            return ISO_E_INVAL;
        }
        if (weight[e] < 0 || weight[e] > iso::kMaxWeight) {
            iso::set_error("iso_build_ch: arc %lld has length %d outside [0, 2^30)", (long long)e, weight[e]);
            return ISO_E_INVAL;
        }
        max_w = std::max(max_w, weight[e]);
    }
    const int threads = (opts && opts->threads > 0) ? opts->threads : omp_get_max_threads();
    const int settle_limit = (opts && opts->witness_settle_limit > 0) ? opts->witness_settle_limit : 400;
    const int prio_limit = (opts && opts->priority_settle_limit > 0) ? opts->priority_settle_limit : 0;
    auto t0 = std::chrono::steady_clock::now();
    // ISO_CH_VERBOSE in the environment: phase and per-round timings on stderr
    const bool verbose = std::getenv("ISO_CH_VERBOSE") != nullptr;
    auto since = [](std::chrono::steady_clock::time_point a) {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - a).count();
    };

    std::unique_ptr<iso_ch> ch;
    try {
        ch.reset(new iso_ch());
        ch->n = n; ch->m = m; ch->max_w = max_w;

        // BFS numbering of the undirected input graph: contraction runs on these
        // internal ids, so neighbouring vertices are close in memory, and the
        // same numbering orders vertices within a level of the sweep.
        std::vector<int32_t> bfs_of(n, -1), orig_of(n);
        {
            std::vector<int64_t> off(n + 1, 0);
            for (int64_t e = 0; e < m; ++e) { off[tail[e] + 1]++; off[head[e] + 1]++; }
            for (int32_t v = 0; v < n; ++v) off[v + 1] += off[v];
            std::vector<int32_t> nb(off[n]);
            std::vector<int64_t> fill(off.begin(), off.end() - 1);
            for (int64_t e = 0; e < m; ++e) { nb[fill[tail[e]]++] = head[e]; nb[fill[head[e]]++] = tail[e]; }
            int32_t next = 0, qh = 0;
            for (int32_t r = 0; r < n; ++r) {
                if (bfs_of[r] >= 0) continue;
                bfs_of[r] = next; orig_of[next++] = r;
                while (qh < next) {
                    int32_t u = orig_of[qh++];
                    for (int64_t j = off[u]; j < off[u + 1]; ++j)
                        if (bfs_of[nb[j]] < 0) { bfs_of[nb[j]] = next; orig_of[next++] = nb[j]; }
                }
            }
        }

        if (verbose) std::fprintf(stderr, "BFS numbering %.2f s\n", since(t0));
        Graph g;
        g.n = n;
        g.adj.resize(n);
        g.lock.reset(new std::atomic<uint8_t>[n]);
        for (int32_t v = 0; v < n; ++v) g.lock[v].store(0, std::memory_order_relaxed);
        {
            std::vector<int32_t> deg(n, 0);
            for (int64_t e = 0; e < m; ++e) {
                if (tail[e] == head[e]) continue;  // a self-loop is never on a shortest path
                deg[bfs_of[tail[e]]]++; deg[bfs_of[head[e]]]++;
            }
            for (int32_t v = 0; v < n; ++v) g.adj[v].reserve(deg[v]);
            for (int64_t e = 0; e < m; ++e) {
                int32_t a = bfs_of[tail[e]], b = bfs_of[head[e]], w = weight[e];
                if (a == b) continue;
                insert_arc(g.adj[a], b, w, kNoArc);
                insert_arc(g.adj[b], a, kNoArc, w);
            }
        }

        if (verbose) std::fprintf(stderr, "setup (BFS numbering, adjacency) %.2f s\n", since(t0));
        auto tp = std::chrono::steady_clock::now();
        std::vector<int32_t> level(n, 0), cn(n, 0);
        std::vector<int64_t> prio(n, 0);
        std::vector<uint8_t> in_set(n, 0), dirty(n, 0), contracted(n, 0);
        std::vector<Work> work(threads);

#pragma omp parallel for schedule(dynamic, 1024) num_threads(threads)
        for (int32_t v = 0; v < n; ++v) {
            Work& w = work[omp_get_thread_num()];
            int sc = prio_limit > 2 ? contract_vertex(g, v, nullptr, prio_limit, w, nullptr) : estimate_shortcuts(g, v, w);
            prio[v] = priority_of(sc, count_arcs(g, v), 0, 0);
        }

        std::vector<int32_t> remaining(n);
        std::iota(remaining.begin(), remaining.end(), 0);
        std::vector<int32_t> chosen;
        std::vector<std::vector<Shortcut>> sc_buf(threads);
        std::vector<std::vector<int32_t>> dirty_buf(threads);
        int64_t shortcuts = 0;

        if (verbose) std::fprintf(stderr, "initial priorities %.2f s\n", since(tp));
        tp = std::chrono::steady_clock::now();
        int round = 0;
        while (!remaining.empty()) {
            auto tr0 = std::chrono::steady_clock::now();
            // 1. independent set: strict local minima of (priority, hash, id)
            const int64_t R = (int64_t)remaining.size();
            chosen.assign(R, -1);
#pragma omp parallel for schedule(dynamic, 4096) num_threads(threads)
            for (int64_t i = 0; i < R; ++i) {
                int32_t v = remaining[i];
                auto key = [&](int32_t x) { return std::make_tuple(prio[x], mix((uint32_t)x), x); };
                auto kv = key(v);
                bool best = true;
                for (const Nbr& e : g.adj[v])
                    if (key(e.v) < kv) { best = false; break; }
                if (best) { chosen[i] = v; in_set[v] = 1; }
            }
            chosen.erase(std::remove(chosen.begin(), chosen.end(), -1), chosen.end());

            auto tr1 = std::chrono::steady_clock::now();
            // 2. shortcuts of every chosen vertex, witnesses avoiding the whole set
            const int64_t C = (int64_t)chosen.size();
#pragma omp parallel for schedule(dynamic, 64) num_threads(threads)
            for (int64_t i = 0; i < C; ++i) {
                int t = omp_get_thread_num();
                contract_vertex(g, chosen[i], in_set.data(), settle_limit, work[t], &sc_buf[t]);
            }

            auto tr2 = std::chrono::steady_clock::now();
            // 3. detach the chosen vertices from their neighbours, raise levels
#pragma omp parallel for schedule(dynamic, 256) num_threads(threads)
            for (int64_t i = 0; i < C; ++i) {
                int t = omp_get_thread_num();
                int32_t v = chosen[i];
                for (const Nbr& e : g.adj[v]) {
                    int32_t x = e.v;
                    g.acquire(x);
                    erase_nbr(g.adj[x], v);
                    level[x] = std::max(level[x], level[v] + 1);
                    cn[x]++;
                    if (!dirty[x]) { dirty[x] = 1; dirty_buf[t].push_back(x); }
                    g.release(x);
                }
            }
            // 4. insert shortcuts
#pragma omp parallel num_threads(threads)
            {
                auto& buf = sc_buf[omp_get_thread_num()];
                for (const Shortcut& s : buf) {
                    g.acquire(s.a); insert_arc(g.adj[s.a], s.b, s.w, kNoArc); g.release(s.a);
                    g.acquire(s.b); insert_arc(g.adj[s.b], s.a, kNoArc, s.w); g.release(s.b);
                }
            }
            for (int t = 0; t < threads; ++t) { shortcuts += (int64_t)sc_buf[t].size(); sc_buf[t].clear(); }
            for (int32_t v : chosen) { contracted[v] = 1; in_set[v] = 0; }

            auto tr3 = std::chrono::steady_clock::now();
            // 5. new priorities around the contracted set
            std::vector<int32_t> upd;
            for (int t = 0; t < threads; ++t) {
                upd.insert(upd.end(), dirty_buf[t].begin(), dirty_buf[t].end());
                dirty_buf[t].clear();
            }
#pragma omp parallel for schedule(dynamic, 256) num_threads(threads)
            for (int64_t i = 0; i < (int64_t)upd.size(); ++i) {
                int32_t x = upd[i];
                dirty[x] = 0;
                Work& w = work[omp_get_thread_num()];
                int sc = prio_limit > 2 ? contract_vertex(g, x, nullptr, prio_limit, w, nullptr) : estimate_shortcuts(g, x, w);
                prio[x] = priority_of(sc, count_arcs(g, x), cn[x], level[x]);
            }
            remaining.erase(std::remove_if(remaining.begin(), remaining.end(),
                                           [&](int32_t v) { return contracted[v] != 0; }),
                            remaining.end());
            if (verbose) {
                int64_t deg = 0;
                for (int32_t v : remaining) deg += (int64_t)g.adj[v].size();
                auto sec = [](auto a, auto b) { return std::chrono::duration<double>(b - a).count(); };
                auto tr4 = std::chrono::steady_clock::now();
                std::fprintf(stderr, "round %d: contracted %lld remaining %lld avgdeg %.1f shortcuts %lld "
                             "sel %.3f contract %.3f apply %.3f prio %.3f (%zu)\n",
                             round, (long long)C, (long long)remaining.size(),
                             remaining.empty() ? 0.0 : (double)deg / remaining.size(), (long long)shortcuts,
                             sec(tr0, tr1), sec(tr1, tr2), sec(tr2, tr3), sec(tr3, tr4), upd.size());
            }
            ++round;
        }
        ch->shortcuts = shortcuts;
        if (verbose) std::fprintf(stderr, "contraction rounds %.2f s\n", since(tp));
        tp = std::chrono::steady_clock::now();

        // ---- sweep order: descending level, BFS numbering within a level ----
        int32_t L = 0;
        for (int32_t v = 0; v < n; ++v) L = std::max(L, level[v] + 1);
        ch->L = L;
        std::vector<int32_t> order(n);  // sweep position -> internal id
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return level[a] > level[b]; });
        std::vector<int32_t> P(n);      // internal id -> sweep position
        for (int32_t p = 0; p < n; ++p) P[order[p]] = p;
        ch->perm.resize(n);
        ch->pos.resize(n);
        ch->bfs.resize(n);
        for (int32_t p = 0; p < n; ++p) {
            ch->perm[p] = orig_of[order[p]];
            ch->bfs[p] = order[p];  // internal ids are BFS ranks
            ch->pos[orig_of[order[p]]] = p;
        }
        ch->level_off.assign(L + 1, 0);
        {
            std::vector<int32_t> cnt(L, 0);
            for (int32_t v = 0; v < n; ++v) cnt[L - 1 - level[v]]++;
            for (int32_t j = 0; j < L; ++j) ch->level_off[j + 1] = ch->level_off[j] + cnt[j];
        }

        // ---- CSRs in sweep order ----
        // adj[v] of a contracted v still lists its neighbours at contraction
        // time, all of higher rank: wout gives upward arcs v -> x, win gives
        // downward arcs x -> v.
        ch->down_off.assign(n + 1, 0);
        ch->up_off.assign(n + 1, 0);
        for (int32_t p = 0; p < n; ++p) {
            int64_t din = 0, dout = 0;
            for (const Nbr& e : g.adj[order[p]]) { din += e.win != kNoArc; dout += e.wout != kNoArc; }
            ch->down_off[p + 1] = ch->down_off[p] + din;
            ch->up_off[p + 1] = ch->up_off[p] + dout;
        }
        if (ch->down_off[n] > (int64_t)UINT32_MAX || ch->up_off[n] > (int64_t)UINT32_MAX) {
            iso::set_error("iso_build_ch: more than 2^32-1 CH arcs");
            return ISO_E_INVAL;
        }
        ch->down_src.resize(ch->down_off[n]); ch->down_w.resize(ch->down_off[n]);
        ch->up_dst.resize(ch->up_off[n]); ch->up_w.resize(ch->up_off[n]);
#pragma omp parallel for schedule(dynamic, 4096) num_threads(threads)
        for (int32_t p = 0; p < n; ++p) {
            std::vector<std::pair<int32_t, int32_t>> dn, up;
            for (const Nbr& e : g.adj[order[p]]) {
                if (e.win != kNoArc) dn.push_back({P[e.v], e.win});
                if (e.wout != kNoArc) up.push_back({P[e.v], e.wout});
            }
            std::sort(dn.begin(), dn.end());
            std::sort(up.begin(), up.end());
            int64_t o = ch->down_off[p];
            for (auto& a : dn) { ch->down_src[o] = a.first; ch->down_w[o] = a.second; ++o; }
            o = ch->up_off[p];
            for (auto& a : up) { ch->up_dst[o] = a.first; ch->up_w[o] = a.second; ++o; }
        }
        ch->orig_off.assign(n + 1, 0);
        const std::vector<int32_t>& Q = ch->pos;
        for (int64_t e = 0; e < m; ++e) ch->orig_off[Q[tail[e]] + 1]++;
        for (int32_t p = 0; p < n; ++p) ch->orig_off[p + 1] += ch->orig_off[p];
        ch->orig_head.resize(m); ch->orig_id.resize(m);
        {
            std::vector<int64_t> fill(ch->orig_off.begin(), ch->orig_off.end() - 1);
            for (int64_t e = 0; e < m; ++e) {
                int64_t o = fill[Q[tail[e]]]++;
                ch->orig_head[o] = Q[head[e]];
                ch->orig_id[o] = (int32_t)e;
            }
        }
        if (verbose) std::fprintf(stderr, "sweep order and CSRs %.2f s\n", since(tp));
    } catch (const std::bad_alloc&) {
        iso::set_error("iso_build_ch: out of host memory");
        return ISO_E_NOMEM;
    }
    ch->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = ch.release();
    return ISO_OK;
}

extern "C" int iso_ch_info(const iso_ch* ch, iso_ch_stats* out) {
    iso::clear_error();
    if (!ch || !out) { iso::set_error("iso_ch_info: NULL argument"); return ISO_E_INVAL; }
    std::memset(out, 0, sizeof(*out));
    out->n = ch->n;
    out->levels = ch->L;
    out->m = ch->m;
    out->m_up = ch->up_off.empty() ? 0 : ch->up_off.back();
    out->m_down = ch->down_off.empty() ? 0 : ch->down_off.back();
    out->shortcuts = ch->shortcuts;
    out->max_weight = ch->max_w;
    int32_t widest = 0;
    for (int32_t j = 0; j < ch->L; ++j) widest = std::max(widest, ch->level_off[j + 1] - ch->level_off[j]);
    out->max_level_width = widest;
    out->build_seconds = ch->build_seconds;
    return ISO_OK;
}

extern "C" int32_t iso_ch_sweep_position(const iso_ch* ch, int32_t v) {
    iso::clear_error();
    if (!ch) { iso::set_error("iso_ch_sweep_position: NULL hierarchy"); return -1; }
    if (v < 0 || v >= ch->n) { iso::set_error("iso_ch_sweep_position: vertex %d outside 0..%d", v, ch->n - 1); return -1; }
    return ch->pos[v];
}

extern "C" void iso_free_ch(iso_ch* ch) { delete ch; }
