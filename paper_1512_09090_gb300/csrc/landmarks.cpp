// Landmark distances for restricted sweeps (host side).
//
// A restricted sweep skips the chunks of the hierarchy that are out of range
// for every query of a batch, in the spirit of RPHAST's restricted scan
// (Section 2) and isoPHAST's active cells (Section 5): only the part of the
// graph that can be in range is scanned.  Which chunks those are follows from
// lower bounds on distances by the triangle inequality with a few landmark
// vertices L (the ALT bounds):
//     d(s,v) >= d(L,v) - d(L,s)      and      d(s,v) >= d(s,L) - d(v,L).
// This file computes d(L,.) and d(.,L) for every landmark with one PHAST
// query each on the contraction hierarchy (Section 2), run on the host:
//   - forward, d(L,v): a Dijkstra from L in the upward graph, then one pass
//     over the vertices in sweep order taking the minimum over their incoming
//     downward arcs;
//   - backward, d(v,L): the same hierarchy serves the reversed graph, whose
//     upward arcs are the reversed downward arcs and whose downward arcs are
//     the reversed upward arcs: a Dijkstra from L over the incoming downward
//     arcs, then a pass in sweep order taking, for each v, the minimum over
//     its outgoing upward arcs (v,x) of d(x,L) + len.
// Landmarks are picked far apart: the first is the vertex farthest from sweep
// position 0 (a top vertex of the hierarchy), each next one the vertex whose
// smallest forward distance to the landmarks chosen so far is largest.
// Unreachable pairs hold kUnreach.
#include <algorithm>
#include <cstdint>
#include <functional>
#include <queue>
#include <utility>
#include <vector>

#include <new>

#include "ch_internal.h"
#include "landmarks.h"
#include "../../include/iso.h"

namespace {

using Dist = std::vector<uint32_t>;

// Dijkstra from sweep position s over the arcs `next(u, visit)` enumerates,
// then a pass over all positions in sweep order: d[v] = min(d[v], min over
// `into(v)` arcs (x, len) of d[x] + len), every x earlier in sweep order.
template <class Up, class Into>
Dist phast(const iso_ch& ch, int32_t s, Up up, Into into) {
    const int n = ch.n;
    Dist d(n, kUnreach);
    using Item = std::pair<uint64_t, int32_t>;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
    d[s] = 0;
    pq.push({0, s});
    while (!pq.empty()) {
        const auto [du, u] = pq.top();
        pq.pop();
        if (du != d[u]) continue;
        up(u, [&](int32_t x, int32_t w) {
            const uint64_t nd = std::min<uint64_t>(du + (uint64_t)w, kSat);
            if (nd < d[x]) { d[x] = (uint32_t)nd; pq.push({nd, x}); }
        });
    }
    for (int v = 0; v < n; ++v) {
        uint64_t best = d[v];
        into(v, [&](int32_t x, int32_t w) {
            if (d[x] != kUnreach) best = std::min<uint64_t>(best, (uint64_t)d[x] + (uint64_t)w);
        });
        d[v] = best == kUnreach ? kUnreach : (uint32_t)std::min<uint64_t>(best, kSat);
    }
    return d;
}

Dist forward(const iso_ch& ch, int32_t s) {
    return phast(
        ch, s,
        [&](int32_t u, auto&& f) { for (int64_t a = ch.up_off[u]; a < ch.up_off[u + 1]; ++a) f(ch.up_dst[a], ch.up_w[a]); },
        [&](int32_t v, auto&& f) {
            for (int64_t a = ch.down_off[v]; a < ch.down_off[v + 1]; ++a) f(ch.down_src[a], ch.down_w[a]);
        });
}

Dist backward(const iso_ch& ch, int32_t s) {
    return phast(
        ch, s,
        [&](int32_t u, auto&& f) {
            for (int64_t a = ch.down_off[u]; a < ch.down_off[u + 1]; ++a) f(ch.down_src[a], ch.down_w[a]);
        },
        [&](int32_t v, auto&& f) { for (int64_t a = ch.up_off[v]; a < ch.up_off[v + 1]; ++a) f(ch.up_dst[a], ch.up_w[a]); });
}

}  // namespace

int iso_landmarks_compute(const iso_ch& ch, int count, LandmarkSet* out) {
    if (count <= 0 || ch.n <= 0) return -1;
    const int n = ch.n;
    out->count = count;
    out->vertex.clear();
    out->fwd.assign((size_t)count * n, kUnreach);
    out->bwd.assign((size_t)count * n, kUnreach);
    // farthest-point choice on forward distances (unreachable vertices never chosen)
    Dist nearest(n, kUnreach);
    {
        const Dist d0 = forward(ch, 0);
        int32_t far = 0;
        for (int v = 0; v < n; ++v)
            if (d0[v] != kUnreach && d0[v] > d0[far]) far = v;
        out->vertex.push_back(far);
    }
    for (int i = 0; i < count; ++i) {
        const int32_t L = out->vertex[i];
        const Dist f = forward(ch, L);
        std::copy(f.begin(), f.end(), out->fwd.begin() + (size_t)i * n);
        for (int v = 0; v < n; ++v) nearest[v] = std::min(nearest[v], f[v]);
        if (i + 1 < count) {
            int32_t far = L;
            for (int v = 0; v < n; ++v)
                if (nearest[v] != kUnreach && nearest[v] > nearest[far]) far = v;
            out->vertex.push_back(far);
        }
    }
    // the backward distances are independent of each other
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < count; ++i) {
        const Dist b = backward(ch, out->vertex[i]);
        std::copy(b.begin(), b.end(), out->bwd.begin() + (size_t)i * n);
    }
    return 0;
}

extern "C" int iso_ch_landmarks(const iso_ch* ch, int32_t count, int32_t* vertices, uint32_t* fwd, uint32_t* bwd) {
    iso::clear_error();
    if (!ch || !vertices || !fwd || !bwd) { iso::set_error("iso_ch_landmarks: NULL argument"); return ISO_E_INVAL; }
    if (count < 1 || count > 16) { iso::set_error("iso_ch_landmarks: count %d outside 1..16", count); return ISO_E_INVAL; }
    LandmarkSet lm;
    try {
        if (iso_landmarks_compute(*ch, count, &lm) != 0) { iso::set_error("iso_ch_landmarks: bad input"); return ISO_E_INVAL; }
    } catch (const std::bad_alloc&) {
        iso::set_error("iso_ch_landmarks: out of host memory");
        return ISO_E_NOMEM;
    }
    const int n = ch->n;
    for (int i = 0; i < count; ++i) {
        vertices[i] = ch->perm[lm.vertex[i]];
        for (int p = 0; p < n; ++p) {
            fwd[(size_t)i * n + ch->perm[p]] = lm.fwd[(size_t)i * n + p];
            bwd[(size_t)i * n + ch->perm[p]] = lm.bwd[(size_t)i * n + p];
        }
    }
    return 0;
}

void iso_landmark_chunk_bounds(const LandmarkSet& lm, int n, int32_t v0, int32_t v1, uint32_t* lo_fwd,
                               uint32_t* hi_bwd) {
    for (int i = 0; i < lm.count; ++i) {
        uint32_t lo = kUnreach, hi = 0;
        const uint32_t* f = lm.fwd.data() + (size_t)i * n;
        const uint32_t* b = lm.bwd.data() + (size_t)i * n;
        for (int v = v0; v < v1; ++v) {
            lo = std::min(lo, f[v]);
            hi = std::max(hi, b[v]);
        }
        lo_fwd[i] = lo;
        hi_bwd[i] = hi;
    }
}
