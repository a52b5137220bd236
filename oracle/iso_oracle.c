/*
 * iso_oracle.c -- CPU oracle for the isochrone problem.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what an isochrone query computes (Baum, Buchhold, Dibbelt,
 * Wagner: "Fast Computation of Isochrones in Road Networks", arXiv 1512.09090).
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (Section 3, problem statement):
 *   input  : directed graph G=(V,E), len: E -> Z>=0, source s, limit tau >= 0;
 *   in range: v with d(s,v) <= tau (inclusive), d the shortest-path distance
 *            of Section 2;
 *   output : the isochrone edges, i.e. every arc (u,v) in E with exactly one
 *            endpoint in range, reported by its input index (arc id), ascending.
 *
 * Two independent extractions are provided:
 *   orc_tau_dijkstra + orc_isochrone_scan : Dijkstra (Section 2) stopped once
 *       the minimum key exceeds tau, then a scan over all m arcs applying the
 *       definition directly;
 *   orc_iso_dijkstra : the isoDijkstra variant of Section 3 (in-neighbours of a
 *       settled vertex enter the queue with key infinity; after the stop, the
 *       vertices left in the queue are swept for isochrone edges).
 *
 * Distances accumulate in int64, so no sum can overflow; the reported label of
 * a vertex is its distance if it is in range and 0x7FFFFFFF otherwise.
 *
 * Readings of the paper (where it is silent): lengths and tau are integers;
 * parallel arcs are all reported; a self-loop never crosses; the sweep of
 * isoDijkstra checks both the incoming and the outgoing arcs of every vertex
 * left in the queue, which is what makes the infinity-key insertions report
 * the arcs that point into the range.
 *
 * The ORC_MUTANT hooks exist only so that the test suite can compile variants
 * with a planted mistake and show that its pins catch each one; the default
 * build (ORC_MUTANT undefined) contains none of them.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

#define ORC_OUT_INF 0x7FFFFFFF
#define ORC_KEY_INF INT64_MAX

/* ---- adjacency arrays (Section 2): arcs grouped by one endpoint --------- */

typedef struct {
    int64_t* off;   /* [n+1] */
    int64_t* arc;   /* [m] arc ids grouped by the chosen endpoint, id order kept */
} adjacency;

static int build_adjacency(int32_t n, int64_t m, const int32_t* endpoint, adjacency* a) {
    a->off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    a->arc = (int64_t*)malloc(((size_t)m + 1) * sizeof(int64_t));
    if (!a->off || !a->arc) return -1;
    for (int64_t e = 0; e < m; ++e) a->off[endpoint[e] + 1]++;
    for (int32_t v = 0; v < n; ++v) a->off[v + 1] += a->off[v];
    int64_t* fill = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!fill) return -1;
    memcpy(fill, a->off, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) a->arc[fill[endpoint[e]]++] = e;
    free(fill);
    return 0;
}

static void free_adjacency(adjacency* a) { free(a->off); free(a->arc); }

/* ---- binary min-heap of (key, vertex); stale entries are skipped -------- */

typedef struct { int64_t key; int32_t v; } heap_entry;
typedef struct { heap_entry* h; int64_t size, cap; } min_heap;

static int heap_push(min_heap* q, int64_t key, int32_t v) {
    if (q->size == q->cap) {
        int64_t nc = q->cap ? 2 * q->cap : 64;
        heap_entry* nh = (heap_entry*)realloc(q->h, (size_t)nc * sizeof(heap_entry));
        if (!nh) return -1;
        q->h = nh; q->cap = nc;
    }
    int64_t i = q->size++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (q->h[p].key <= key) break;
        q->h[i] = q->h[p];
        i = p;
    }
    q->h[i].key = key; q->h[i].v = v;
    return 0;
}

static heap_entry heap_pop(min_heap* q) {
    heap_entry top = q->h[0];
    heap_entry last = q->h[--q->size];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= q->size) break;
        if (c + 1 < q->size && q->h[c + 1].key < q->h[c].key) c++;
        if (q->h[c].key >= last.key) break;
        q->h[i] = q->h[c];
        i = c;
    }
    if (q->size > 0) q->h[i] = last;
    return top;
}

/* ---- in-range predicate (Section 3): d(s,v) <= tau ------------------------ */

static int in_range(int64_t d, int64_t tau) {
#if ORC_MUTANT == 1
    return d < tau;                       /* planted: strict inequality */
#else
    return d <= tau;
#endif
}

/* ---- Dijkstra stopped at tau (Sections 2 and 3) --------------------------- */

/* Settles, in order of distance, every vertex with d(s,v) <= tau.  dist[v] is
 * d(s,v) for settled vertices and ORC_OUT_INF for all others.  Returns the
 * number of settled vertices, or -1 on bad input / allocation failure. */
static int64_t tau_dijkstra(int32_t n, const adjacency* out, const int32_t* tail,
                            const int32_t* head, const int32_t* len, int32_t s,
                            int64_t tau, int32_t* dist) {
    (void)tail;
    int64_t* d = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    char* settled = (char*)calloc((size_t)n, 1);
    min_heap q = {0, 0, 0};
    if (!d || !settled) { free(d); free(settled); return -1; }
    for (int32_t v = 0; v < n; ++v) d[v] = ORC_KEY_INF;
    d[s] = 0;
    int64_t count = 0;
    if (heap_push(&q, 0, s)) count = -1;
    while (count >= 0 && q.size > 0) {
        heap_entry top = heap_pop(&q);
        if (settled[top.v] || top.key != d[top.v]) continue;   /* stale entry */
        if (!in_range(top.key, tau)) break;                     /* stopping criterion */
        int32_t u = top.v;
        settled[u] = 1;
        ++count;
        for (int64_t j = out->off[u]; j < out->off[u + 1]; ++j) {
            int64_t e = out->arc[j];
#if ORC_MUTANT == 2
            int32_t v = tail[e];                                 /* planted: wrong endpoint */
#else
            int32_t v = head[e];
#endif
#if ORC_MUTANT == 3
            int64_t nd = d[u];                                   /* planted: dropped length */
#else
            int64_t nd = d[u] + (int64_t)len[e];
#endif
            if (nd < d[v]) {
                d[v] = nd;
                if (heap_push(&q, nd, v)) { count = -1; break; }
            }
        }
    }
    for (int32_t v = 0; v < n; ++v) dist[v] = settled[v] ? (int32_t)d[v] : ORC_OUT_INF;
    free(d); free(settled); free(q.h);
    return count;
}

int64_t orc_tau_dijkstra(int32_t n, int64_t m, const int32_t* tail, const int32_t* head,
                         const int32_t* len, int32_t s, int64_t tau, int32_t* dist) {
    if (n <= 0 || m < 0 || s < 0 || s >= n || tau < 0 || !dist) return -1;
    adjacency out;
    if (build_adjacency(n, m, tail, &out)) { free_adjacency(&out); return -1; }
    int64_t c = tau_dijkstra(n, &out, tail, head, len, s, tau, dist);
    free_adjacency(&out);
    return c;
}

/* ---- isochrone edges straight from the definition (Section 3) ------------ */

/* Scans arcs 0..m-1 and reports those with exactly one endpoint in range.
 * dist holds the labels of orc_tau_dijkstra.  Writes at most cap ids; returns
 * the total number of isochrone edges. */
int64_t orc_isochrone_scan(int64_t m, const int32_t* tail, const int32_t* head,
                           const int32_t* dist, int64_t tau, int32_t* out, int64_t cap) {
    int64_t cnt = 0;
    for (int64_t e = 0; e < m; ++e) {
        int a = dist[tail[e]] != ORC_OUT_INF && in_range(dist[tail[e]], tau);
        int b = dist[head[e]] != ORC_OUT_INF && in_range(dist[head[e]], tau);
#if ORC_MUTANT == 4
        int crosses = a || b;                                    /* planted: OR for XOR */
#else
        int crosses = a != b;
#endif
        if (crosses) {
            if (cnt < cap) out[cnt] = (int32_t)e;
            ++cnt;
        }
    }
    return cnt;
}

/* ---- isoDijkstra (Section 3) ---------------------------------------------- */

static int cmp_i32(const void* x, const void* y) {
    int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
    return (a > b) - (a < b);
}

/* Runs isoDijkstra from s and writes the isochrone edges, ascending, to out
 * (at most cap).  Returns the total count or -1 on error. */
int64_t orc_iso_dijkstra(int32_t n, int64_t m, const int32_t* tail, const int32_t* head,
                         const int32_t* len, int32_t s, int64_t tau, int32_t* out, int64_t cap) {
    if (n <= 0 || m < 0 || s < 0 || s >= n || tau < 0) return -1;
    adjacency outa, ina;
    if (build_adjacency(n, m, tail, &outa) || build_adjacency(n, m, head, &ina)) return -1;
    int64_t* d = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    char* queued = (char*)calloc((size_t)n, 1);   /* inserted, not settled */
    char* settled = (char*)calloc((size_t)n, 1);
    int32_t* found = (int32_t*)malloc(((size_t)m + 1) * sizeof(int32_t));
    min_heap q = {0, 0, 0};
    int64_t cnt = 0;
    if (!d || !queued || !settled || !found) { cnt = -1; goto done; }
    for (int32_t v = 0; v < n; ++v) d[v] = ORC_KEY_INF;
    d[s] = 0; queued[s] = 1;
    if (heap_push(&q, 0, s)) { cnt = -1; goto done; }
    while (q.size > 0) {
        heap_entry top = q.h[0];
        if (settled[top.v] || top.key != d[top.v]) { heap_pop(&q); continue; }
        if (top.key == ORC_KEY_INF || !in_range(top.key, tau)) break;  /* stop: min key > tau */
        heap_pop(&q);
        int32_t u = top.v;
        settled[u] = 1; queued[u] = 0;
        for (int64_t j = outa.off[u]; j < outa.off[u + 1]; ++j) {   /* scan (u,v) */
            int64_t e = outa.arc[j];
            int32_t v = head[e];
            int64_t nd = d[u] + (int64_t)len[e];
            if (!settled[v] && nd < d[v]) {
                d[v] = nd; queued[v] = 1;
                if (heap_push(&q, nd, v)) { cnt = -1; goto done; }
            }
        }
#if ORC_MUTANT != 5
        for (int64_t j = ina.off[u]; j < ina.off[u + 1]; ++j) {     /* in-arcs (v,u) */
            int32_t v = tail[ina.arc[j]];
            if (!settled[v] && d[v] == ORC_KEY_INF && !queued[v]) {
                queued[v] = 1;                                       /* key infinity */
                if (heap_push(&q, ORC_KEY_INF, v)) { cnt = -1; goto done; }
            }
        }
#endif
    }
    /* sweep the vertices left in the queue (all out of range) */
    for (int32_t v = 0; v < n; ++v) {
        if (!queued[v]) continue;
        for (int64_t j = ina.off[v]; j < ina.off[v + 1]; ++j) {      /* (u,v), u in range */
            int64_t e = ina.arc[j];
            if (settled[tail[e]]) found[cnt++] = (int32_t)e;
        }
        for (int64_t j = outa.off[v]; j < outa.off[v + 1]; ++j) {    /* (v,u), u in range */
            int64_t e = outa.arc[j];
            if (settled[head[e]]) found[cnt++] = (int32_t)e;
        }
    }
    qsort(found, (size_t)cnt, sizeof(int32_t), cmp_i32);
    for (int64_t i = 0; i < cnt && i < cap; ++i) out[i] = found[i];
done:
    free_adjacency(&outa); free_adjacency(&ina);
    free(d); free(queued); free(settled); free(found); free(q.h);
    return cnt;
}

/* ---- a batch of independent queries -------------------------------------- */

/* For query i (source sources[i], limit taus[i]) runs orc_tau_dijkstra and
 * orc_isochrone_scan.  out_off[0..k] receives the list offsets; the lists are
 * written to out_arcs only if the total fits cap.  out_dist (nullable) receives
 * the labels of query i at out_dist[i*n + v].  Queries are independent and run
 * on up to `threads` OpenMP threads.  Returns the total count, or -1 on error. */
int64_t orc_query_batch(int32_t n, int64_t m, const int32_t* tail, const int32_t* head,
                        const int32_t* len, int32_t k, const int32_t* sources,
                        const int32_t* taus, int64_t* out_off, int32_t* out_arcs, int64_t cap,
                        int32_t* out_dist, int threads) {
    if (n <= 0 || m < 0 || k < 0 || !out_off) return -1;
    for (int32_t i = 0; i < k; ++i)
        if (sources[i] < 0 || sources[i] >= n || taus[i] < 0) return -1;
    adjacency out;
    if (build_adjacency(n, m, tail, &out)) { free_adjacency(&out); return -1; }
    int32_t** lists = (int32_t**)calloc((size_t)k + 1, sizeof(int32_t*));
    int64_t* counts = (int64_t*)calloc((size_t)k + 1, sizeof(int64_t));
    int failed = 0;
    if (threads < 1) threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
    for (int32_t i = 0; i < k; ++i) {
        int32_t* dist = out_dist ? out_dist + (size_t)i * n : (int32_t*)malloc((size_t)n * 4);
        if (!dist || tau_dijkstra(n, &out, tail, head, len, sources[i], taus[i], dist) < 0) {
            failed = 1;
        } else {
            int64_t c = orc_isochrone_scan(m, tail, head, dist, taus[i], NULL, 0);
            lists[i] = (int32_t*)malloc(((size_t)c + 1) * sizeof(int32_t));
            if (!lists[i]) failed = 1;
            else counts[i] = orc_isochrone_scan(m, tail, head, dist, taus[i], lists[i], c);
        }
        if (!out_dist) free(dist);
    }
    int64_t total = 0;
    out_off[0] = 0;
    for (int32_t i = 0; i < k; ++i) { total += counts[i]; out_off[i + 1] = total; }
    if (!failed && total <= cap)
        for (int32_t i = 0; i < k; ++i)
            if (counts[i]) memcpy(out_arcs + out_off[i], lists[i], (size_t)counts[i] * 4);
    for (int32_t i = 0; i < k; ++i) free(lists[i]);
    free(lists); free(counts); free_adjacency(&out);
    return failed ? -1 : total;
}
