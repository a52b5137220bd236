/*
 * iso.h -- C ABI of the GB300 isochrone library (libiso.so).
 *
 * An isochrone query (Baum, Buchhold, Dibbelt, Wagner, "Fast Computation of
 * Isochrones in Road Networks", Section 3) takes a source s and a time limit
 * tau and returns the isochrone edges: every arc (u,v) of the input graph with
 * exactly one endpoint in range, where v is in range iff d(s,v) <= tau.
 *
 * The library answers it PHAST-style (Section 2): a contraction hierarchy (CH)
 * is built once on the host (iso_build_ch); a query runs an upward CH search
 * from s, then one sweep over all vertices in descending CH level in which each
 * vertex takes the minimum over its incoming downward arcs, pruned at tau, and
 * finally a pass that emits the arcs whose endpoints are on different sides of
 * tau.  k queries share one sweep ("lanes").
 *
 * Conventions for every call:
 *   - vertices are 0..n-1, arcs are identified by their input index 0..m-1;
 *   - lengths and limits are int32 >= 0, in the same unit;
 *   - a distance label is d(s,v) if v is in range and 0x7FFFFFFF otherwise;
 *   - every call returns an ISO_* status; nothing throws across the ABI; the
 *     calling thread's last error message is available from iso_last_error();
 *   - objects (iso_ch, iso_graph, iso_workspace) are owned by the library and
 *     released with the matching iso_free_* call; input arrays are borrowed
 *     only for the duration of the call; output arrays belong to the caller.
 */
#ifndef ISO_H
#define ISO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ISO_OK          0
#define ISO_E_INVAL     1  /* bad argument (null pointer, id out of range, negative length/limit, ...) */
#define ISO_E_NOMEM     2  /* host or device allocation failed */
#define ISO_E_OVERFLOW  3  /* output capacity too small; offsets hold the sizes needed */
#define ISO_E_CUDA      4  /* a CUDA runtime call or kernel launch failed */
#define ISO_E_TIMEOUT   5  /* a device-side wait (grid barrier or dependency flag) gave up; results are invalid */
#define ISO_E_IO        6  /* file could not be read or written, or is not a CH file */
#define ISO_E_NODEV     7  /* no usable CUDA device (the library never falls back to the CPU) */

#define ISO_DIST_INF 0x7FFFFFFF

typedef struct iso_ch iso_ch;               /* host contraction hierarchy */
typedef struct iso_graph iso_graph;         /* device-resident copy of a CH */
typedef struct iso_workspace iso_workspace; /* per-batch device buffers + stream state */

/* ---------------------------------------------------------------------------
 * Contraction hierarchy (Section 2: vertices are contracted in an order rank,
 * shortcuts preserve distances, and levels satisfy l(v) = max(l(v), l(u)+1)
 * for every neighbour v still present when u is contracted).
 * ------------------------------------------------------------------------- */

typedef struct {
    int32_t threads;              /* host threads for contraction; 0 = all available */
    int32_t witness_settle_limit; /* vertices a witness search may settle; 0 = default (400) */
    int32_t priority_settle_limit;/* > 2: priorities count shortcuts with witness searches of
                                     this many settled vertices; 0 = default: witnesses of at
                                     most two arcs (cheaper, slightly larger hierarchy) */
    int32_t reserved[5];          /* must be zero */
} iso_ch_opts;

typedef struct {
    int32_t n;          /* vertices */
    int32_t levels;     /* number of CH levels L */
    int64_t m;          /* original arcs */
    int64_t m_up;       /* arcs of the upward graph (original + shortcuts, rank increasing) */
    int64_t m_down;     /* arcs of the downward graph (rank decreasing) */
    int64_t shortcuts;  /* shortcut arcs added by contraction */
    int32_t max_weight; /* largest input length */
    int32_t max_level_width; /* vertices in the widest level */
    double  build_seconds;
} iso_ch_stats;

/* Build a CH of the directed graph with n vertices and m arcs (tail[e] ->
 * head[e], length weight[e]).  Arrays are host memory and are copied.
 * Parallel arcs and self-loops are accepted.  Errors: ISO_E_INVAL for n <= 0,
 * m < 0, null arrays with m > 0, endpoints outside [0,n), negative lengths, or
 * a graph whose downward arc count exceeds 2^32-1; ISO_E_NOMEM. */
int iso_build_ch(int32_t n, int64_t m, const int32_t* tail, const int32_t* head,
                 const int32_t* weight, const iso_ch_opts* opts /* nullable */, iso_ch** out);

int  iso_ch_info(const iso_ch* ch, iso_ch_stats* out);
/* Write / read a CH in the library's own binary format (little-endian, with a
 * magic header and sizes).  Loading validates sizes and ids; ISO_E_IO otherwise. */
int  iso_save_ch(const iso_ch* ch, const char* path);
int  iso_load_ch(const char* path, iso_ch** out);
/* Read-only views of the CH arrays, valid until iso_free_ch.  Sweep order is
 * descending level; level_off[j]..level_off[j+1] holds level L-1-j.  Downward
 * arcs are listed at their head, upward arcs at their tail, original arcs at
 * their tail; all vertex ids in the arrays are sweep positions. */
typedef struct {
    const int32_t* perm;      /* [n] sweep position -> original id */
    const int32_t* pos;       /* [n] original id -> sweep position */
    const int32_t* level_off; /* [L+1] */
    const int64_t* down_off;  /* [n+1] */
    const int32_t* down_src;  /* [m_down] */
    const int32_t* down_w;    /* [m_down] */
    const int64_t* up_off;    /* [n+1] */
    const int32_t* up_dst;    /* [m_up] */
    const int32_t* up_w;      /* [m_up] */
    const int64_t* orig_off;  /* [n+1] */
    const int32_t* orig_head; /* [m] */
    const int32_t* orig_id;   /* [m] input arc index */
    const int32_t* bfs;       /* [n] BFS rank of each sweep position in the undirected input graph */
} iso_ch_view;
int  iso_ch_view_arrays(const iso_ch* ch, iso_ch_view* out);
/* Position of original vertex v in sweep order (descending level), or -1. */
int32_t iso_ch_sweep_position(const iso_ch* ch, int32_t v);
void iso_free_ch(iso_ch* ch);

/* ---------------------------------------------------------------------------
 * Device graph.
 * ------------------------------------------------------------------------- */

/* Device memory comes from these callbacks (the Python binding backs them with
 * PyTorch's caching allocator).  alloc returns NULL on failure; free accepts
 * what alloc returned.  stream is the cudaStream_t the memory is used on. */
typedef struct {
    void* (*alloc)(void* ctx, size_t bytes, void* stream);
    void  (*free)(void* ctx, void* ptr, void* stream);
    void* ctx;
} iso_alloc;

/* Copy the CH to the current CUDA device as sweep-ordered CSRs (Section 2:
 * vertices are renumbered so that the scan reads one array of arcs from front
 * to back).  alloc may be NULL, in which case
 * cudaMalloc/cudaFree are used.  The iso_ch may be freed
 * afterwards.  Errors: ISO_E_INVAL, ISO_E_NOMEM, ISO_E_CUDA, ISO_E_NODEV. */
int iso_upload_graph(const iso_ch* ch, const iso_alloc* alloc, void* stream, iso_graph** out);
void iso_free_graph(iso_graph* g);  /* after every workspace created on g (iso_free_workspace) */

/* Landmarks for restricted sweeps: picks `count` far-apart vertices and stores,
 * on the device, every vertex's distance from and to each of them (two PHAST
 * queries per landmark on the host, over `ch`, which must be the hierarchy g
 * was uploaded from).  A sweep then skips a chunk when, for every query,
 * max over landmarks L of (d(L,v) - d(L,s), d(s,L) - d(v,L)) -- a lower bound
 * on d(s,v) by the triangle inequality -- exceeds the query's limit for every
 * vertex v of the chunk.  Device memory: 8 * count * n bytes.  Calling it again
 * replaces the landmarks; it is refused with ISO_E_INVAL while a workspace
 * created with restrict_sweep exists (such a workspace keeps using the current
 * ones; iso_query's own workspaces are dropped and made again).  Errors:
 * ISO_E_INVAL (count outside 1..ISO_MAX_LANDMARKS, another hierarchy,
 * restricted workspaces alive), ISO_E_NOMEM, ISO_E_CUDA. */
#define ISO_MAX_LANDMARKS 16
int iso_graph_add_landmarks(iso_graph* g, const iso_ch* ch, int32_t count);
/* The same landmarks and distances on the host (no device needed): vertices[i]
 * is landmark i's original vertex id; fwd[i*n + v] = d(L_i, v) and
 * bwd[i*n + v] = d(v, L_i) for original vertex v, 0xFFFFFFFF where there is
 * no path (0xFFFFFFFE: a distance that does not fit 32 bits).  Arrays are
 * caller-owned: vertices[count], fwd and bwd [count * n]. */
int iso_ch_landmarks(const iso_ch* ch, int32_t count, int32_t* vertices, uint32_t* fwd, uint32_t* bwd);

/* ---------------------------------------------------------------------------
 * Queries.
 * ------------------------------------------------------------------------- */

typedef struct {
    int32_t threads_per_vertex; /* sweep threads per vertex (each owns K/threads lanes); 0 = auto */
    int32_t ctas_per_sm;        /* persistent sweep CTAs per SM; 0 = auto (occupancy) */
    int32_t fuse_width;         /* narrow-level threshold.  Plain sweep: levels with fewer vertices
                                   run in one CTA between grid barriers.  TMA-staged sweep: the
                                   leading levels with fewer vertices are swept level by level with
                                   a grid barrier each before the chunk schedule starts (0 = auto:
                                   one chunk per CTA), later ones get a warp per vertex.
                                   -1 = never */
    int32_t use_cuda_graph;     /* 1 = capture the launch sequence once per workspace and replay */
    int64_t barrier_timeout_ns; /* give up a device-side wait (grid barrier, dependency flag, copy)
                                   after this long without progress; 0 = 2 s */
    int32_t debug_barrier_extra;/* testing only: the sweep's barriers and dependency checks wait
                                   for this many extra arrivals or flags that never come, so the
                                   sweep times out */
    int32_t sweep_kernel;       /* 0 = auto (TMA-staged arc blocks), 1 = TMA-staged, 2 = plain loads */
    int32_t record_trace;       /* 1 = record the device time of every sweep step (iso_workspace_trace) */
    int32_t schedule_delay;     /* TMA-staged sweep: a chunk is scheduled at least this many positions
                                   after the chunks it depends on; 0 = auto (three times the CTA count) */
    int32_t solo_width;         /* TMA-staged sweep: the top levels of the hierarchy, as long as each
                                   has at most this many vertices, run in one CTA level by level
                                   (CTA barriers instead of flags between CTAs); 0 = auto (124),
                                   -1 = never */
    int32_t chunk_span;         /* TMA-staged sweep: a chunk also ends where the BFS rank of its next
                                   vertex is this far or more above its first one's, so that chunks
                                   of sparse levels cover small parts of the map; 0 = no limit */
    int32_t core_vertices;      /* TMA-staged sweep: the top level blocks of the hierarchy, as long as
                                   they hold at most this many vertices in total, are swept for each
                                   lane by one CTA with the lane's labels in shared memory (Section 5's
                                   small top graph swept first); 0 = auto (the most that fit, 53,248),
                                   -1 = never */
    int32_t debug_stage_arcs;   /* testing only (TMA-staged sweep): stage at most this many arcs per
                                   chunk in shared memory (0 = the buffer size, 3,072); chunks with
                                   more read their arcs from global memory */
    int32_t debug_stage_deps;   /* testing only: likewise for dependency-list entries (0 = 128) */
    int32_t restrict_sweep;     /* TMA-staged sweep: 1 = skip the chunks that landmark lower bounds show
                                   to be out of range for every query of the batch (Section 2's
                                   restricted scan, Section 5's active cells); needs
                                   iso_graph_add_landmarks; 0 = sweep everything */
    int32_t fused_emission;     /* TMA-staged sweep: 1 = the sweep emits the isochrone edges itself
                                   (Section 5: each input arc is checked at its later-swept endpoint
                                   once that vertex is final), with no separate emission pass;
                                   0 = a separate pass over all arcs after the sweep */
    int32_t reserved[1];        /* must be zero */
} iso_query_opts;

/* Answer k isochrone queries (source sources[i], limit taus[i]) in sweeps of
 * up to 64 lanes.  sources/taus may be host or device memory (detected).
 * On success out_offsets[0..k] (host or device) holds list boundaries and
 * out_arcs[out_offsets[i] .. out_offsets[i+1]) the arc ids of query i in
 * ascending order.  out_dist (nullable; host or device) receives the labels,
 * query-major: out_dist[i*n + v] for original vertex v.  If the lists need
 * more than cap entries, out_offsets is filled with the needed offsets, nothing
 * is written to out_arcs, and ISO_E_OVERFLOW is returned.  Validation: k >= 0,
 * 0 <= sources[i] < n, 0 <= taus[i] <= 0x7FFFFFFE - max_weight.
 * The call returns after the results are in place (it synchronizes `stream`,
 * the cudaStream_t to run on; NULL = the legacy default stream). */
int iso_query(iso_graph* g, int32_t k, const int32_t* sources, const int32_t* taus,
              int64_t* out_offsets, int32_t* out_arcs, int64_t cap, int32_t* out_dist,
              const iso_query_opts* opts /* nullable */, void* stream);

/* Workspaces hold the per-batch device buffers for up to `lanes` queries
 * (lanes in 1..64) so that batches can be kept in flight on several streams. */
int iso_workspace_create(iso_graph* g, int32_t lanes, const iso_query_opts* opts /* nullable */,
                         void* stream, iso_workspace** out);
/* Enqueue one batch of k <= lanes queries on `stream` and return without
 * waiting for the device.  sources/taus: host or device memory (detected);
 * host values are validated here, device values by the first kernel (a bad one
 * makes iso_collect return ISO_E_INVAL).  flags: ISO_SUBMIT_DIST to also keep
 * the labels for iso_collect's out_dist.  A workspace holds one batch at a
 * time: collect before submitting again. */
#define ISO_SUBMIT_DIST 1
int iso_submit(iso_workspace* ws, int32_t k, const int32_t* sources, const int32_t* taus, int32_t flags,
               void* stream);
/* iso_submit whose batch starts only once the sweep of the batch last
 * submitted on `after` (another workspace of the same graph; NULL = no wait)
 * has finished.  Chaining each batch to the one before lets batches on
 * several workspaces take the GPU one sweep after another -- the sweep holds
 * every SM -- while the next batch's upward search and core overlap the
 * previous batch's emission and sort, instead of contending with its sweep.
 * The wait is enqueued on `stream` before the batch. */
int iso_submit_after(iso_workspace* ws, const iso_workspace* after, int32_t k, const int32_t* sources,
                     const int32_t* taus, int32_t flags, void* stream);
/* Wait for the batch last submitted on ws and copy its results as iso_query
 * does (same layout, overflow and distance conventions). */
int iso_collect(iso_workspace* ws, int64_t* out_offsets, int32_t* out_arcs, int64_t cap,
                int32_t* out_dist);
/* Vertices in range (Section 3 names this as another output the problem can
 * ask for) of the batch last collected on ws: for query i, bit v of the
 * bitset out_bits[i * words_per_query .. + ceil(n/32)) (32-bit words, bit v
 * = bit v % 32 of word v / 32, v an original vertex id) is set iff
 * d(sources[i], v) <= taus[i].  out_bits is host or device memory (detected);
 * words_per_query >= ceil(n/32); words beyond ceil(n/32) are not written.
 * Valid after iso_collect returned ISO_OK or ISO_E_OVERFLOW and before the
 * next iso_submit on ws; synchronizes the workspace's stream.  Errors:
 * ISO_E_INVAL (nothing collected, NULL or short buffer), ISO_E_NOMEM,
 * ISO_E_CUDA. */
int iso_collect_range(iso_workspace* ws, uint32_t* out_bits, int64_t words_per_query);
/* Per-phase device times of the last collected batch in milliseconds:
 * [0] upward search, [1] sweep, [2] emission, [3] sort + gather. */
int iso_workspace_timings(const iso_workspace* ws, float* ms4);
/* Per-level times of the last collected batch (workspaces created with
 * record_trace = 1 and the TMA-staged sweep).  Entry i < L: steps4[4i..4i+3] =
 * {0, i, i+1, 0} and ns[i] = device nanoseconds from the start of the sweep
 * until level block i was complete (blocks in sweep order, block 0 = top
 * level; below the leading levels the sweep interleaves levels, so these need
 * not grow).  Entry L: steps4 = {2, 0, 0, 0} and ns[L] = time before the walk
 * over the levels starts (0: the upward search writes its labels straight into
 * the label rows).  Returns L+1 (at most cap entries are written) or -1 on
 * error. */
int32_t iso_workspace_trace(const iso_workspace* ws, int32_t* steps4, int64_t* ns, int32_t cap);
/* Shape of a workspace's sweep on its graph (TMA-staged sweep; zeros for the
 * plain one): how the level blocks are split between the phases and the chunk
 * schedule's extremes against the shared-memory staging limits. */
typedef struct {
    int32_t levels;              /* level blocks L */
    int32_t core_levels;         /* blocks 0 .. core_levels-1: per-lane core */
    int32_t core_vertices;       /* vertices in those blocks */
    int32_t solo_levels;         /* blocks core_levels .. solo_levels-1: CTA 0 alone */
    int32_t sync_levels;         /* blocks solo_levels .. sync_levels-1: grid-synchronous */
    int32_t chunks;              /* chunks of the schedule (blocks sync_levels .. L-1) */
    int32_t max_chunk_arcs;      /* largest arc block of a chunk */
    int32_t max_chunk_deps;      /* longest dependency list of a chunk */
    int32_t chunks_over_arc_cap; /* chunks whose arcs are read from global memory */
    int32_t chunks_over_dep_cap; /* chunks whose dependency list is checked in global memory */
    int32_t arc_cap, dep_cap;    /* staging limits in force */
    int32_t reserved[4];
} iso_sweep_info;
int iso_workspace_sweep_info(const iso_workspace* ws, iso_sweep_info* out);
/* Chunks the last collected batch skipped (restricted sweep; 0 otherwise). */
int iso_workspace_skipped_chunks(const iso_workspace* ws, int64_t* out);
/* Waits for the workspace's stream and frees its device buffers (into the
 * graph's allocator).  Free every workspace before the graph it was created
 * on: iso_free_graph frees only the workspaces iso_query made for itself. */
void iso_free_workspace(iso_workspace* ws);

/* ---------------------------------------------------------------------------
 * Allocation-free query (the paper has no counterpart; this is a library
 * service).  For callers that cannot allocate device memory while answering a
 * query -- a process whose device memory is fully reserved by another
 * framework's pool, a latency-critical thread that must not wait on allocator
 * locks or on the device-wide synchronisation a cudaFree can imply, a host that
 * forbids allocation after start-up.  It runs the same kernels as iso_query on
 * slices of one fixed static device array of ISO_NOALLOC_SCRATCH_BYTES bytes,
 * which every GPU that loads the library holds until the process exits, and
 * calls no allocator (CUDA's, PyTorch's or any other).
 *
 * Limits (larger requests return ISO_E_INVAL with a message): k <=
 * ISO_NOALLOC_MAX_QUERIES, a graph of at most ISO_NOALLOC_MAX_VERTICES vertices
 * and 4096 CH levels, at most ISO_NOALLOC_MAX_ARCS isochrone edges and 8192
 * upward-search vertices per query.  Inputs, outputs, overflow and errors are
 * as for iso_query (without out_dist).  g must live on the current device
 * (ISO_E_INVAL otherwise).  The first call on each device looks up
 * the array's device address, so make it before any stream capture on that
 * device.  All calls share the array: calls that overlap on the GPU (two
 * streams or two host threads at once) race and must be serialised by the
 * caller.  The call synchronizes `stream` before returning, on failure too
 * once anything was enqueued, so a failed call never leaves work running on
 * the array.
 * ------------------------------------------------------------------------- */
#define ISO_NOALLOC_MAX_VERTICES (1 << 20)
#define ISO_NOALLOC_MAX_QUERIES 4
#define ISO_NOALLOC_MAX_ARCS 65536
#define ISO_NOALLOC_SCRATCH_BYTES 23921408
int iso_query_noalloc(iso_graph* g, int32_t k, const int32_t* sources, const int32_t* taus,
                      int64_t* out_offsets, int32_t* out_arcs, int64_t cap, void* stream);

/* Message describing the last error on the calling thread ("" if none). */
const char* iso_last_error(void);
/* Library version string. */
const char* iso_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ISO_H */
