// C ABI: device upload, workspaces, batched submission and result collection.
//
// A batch of up to K lanes runs as one fixed launch sequence on the caller's
// stream (optionally captured once into a CUDA graph and replayed):
//   memset control block -> k_upward (one CTA per lane) -> k_sweep (persistent,
//   cooperative) -> k_emit -> k_sort_gather [-> k_dist] -> copy summary to host.
// Collecting waits for the summary, grows internal buffers and replays the
// batch if an upward search or an emission list outgrew them, then copies the
// lists (and labels) to the caller.  No step falls back to the CPU: without a
// device every call returns ISO_E_NODEV.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "ch_internal.h"
#include "iso_device.cuh"
#include "sweep_schedule.h"
#include "../../include/iso.h"
#include "graph_view.h"
#include "landmarks.h"

namespace {

using namespace isod;

int cuda_status(cudaError_t e) {
    return e == cudaErrorMemoryAllocation ? ISO_E_NOMEM
         : (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) ? ISO_E_NODEV
         : ISO_E_CUDA;
}

#define ISO_CK(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            iso::set_error("%s failed: %s", #call, cudaGetErrorString(e_));                   \
            return cuda_status(e_);                                                           \
        }                                                                                     \
    } while (0)

struct Allocator {
    iso_alloc cb{};
    bool custom = false;
    void* get(size_t bytes, cudaStream_t s) {
        if (bytes == 0) bytes = 16;
        bytes = (bytes + 255) & ~(size_t)255;
        if (custom) return cb.alloc(cb.ctx, bytes, s);
        void* p = nullptr;
        return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
    }
    void put(void* p, cudaStream_t s) {
        if (!p) return;
        if (custom) cb.free(cb.ctx, p, s);
        else cudaFree(p);
    }
};

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

constexpr int kMaxLanes = 64;
// default size limit of the top levels that CTA 0 sweeps alone in the TMA
// sweep (four vertices per consumer warp)
constexpr int kSoloWidth = 124;

int lanes_class(int k) {
    if (k <= 1) return 1;
    for (int K : {4, 8, 16, 32, 64})
        if (k <= K) return K;
    return 64;
}

int default_tpv(int K) { return K <= 8 ? 1 : K / 8; }

// Largest per-lane core (vertices) that options o allow on a graph of n vertices.
int core_limit_of(const iso_query_opts& o, int n) {
    if (o.core_vertices < 0) return 0;
    const int lim = o.core_vertices > 0 ? std::min(o.core_vertices, kCoreMaxVertices) : kCoreMaxVertices;
    return std::min(lim, n);
}

// Sweep kernel, threads per vertex, CTAs per SM and vertices per CTA batch that
// options o select for K lanes.  Returns false if the combination is unsupported.
bool sweep_shape(int K, const iso_query_opts& o, int* kernel, int* tpv, int* occ, int* vpb) {
    *kernel = o.sweep_kernel == 2 ? 2 : 1;
    *tpv = o.threads_per_vertex ? o.threads_per_vertex : default_tpv(K);
    int block = 0;
    if (*kernel == 1) {
        if (!iso_sweep_tma_supported(K, *tpv)) return false;
        *occ = iso_sweep_tma_occupancy(K, *tpv, &block, vpb);
    } else {
        if (!iso_sweep_supported(K, *tpv)) return false;
        *occ = iso_sweep_occupancy(K, *tpv, &block);
        *vpb = block / *tpv;
    }
    return *occ > 0;
}

}  // namespace

struct iso_graph {
    int device = 0;
    int n = 0, L = 0, max_w = 0, tau_max = 0, num_sms = 0;
    int64_t m = 0, m_down = 0, m_up = 0;
    Allocator A;
    cudaStream_t stream = nullptr;
    uint32_t* down_off = nullptr;
    int2* down_arc = nullptr;
    uint32_t* up_off = nullptr;
    int2* up_arc = nullptr;
    // input arcs grouped by tail, tails in BFS order of the input graph (so
    // that emission reads the masks of neighbouring vertices close in time)
    uint32_t* orig_off = nullptr;   // [n+1] by emission index
    int32_t* orig_head = nullptr;   // heads as sweep positions
    int32_t* orig_id = nullptr;     // input arc ids
    int32_t* emit_tail = nullptr;   // [n] sweep position of the tail at each emission index
    // per-lane core of the TMA sweep: downward arcs into the first
    // core_cap_n sweep positions packed as {src | head << 16, len}, and the
    // first downward arc of every level block
    uint2* core_arc = nullptr;
    uint32_t* level_arc = nullptr;
    int core_cap_n = 0;
    // fused emission: input arcs by their later-swept endpoint {other endpoint, arc id}
    uint32_t* emit_off = nullptr;   // [n+1]
    int2* emit_ent = nullptr;
    int64_t dummy_arcs = 0;         // dummy downward arcs added for one-way input arcs
    // landmark distances for restricted sweeps (iso_graph_add_landmarks)
    LandmarkSet lm;
    uint32_t* lm_fwd = nullptr;
    uint32_t* lm_bwd = nullptr;
    std::atomic<int> restricted_ws{0};  // live workspaces with restricted sweeps (they use lm_*)
    int32_t* perm = nullptr;
    int32_t* pos = nullptr;
    int32_t* level_off = nullptr;
    std::vector<int32_t> h_level_off;
    // host copies for building sweep schedules
    std::vector<uint32_t> h_down_off;
    std::vector<int32_t> h_down_src, h_bfs;
    struct CachedSchedule {
        int vpb, narrow_width, sync_levels, delay, chunk_span;
        std::shared_ptr<SweepSchedule> s;
    };
    std::vector<CachedSchedule> schedules;
    std::mutex mu;
    iso_workspace* query_ws[7] = {};
    std::vector<void*> owned;

    template <class T>
    int upload(T** dst, const T* src, size_t count) {
        *dst = (T*)A.get(count * sizeof(T), stream);
        if (!*dst) { iso::set_error("iso_upload_graph: device allocation of %zu bytes failed", count * sizeof(T)); return ISO_E_NOMEM; }
        owned.push_back(*dst);
        if (count) ISO_CK(cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, stream));
        return ISO_OK;
    }
};

struct iso_workspace {
    iso_graph* g = nullptr;
    int K = 0, tpv = 0, grid = 0, fuse_width = 0;
    int kernel = 1;              // 1 = TMA-staged sweep, 2 = plain loads
    int narrow_width = 0;        // TMA sweep: levels narrower than this use a warp per vertex
    int sched_delay = 0;         // TMA sweep: schedule distance to dependencies
    int solo_width = 0;          // TMA sweep: top levels up to this size run in one CTA (0: none)
    int solo_levels = 0;         // ... how many levels that is on this graph
    int sync_levels = 0;         // TMA sweep: leading levels swept level by level before the schedule
    int chunk_span = 0;          // TMA sweep: largest BFS-rank span of a chunk (0: no limit)
    int core_limit = 0;          // TMA sweep: largest per-lane core (vertices; 0: none)
    int core_levels = 0, core_n = 0;  // ... the level blocks and vertices it covers on this graph
    int stage_arc_cap = 0, stage_pred_cap = 0;  // testing: lower staging limits (0: buffer sizes)
    bool restrict_sweep = false;  // skip chunks out of range for every lane (landmark bounds)
    bool fused_emit = false;      // the sweep emits the isochrone edges (no k_emit)
    uint32_t* chunk_lo = nullptr;  // [Q * landmarks] per-chunk bounds (restricted sweep)
    uint32_t* chunk_hi = nullptr;
    uint8_t* skip = nullptr;       // [Q] per batch
    int64_t skipped = 0;           // chunks skipped by the last collected batch
    iso_sweep_info info{};       // the sweep's shape (iso_workspace_sweep_info)
    bool record_trace = false;
    long long* trace = nullptr;  // device [nsched + 1]
    std::vector<long long> h_trace;
    std::vector<int4> h_sched;
    bool use_graph = false;
    long long timeout_ns = 2000000000LL;
    int bar_extra = 0;
    cudaStream_t stream = nullptr;  // stream of the last submit
    // device buffers
    uint32_t* d = nullptr;
    void* mask = nullptr;
    uint8_t* upflag = nullptr;
    int32_t* io = nullptr;       // src[K], tau[K]
    int32_t* ctl = nullptr;      // status[4], bar[2], pad[2], ecnt[K], upcnt[K]
    int4* sched_info = nullptr;    // [2Q] TMA sweep schedule: one SchedChunk per position
    int32_t* pred = nullptr;       // dependency lists (padded, see sweep_schedule.h)
    int32_t* done = nullptr;       // [Q] zeroed per batch
    int Q = 0;
    unsigned long long* upmask = nullptr;  // [n] TMA sweep: lanes with upward labels
    uint32_t* core_out = nullptr;  // [K * core_n] TMA sweep: the per-lane core's labels, lane-major
    int vpb = 0;
    int2* pairs = nullptr;
    uint32_t* gtab = nullptr;
    int gcap = 1 << 14;
    int32_t* ebuf = nullptr;
    int32_t* tmp = nullptr;
    int ecap = 1 << 15;
    int32_t* out = nullptr;
    int64_t* out_off = nullptr;
    int4* sched = nullptr;
    int nsched = 0;
    int32_t* dist = nullptr;     // [K * n] labels, query-major, original vertex order
    uint32_t* range = nullptr;   // [K * ceil(n/32)] vertices-in-range bitsets (iso_collect_range)
    bool collected = false;      // the last batch was collected successfully
    // pinned host mirrors
    int32_t* h_io = nullptr;     // src[K], tau[K]
    int32_t* h_ctl = nullptr;    // ctl after the last batch
    // state of the last batch
    int k = 0;
    bool want_dist = false;
    bool submitted = false;
    // a failed batch can stop the sweep before it clears every upward-label
    // flag; the next batch then starts by clearing them all
    bool stale_flags = false;
    float phase_ms[4] = {};
    cudaEvent_t ev[6] = {};
    cudaEvent_t ev_swept = nullptr;  // recorded right after the sweep of each batch (iso_submit_after)
    cudaGraphExec_t gexec[2] = {};  // indexed by want_dist
    bool graph_failed = false;
    std::vector<void*> owned;

    int32_t* src() { return io; }
    int32_t* tau() { return io + K; }
    int32_t* status() { return ctl; }
    uint32_t* bar() { return (uint32_t*)(ctl + 4); }
    int32_t* ecnt() { return ctl + 8; }
    int32_t* upcnt() { return ctl + 8 + K; }
    size_t ctl_words() const { return 8 + 2 * (size_t)K; }

    void* alloc(size_t bytes) {
        void* p = g->A.get(bytes, stream);
        if (p) owned.push_back(p);
        return p;
    }
    void release(void*& p) {
        if (!p) return;
        owned.erase(std::remove(owned.begin(), owned.end(), p), owned.end());
        g->A.put(p, stream);
        p = nullptr;
    }
    void drop_graphs() {
        for (auto& x : gexec)
            if (x) { cudaGraphExecDestroy(x); x = nullptr; }
    }
};

namespace {

int build_schedule(iso_workspace* ws) {
    iso_graph* g = ws->g;
    std::vector<int4> steps;
    for (int j = 0; j < g->L;) {
        const int w = g->h_level_off[j + 1] - g->h_level_off[j];
        if (ws->fuse_width > 0 && w < ws->fuse_width) {
            int j1 = j + 1;
            while (j1 < g->L && g->h_level_off[j1 + 1] - g->h_level_off[j1] < ws->fuse_width) ++j1;
            steps.push_back(make_int4(kStepFused, j, j1, 0));
            j = j1;
        } else {
            steps.push_back(make_int4(kStepWide, j, j + 1, 0));
            ++j;
        }
    }
    ws->nsched = (int)steps.size();
    ws->h_sched = steps;
    ws->sched = (int4*)ws->alloc(steps.size() * sizeof(int4));
    if (!ws->sched) { iso::set_error("workspace: device allocation failed"); return ISO_E_NOMEM; }
    ISO_CK(cudaMemcpyAsync(ws->sched, steps.data(), steps.size() * sizeof(int4), cudaMemcpyHostToDevice,
                           ws->stream));
    if (ws->kernel == 1) {
        // TMA sweep: locality-ordered chunk schedule, cached on the graph
        const int delay = ws->sched_delay;
        // The leading levels sweep level by level before the schedule: those
        // with at most solo_width vertices in CTA 0 alone, the following ones
        // narrower than narrow_width in all CTAs with a grid barrier per level.
        // The per-lane core: the longest run of top level blocks whose vertices
        // fit core_limit (it replaces the CTA-0-alone levels).
        int core = 0;
        while (core < g->L && core < kCoreMaxLevels && g->h_level_off[core + 1] <= ws->core_limit) ++core;
        ws->core_levels = core;
        ws->core_n = g->h_level_off[core];
        int solo = core;
        while (core == 0 && ws->solo_width > 0 && solo < g->L &&
               g->h_level_off[solo + 1] - g->h_level_off[solo] <= ws->solo_width)
            ++solo;
        int sync = solo;
        while (sync < g->L && g->h_level_off[sync + 1] - g->h_level_off[sync] < ws->narrow_width) ++sync;
        ws->solo_levels = solo;
        ws->sync_levels = sync;
        static_assert(sizeof(SchedChunk) == 2 * sizeof(int4), "schedule record layout");
        std::shared_ptr<SweepSchedule> sc;
        for (auto& c : g->schedules)
            if (c.vpb == ws->vpb && c.narrow_width == ws->narrow_width && c.sync_levels == sync && c.delay == delay &&
                c.chunk_span == ws->chunk_span)
                sc = c.s;
        if (!sc) {
            sc = std::make_shared<SweepSchedule>();
            if (iso_make_schedule(g->n, g->L, g->h_level_off.data(), g->h_down_off.data(), g->h_down_src.data(),
                                  g->h_bfs.data(), ws->vpb, 31, ws->narrow_width, sync, delay, ws->chunk_span,
                                  sc.get()) != 0) {
                iso::set_error("workspace: could not build the sweep schedule");
                return ISO_E_INVAL;
            }
            g->schedules.push_back({ws->vpb, ws->narrow_width, sync, delay, ws->chunk_span, sc});
        }
        ws->Q = sc->Q;
        {
            iso_sweep_info& in = ws->info;
            in.levels = g->L;
            in.core_levels = core;
            in.core_vertices = ws->core_n;
            in.solo_levels = solo;
            in.sync_levels = sync;
            in.chunks = sc->Q;
            int acap = 0, dcap = 0;
            iso_sweep_tma_stage_caps(&acap, &dcap);
            if (ws->stage_arc_cap > 0 && ws->stage_arc_cap < acap) acap = ws->stage_arc_cap;
            if (ws->stage_pred_cap > 0 && ws->stage_pred_cap < dcap) dcap = ws->stage_pred_cap;
            in.arc_cap = acap;
            in.dep_cap = dcap;
            for (const SchedChunk& c : sc->info) {
                in.max_chunk_arcs = std::max(in.max_chunk_arcs, c.na);
                in.max_chunk_deps = std::max(in.max_chunk_deps, c.np);
                in.chunks_over_arc_cap += c.na > acap;
                in.chunks_over_dep_cap += c.np > dcap;
            }
        }
        ws->sched_info = (int4*)ws->alloc(std::max<size_t>(sc->Q, 1) * sizeof(SchedChunk));
        ws->pred = (int32_t*)ws->alloc(sc->pred.size() * 4);
        ws->done = (int32_t*)ws->alloc(std::max<size_t>(sc->Q, 1) * 4);
        if (!ws->sched_info || !ws->pred || !ws->done) {
            iso::set_error("workspace: device allocation failed");
            return ISO_E_NOMEM;
        }
        if (sc->Q)
            ISO_CK(cudaMemcpyAsync(ws->sched_info, sc->info.data(), (size_t)sc->Q * sizeof(SchedChunk),
                                   cudaMemcpyHostToDevice, ws->stream));
        ISO_CK(cudaMemcpyAsync(ws->pred, sc->pred.data(), sc->pred.size() * 4, cudaMemcpyHostToDevice, ws->stream));
        if (ws->restrict_sweep) {
            // per-chunk landmark bounds in schedule order
            const int c = g->lm.count;
            std::vector<uint32_t> lo(std::max<size_t>((size_t)sc->Q * c, 1)), hi(lo.size());
            for (int q = 0; q < sc->Q; ++q)
                iso_landmark_chunk_bounds(g->lm, g->n, sc->info[q].v0, sc->info[q].v1, lo.data() + (size_t)q * c,
                                          hi.data() + (size_t)q * c);
            ws->chunk_lo = (uint32_t*)ws->alloc(lo.size() * 4);
            ws->chunk_hi = (uint32_t*)ws->alloc(hi.size() * 4);
            ws->skip = (uint8_t*)ws->alloc(std::max<size_t>(sc->Q, 1));
            if (!ws->chunk_lo || !ws->chunk_hi || !ws->skip) {
                iso::set_error("workspace: device allocation failed");
                return ISO_E_NOMEM;
            }
            ISO_CK(cudaMemcpyAsync(ws->chunk_lo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice, ws->stream));
            ISO_CK(cudaMemcpyAsync(ws->chunk_hi, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice, ws->stream));
            ISO_CK(cudaStreamSynchronize(ws->stream));  // lo/hi are freed on return
        }
    }
    ISO_CK(cudaStreamSynchronize(ws->stream));
    return ISO_OK;
}

int alloc_up(iso_workspace* ws) {
    ws->pairs = (int2*)ws->alloc((size_t)ws->K * ws->gcap * sizeof(int2));
    ws->gtab = (uint32_t*)ws->alloc((size_t)ws->K * iso_upward_table_words(ws->gcap) * sizeof(uint32_t));
    if (!ws->pairs || !ws->gtab) { iso::set_error("workspace: device allocation failed"); return ISO_E_NOMEM; }
    return ISO_OK;
}

int alloc_emit(iso_workspace* ws) {
    const size_t cells = (size_t)ws->K * ws->ecap;
    ws->ebuf = (int32_t*)ws->alloc(cells * 4);
    ws->tmp = (int32_t*)ws->alloc(cells * 4);
    ws->out = (int32_t*)ws->alloc(cells * 4);
    if (!ws->ebuf || !ws->tmp || !ws->out) { iso::set_error("workspace: device allocation failed"); return ISO_E_NOMEM; }
    return ISO_OK;
}

// Timing events become event-record nodes when the sequence is captured.
cudaError_t record(cudaEvent_t e, cudaStream_t s, bool capturing) {
    return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

// The launch sequence of one batch on ws->stream; inputs are already in ws->io.
int enqueue(iso_workspace* ws, bool want_dist, bool capturing) {
    iso_graph* g = ws->g;
    cudaStream_t s = ws->stream;
    const int K = ws->K;
    ISO_CK(cudaMemsetAsync(ws->ctl, 0, ws->ctl_words() * 4, s));
    if (ws->done) ISO_CK(cudaMemsetAsync(ws->done, 0, (size_t)ws->Q * 4, s));
    if (ws->trace) ISO_CK(cudaMemsetAsync(ws->trace, 0, ((size_t)g->L + 2) * 8, s));
    ISO_CK(record(ws->ev[0], s, capturing));

    UpParams up{};
    up.up_off = g->up_off; up.up_arc = g->up_arc; up.pos = g->pos;
    up.src = ws->src(); up.tau = ws->tau();
    up.pairs = ws->pairs; up.cnt = ws->upcnt(); up.gtab = ws->gtab; up.status = ws->status();
    up.n = g->n; up.cap = ws->gcap; up.gcap = ws->gcap; up.tau_max = g->tau_max;
    up.direct = ws->kernel == 1 ? 1 : 0;
    up.core_n = ws->kernel == 1 ? ws->core_n : 0;
    up.K = K; up.d = ws->d; up.upmask = ws->upmask; up.upflag = ws->upflag;
    ISO_CK(iso_launch_upward(up, K, s));
    if (ws->skip && ws->Q > 0) {
        SkipParams sk{};
        sk.src = ws->src(); sk.tau = ws->tau(); sk.pos = g->pos; sk.lm_fwd = g->lm_fwd; sk.lm_bwd = g->lm_bwd;
        sk.chunk_lo = ws->chunk_lo; sk.chunk_hi = ws->chunk_hi; sk.skip = ws->skip; sk.skipped = ws->status() + 1;
        sk.n = g->n; sk.K = K; sk.Q = ws->Q; sk.count = g->lm.count;
        ISO_CK(iso_launch_skip(sk, g->num_sms, s));
    }
    ISO_CK(record(ws->ev[1], s, capturing));

    SweepParams sw{};
    sw.down_off = g->down_off; sw.down_arc = g->down_arc; sw.level_off = g->level_off;
    sw.sched = ws->sched; sw.pairs = ws->pairs; sw.cnt = ws->upcnt(); sw.tau = ws->tau();
    sw.d = ws->d; sw.mask = ws->mask; sw.upflag = ws->upflag; sw.bar = ws->bar(); sw.status = ws->status();
    sw.timeout_ns = ws->timeout_ns; sw.n = g->n; sw.L = g->L; sw.nsched = ws->nsched; sw.cap = ws->gcap;
    sw.last_level_block = g->L - 1; sw.write_all = want_dist ? 1 : 0; sw.bar_extra = ws->bar_extra;
    sw.trace = ws->trace;
    sw.sched_info = ws->sched_info;
    sw.pred = ws->pred;
    sw.done = ws->done;
    sw.solo_levels = ws->solo_levels;
    sw.sync_levels = ws->sync_levels;
    sw.Q = ws->Q;
    sw.upmask = ws->upmask;
    sw.core_levels = ws->core_levels;
    sw.core_n = ws->core_n;
    sw.core_arc = g->core_arc;
    sw.level_arc = g->level_arc;
    sw.core_out = ws->core_out;
    sw.stage_arc_cap = ws->stage_arc_cap;
    sw.stage_pred_cap = ws->stage_pred_cap;
    sw.skip = ws->skip;
    sw.fused_emit = ws->fused_emit ? 1 : 0;
    sw.emit_off = g->emit_off;
    sw.emit_ent = g->emit_ent;
    sw.ecnt = ws->ecnt();
    sw.ebuf = ws->ebuf;
    sw.ecap = ws->ecap;
    sw.sync_n = g->h_level_off[ws->sync_levels];
    if (ws->kernel == 1 && ws->core_levels > 0) ISO_CK(iso_launch_core(sw, K, s));
    if (ws->kernel == 1) ISO_CK(iso_launch_sweep_tma(sw, K, ws->tpv, ws->grid, s));
    else ISO_CK(iso_launch_sweep(sw, K, ws->tpv, ws->grid, s));
    ISO_CK(record(ws->ev[2], s, capturing));
    ISO_CK(record(ws->ev_swept, s, capturing));

    EmitParams em{};
    em.orig_off = g->orig_off; em.orig_head = g->orig_head; em.orig_id = g->orig_id; em.mask = ws->mask;
    em.tail_of = g->emit_tail;
    em.status = ws->status();
    em.ecnt = ws->ecnt(); em.ebuf = ws->ebuf; em.n = g->n; em.ecap = ws->ecap;
    // four 256-thread CTAs per SM: half an SM's threads, so that the next
    // batch's upward search (1024 threads per CTA) can be placed beside them
    // (with fused emission the sweep has emitted already)
    if (!ws->fused_emit) ISO_CK(iso_launch_emit(em, K, g->num_sms * 4, s));
    ISO_CK(record(ws->ev[3], s, capturing));

    GatherParams ga{};
    ga.ebuf = ws->ebuf; ga.ecnt = ws->ecnt(); ga.tmp = ws->tmp; ga.out = ws->out; ga.out_off = ws->out_off;
    ga.k = K; ga.ecap = ws->ecap;
    ga.status = ws->status();
    ga.key_bits = 1;
    while (ga.key_bits < 31 && (int64_t(1) << ga.key_bits) < g->m) ++ga.key_bits;
    ga.m = g->m;
    ISO_CK(iso_launch_sort_gather(ga, K, s));
    if (want_dist) {
        DistParams dp{};
        dp.d = ws->d; dp.perm = g->perm; dp.out = ws->dist; dp.n = g->n; dp.k = K; dp.K = K;
        ISO_CK(iso_launch_dist(dp, s));
    }
    ISO_CK(record(ws->ev[4], s, capturing));
    ISO_CK(cudaMemcpyAsync(ws->h_ctl, ws->ctl, ws->ctl_words() * 4, cudaMemcpyDeviceToHost, s));
    ISO_CK(record(ws->ev[5], s, capturing));
    return ISO_OK;
}

int launch_batch(iso_workspace* ws, bool want_dist) {
    if (ws->stale_flags) {
        ISO_CK(cudaMemsetAsync(ws->upflag, 0, (size_t)ws->g->n, ws->stream));
        if (ws->upmask) ISO_CK(cudaMemsetAsync(ws->upmask, 0, (size_t)ws->g->n * 8, ws->stream));
        ws->stale_flags = false;
    }
    if (want_dist && !ws->dist) {
        ws->dist = (int32_t*)ws->alloc((size_t)ws->K * ws->g->n * 4);
        if (!ws->dist) { iso::set_error("workspace: device allocation failed"); return ISO_E_NOMEM; }
    }
    if (ws->use_graph && !ws->graph_failed) {
        cudaGraphExec_t& ex = ws->gexec[want_dist ? 1 : 0];
        if (!ex) {
            cudaGraph_t graph = nullptr;
            bool ok = cudaStreamBeginCapture(ws->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            int rc = ok ? enqueue(ws, want_dist, true) : ISO_E_CUDA;
            cudaError_t ce = ok ? cudaStreamEndCapture(ws->stream, &graph) : cudaErrorUnknown;
            ok = ok && rc == ISO_OK && ce == cudaSuccess && graph &&
                 cudaGraphInstantiate(&ex, graph, 0) == cudaSuccess;
            if (graph) cudaGraphDestroy(graph);
            if (!ok) {
                cudaGetLastError();
                ex = nullptr;
                ws->graph_failed = true;  // run the same sequence without a graph from now on
            }
        }
        if (ex) {
            ISO_CK(cudaGraphLaunch(ex, ws->stream));
            return ISO_OK;
        }
    }
    return enqueue(ws, want_dist, false);
}

int copy_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return ISO_OK;
    ISO_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
    return ISO_OK;
}

int check_opts(const iso_query_opts* o) {
    if (!o) return ISO_OK;
    for (int r : o->reserved)
        if (r) { iso::set_error("iso_query_opts: reserved fields must be zero"); return ISO_E_INVAL; }
    if (o->threads_per_vertex < 0 || o->ctas_per_sm < 0 || o->fuse_width < -1 || o->barrier_timeout_ns < 0 ||
        o->debug_barrier_extra < 0 || o->schedule_delay < 0 || o->solo_width < -1 || o->chunk_span < 0 ||
        o->core_vertices < -1 || o->debug_stage_arcs < 0 || o->debug_stage_deps < 0 || o->restrict_sweep < 0 ||
        o->restrict_sweep > 1 || o->fused_emission < 0 || o->fused_emission > 1) {
        iso::set_error("iso_query_opts: negative field");
        return ISO_E_INVAL;
    }
    return ISO_OK;
}

}  // namespace

extern "C" int iso_upload_graph(const iso_ch* ch, const iso_alloc* alloc, void* stream, iso_graph** out) {
    iso::clear_error();
    if (!ch || !out) { iso::set_error("iso_upload_graph: NULL argument"); return ISO_E_INVAL; }
    *out = nullptr;
    if (alloc && (!alloc->alloc || !alloc->free)) { iso::set_error("iso_upload_graph: incomplete allocator"); return ISO_E_INVAL; }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        iso::set_error("iso_upload_graph: no CUDA device");
        return ISO_E_NODEV;
    }
    std::unique_ptr<iso_graph> g(new iso_graph());
    ISO_CK(cudaGetDevice(&g->device));
    ISO_CK(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device));
    if (alloc) { g->A.cb = *alloc; g->A.custom = true; }
    g->stream = (cudaStream_t)stream;
    g->n = ch->n; g->L = ch->L; g->m = ch->m; g->max_w = ch->max_w;
    g->m_down = ch->down_off.back(); g->m_up = ch->up_off.back();
    g->tau_max = 0x7FFFFFFE - ch->max_w;
    g->h_level_off = ch->level_off;
    const size_t n = (size_t)ch->n;
    std::vector<uint32_t> off32(n + 5);  // four spare entries keep 16-byte bulk copies in bounds
    std::vector<int2> arcs;
    std::vector<int32_t> dsrc;
    int rc = ISO_OK;
    auto free_all = [&]() { for (void* p : g->owned) g->A.put(p, g->stream); g->owned.clear(); };
    // Emission entries for fused emission (Section 5): every input arc except
    // self-loops is checked at its endpoint of lower level (later in sweep
    // order), against the other one, which the sweep must have finished by
    // then.  That holds where a downward arc joins the two (the arc itself, or
    // the reverse arc of a two-way road); for a one-way arc from the lower to
    // the higher endpoint without one, a dummy downward arc of length
    // 0x7FFFFFFF is added, which never lowers a label (a sum with it is at
    // least kInf) but makes the sweep order the two.
    std::vector<uint32_t> eoff(n + 1, 0);
    std::vector<int2> ents;
    std::vector<std::vector<int32_t>> dummy;  // per vertex: dummy arc sources
    size_t ndummy = 0;
    try {
        for (size_t t = 0; t < n; ++t)
            for (int64_t a = ch->orig_off[t]; a < ch->orig_off[t + 1]; ++a) {
                const size_t h = (size_t)ch->orig_head[a];
                if (h != t) eoff[std::max(t, h) + 1]++;
            }
        for (size_t v = 0; v < n; ++v) eoff[v + 1] += eoff[v];
        ents.resize(std::max<size_t>(eoff[n], 1));
        {
            std::vector<uint32_t> fill(eoff.begin(), eoff.end() - 1);
            for (size_t t = 0; t < n; ++t)
                for (int64_t a = ch->orig_off[t]; a < ch->orig_off[t + 1]; ++a) {
                    const size_t h = (size_t)ch->orig_head[a];
                    if (h == t) continue;
                    ents[fill[std::max(t, h)]++] = make_int2((int)std::min(t, h), ch->orig_id[a]);
                }
        }
        std::vector<int32_t> mark(n, -1);
        dummy.resize(n);
        for (size_t v = 0; v < n; ++v) {
            for (int64_t a = ch->down_off[v]; a < ch->down_off[v + 1]; ++a) mark[ch->down_src[a]] = (int32_t)v;
            for (uint32_t e = eoff[v]; e < eoff[v + 1]; ++e) {
                const int32_t hi = ents[e].x;
                if (mark[hi] != (int32_t)v) { mark[hi] = (int32_t)v; dummy[v].push_back(hi); ++ndummy; }
            }
        }
        // downward CSR with the dummy arcs after each vertex's own
        const size_t md = ch->down_src.size() + ndummy;
        if (md > 0xFFFFFFF0u) { free_all(); iso::set_error("iso_upload_graph: too many downward arcs"); return ISO_E_INVAL; }
        arcs.resize(md + 2);  // two spare entries keep 16-byte loads in bounds
        dsrc.resize(md);
        size_t o = 0;
        for (size_t v = 0; v < n; ++v) {
            off32[v] = (uint32_t)o;
            for (int64_t a = ch->down_off[v]; a < ch->down_off[v + 1]; ++a, ++o) {
                arcs[o] = make_int2(ch->down_src[a], ch->down_w[a]);
                dsrc[o] = ch->down_src[a];
            }
            for (int32_t hi : dummy[v]) { arcs[o] = make_int2(hi, 0x7FFFFFFF); dsrc[o] = hi; ++o; }
        }
        off32[n] = (uint32_t)o;
    } catch (const std::bad_alloc&) {
        free_all();
        iso::set_error("iso_upload_graph: out of host memory");
        return ISO_E_NOMEM;
    }
    dummy.clear();
    dummy.shrink_to_fit();
    g->dummy_arcs = (int64_t)ndummy;
    for (size_t i = n + 1; i < n + 5; ++i) off32[i] = off32[n];
    arcs[arcs.size() - 1] = arcs[arcs.size() - 2] = make_int2(0, 0);
    if ((rc = g->upload(&g->down_off, off32.data(), n + 5)) || (rc = g->upload(&g->down_arc, arcs.data(), arcs.size())) ||
        (rc = g->upload(&g->emit_off, eoff.data(), n + 1)) || (rc = g->upload(&g->emit_ent, ents.data(), ents.size()))) {
        free_all(); return rc;
    }
    {
        g->core_cap_n = (int)std::min<size_t>(n, (size_t)kCoreMaxVertices);
        const uint32_t na = off32[g->core_cap_n];
        std::vector<uint2> ca(std::max<uint32_t>(na, 1u), make_uint2(0u, 0u));
        for (int v = 0; v < g->core_cap_n; ++v)
            for (uint32_t a = off32[v]; a < off32[v + 1]; ++a)
                ca[a] = make_uint2((uint32_t)arcs[a].x | ((uint32_t)v << 16), (uint32_t)arcs[a].y);
        std::vector<uint32_t> la(ch->level_off.size());
        for (size_t j = 0; j < la.size(); ++j) la[j] = off32[ch->level_off[j]];
        if ((rc = g->upload(&g->core_arc, ca.data(), ca.size())) || (rc = g->upload(&g->level_arc, la.data(), la.size()))) {
            free_all(); return rc;
        }
        ISO_CK(cudaStreamSynchronize(g->stream));
    }
    ISO_CK(cudaStreamSynchronize(g->stream));
    try {
        g->h_down_off = off32;
        g->h_down_src = std::move(dsrc);
        g->h_bfs = ch->bfs;
    } catch (const std::bad_alloc&) {
        free_all();
        iso::set_error("iso_upload_graph: out of host memory");
        return ISO_E_NOMEM;
    }
    for (size_t i = 0; i <= n; ++i) off32[i] = (uint32_t)ch->up_off[i];
    arcs.assign(ch->up_dst.size() + 2, make_int2(0, 0));
    for (size_t i = 0; i < ch->up_dst.size(); ++i) arcs[i] = make_int2(ch->up_dst[i], ch->up_w[i]);
    if ((rc = g->upload(&g->up_off, off32.data(), n + 1)) || (rc = g->upload(&g->up_arc, arcs.data(), arcs.size()))) {
        free_all(); return rc;
    }
    ISO_CK(cudaStreamSynchronize(g->stream));
    std::vector<int32_t> tail(n), head, aid;
    try {
        head.resize(ch->orig_head.size());
        aid.resize(ch->orig_id.size());
    } catch (const std::bad_alloc&) {
        free_all();
        iso::set_error("iso_upload_graph: out of host memory");
        return ISO_E_NOMEM;
    }
    for (size_t v = 0; v < n; ++v) tail[(size_t)ch->bfs[v]] = (int32_t)v;
    off32[0] = 0;
    for (size_t i = 0; i < n; ++i) {
        const int32_t v = tail[i];
        const int64_t a = ch->orig_off[v], b = ch->orig_off[v + 1];
        std::copy(ch->orig_head.begin() + a, ch->orig_head.begin() + b, head.begin() + off32[i]);
        std::copy(ch->orig_id.begin() + a, ch->orig_id.begin() + b, aid.begin() + off32[i]);
        off32[i + 1] = off32[i] + (uint32_t)(b - a);
    }
    if ((rc = g->upload(&g->orig_off, off32.data(), n + 1)) ||
        (rc = g->upload(&g->orig_head, head.data(), head.size())) ||
        (rc = g->upload(&g->orig_id, aid.data(), aid.size())) ||
        (rc = g->upload(&g->emit_tail, tail.data(), n)) ||
        (rc = g->upload(&g->perm, ch->perm.data(), n)) || (rc = g->upload(&g->pos, ch->pos.data(), n)) ||
        (rc = g->upload(&g->level_off, ch->level_off.data(), ch->level_off.size()))) {
        free_all(); return rc;
    }
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) { free_all(); iso::set_error("iso_upload_graph: %s", cudaGetErrorString(e)); return cuda_status(e); }
    *out = g.release();
    return ISO_OK;
}

extern "C" void iso_free_workspace(iso_workspace* ws);

extern "C" void iso_free_graph(iso_graph* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    for (auto*& ws : g->query_ws) { iso_free_workspace(ws); ws = nullptr; }
    for (void* p : g->owned) g->A.put(p, g->stream);
    delete g;
}

extern "C" int iso_workspace_create(iso_graph* g, int32_t lanes, const iso_query_opts* opts, void* stream,
                                    iso_workspace** out) {
    iso::clear_error();
    if (!g || !out) { iso::set_error("iso_workspace_create: NULL argument"); return ISO_E_INVAL; }
    *out = nullptr;
    if (lanes < 1 || lanes > kMaxLanes) { iso::set_error("iso_workspace_create: lanes must be in 1..64"); return ISO_E_INVAL; }
    int rc = check_opts(opts);
    if (rc) return rc;
    std::unique_ptr<iso_workspace> ws(new iso_workspace());
    ws->g = g;
    ws->stream = (cudaStream_t)stream;
    ws->K = lanes_class(lanes);
    const iso_query_opts o = opts ? *opts : iso_query_opts{};
    int occ = 0, vpb = 0;
    if (o.sweep_kernel < 0 || o.sweep_kernel > 2 || !sweep_shape(ws->K, o, &ws->kernel, &ws->tpv, &occ, &vpb)) {
        iso::set_error("iso_workspace_create: sweep kernel %d with %d threads per vertex unsupported for %d lanes",
                       o.sweep_kernel, o.threads_per_vertex, ws->K);
        return ISO_E_INVAL;
    }
    const int per_sm = o.ctas_per_sm ? std::min<int>(o.ctas_per_sm, occ) : occ;
    ws->grid = g->num_sms * per_sm;
    ws->fuse_width = o.fuse_width == 0 ? vpb : (o.fuse_width < 0 ? 0 : o.fuse_width);
    ws->vpb = vpb;
    // a level narrower than one chunk of ws->vpb vertices per CTA runs with a warp per vertex
    ws->narrow_width = o.fuse_width < 0 ? 0 : (o.fuse_width > 0 ? o.fuse_width : ws->grid * vpb);
    ws->record_trace = o.record_trace != 0 && ws->kernel == 1;
    ws->sched_delay = o.schedule_delay > 0 ? o.schedule_delay : 3 * ws->grid;
    ws->solo_width = o.solo_width < 0 ? 0 : (o.solo_width > 0 ? o.solo_width : kSoloWidth);
    ws->chunk_span = o.chunk_span;
    ws->core_limit = core_limit_of(o, g->n);
    ws->stage_arc_cap = o.debug_stage_arcs;
    ws->stage_pred_cap = o.debug_stage_deps;
    ws->restrict_sweep = o.restrict_sweep != 0;
    ws->fused_emit = o.fused_emission != 0;
    if (ws->fused_emit && ws->kernel != 1) {
        iso::set_error("iso_workspace_create: fused_emission needs the TMA-staged sweep");
        return ISO_E_INVAL;
    }
    if (ws->restrict_sweep && (g->lm.count == 0 || ws->kernel != 1)) {
        iso::set_error("iso_workspace_create: restrict_sweep needs landmarks on the graph (iso_graph_add_landmarks) "
                       "and the TMA-staged sweep");
        return ISO_E_INVAL;
    }
    ws->use_graph = opts ? opts->use_cuda_graph != 0 : false;
    if (opts && opts->barrier_timeout_ns) ws->timeout_ns = opts->barrier_timeout_ns;
    ws->bar_extra = opts ? opts->debug_barrier_extra : 0;
    auto fail = [&](int code) {
        for (void* p : ws->owned) g->A.put(p, ws->stream);
        ws->owned.clear();
        if (ws->h_io) cudaFreeHost(ws->h_io);
        if (ws->h_ctl) cudaFreeHost(ws->h_ctl);
        ws->h_io = ws->h_ctl = nullptr;
        return code;
    };
    const size_t n = (size_t)g->n, K = (size_t)ws->K;
    const size_t mask_bytes = K <= 8 ? 1 : K / 8;
    ws->d = (uint32_t*)ws->alloc(n * K * 4);
    ws->mask = ws->alloc(n * mask_bytes);
    ws->upflag = (uint8_t*)ws->alloc(n);
    ws->io = (int32_t*)ws->alloc(2 * K * 4);
    ws->ctl = (int32_t*)ws->alloc(ws->ctl_words() * 4);
    ws->out_off = (int64_t*)ws->alloc((K + 1) * 8);
    if (!ws->d || !ws->mask || !ws->upflag || !ws->io || !ws->ctl || !ws->out_off) {
        iso::set_error("iso_workspace_create: device allocation failed");
        return fail(ISO_E_NOMEM);
    }
    if ((rc = alloc_up(ws.get())) || (rc = alloc_emit(ws.get())) || (rc = build_schedule(ws.get()))) return fail(rc);
    if (ws->record_trace) {
        ws->trace = (long long*)ws->alloc(((size_t)g->L + 2) * 8);
        if (!ws->trace) { iso::set_error("iso_workspace_create: device allocation failed"); return fail(ISO_E_NOMEM); }
        ws->h_trace.assign((size_t)g->L + 2, 0);
    }
    if (cudaMallocHost(&ws->h_io, 2 * K * 4) != cudaSuccess ||
        cudaMallocHost(&ws->h_ctl, ws->ctl_words() * 4) != cudaSuccess) {
        cudaGetLastError();
        iso::set_error("iso_workspace_create: pinned host allocation failed");
        return fail(ISO_E_NOMEM);
    }
    for (auto& e : ws->ev)
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); iso::set_error("iso_workspace_create: event"); return fail(ISO_E_CUDA); }
    if (cudaEventCreateWithFlags(&ws->ev_swept, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        iso::set_error("iso_workspace_create: event");
        return fail(ISO_E_CUDA);
    }
    if (ws->kernel == 1 && ws->core_levels > 0) {
        ws->core_out = (uint32_t*)ws->alloc(K * (size_t)ws->core_n * 4);
        if (!ws->core_out) { iso::set_error("iso_workspace_create: device allocation failed"); return fail(ISO_E_NOMEM); }
    }
    if (ws->kernel == 1) {
        ws->upmask = (unsigned long long*)ws->alloc(n * 8);
        if (!ws->upmask) { iso::set_error("iso_workspace_create: device allocation failed"); return fail(ISO_E_NOMEM); }
        if (cudaMemsetAsync(ws->upmask, 0, n * 8, ws->stream) != cudaSuccess) {
            cudaGetLastError();
            iso::set_error("iso_workspace_create: initialisation failed");
            return fail(ISO_E_CUDA);
        }
    }
    if (cudaMemsetAsync(ws->upflag, 0, n, ws->stream) != cudaSuccess ||
        cudaStreamSynchronize(ws->stream) != cudaSuccess) {
        cudaGetLastError();
        iso::set_error("iso_workspace_create: initialisation failed");
        return fail(ISO_E_CUDA);
    }
    if (ws->restrict_sweep) ++g->restricted_ws;
    *out = ws.release();
    return ISO_OK;
}

extern "C" void iso_free_workspace(iso_workspace* ws) {
    if (!ws) return;
    if (ws->stream) cudaStreamSynchronize(ws->stream);
    ws->drop_graphs();
    for (auto& e : ws->ev)
        if (e) cudaEventDestroy(e);
    if (ws->ev_swept) cudaEventDestroy(ws->ev_swept);
    for (void* p : ws->owned) ws->g->A.put(p, ws->stream);
    if (ws->h_io) cudaFreeHost(ws->h_io);
    if (ws->h_ctl) cudaFreeHost(ws->h_ctl);
    if (ws->restrict_sweep) --ws->g->restricted_ws;
    delete ws;
}

namespace {
int submit_impl(iso_workspace* ws, int32_t k, const int32_t* sources, const int32_t* taus, bool want_dist,
                cudaStream_t stream, const iso_workspace* after = nullptr) {
    iso_graph* g = ws->g;
    if (k < 0 || k > ws->K) { iso::set_error("iso_submit: k=%d outside 0..%d", k, ws->K); return ISO_E_INVAL; }
    if (k > 0 && (!sources || !taus)) { iso::set_error("iso_submit: NULL sources or taus"); return ISO_E_INVAL; }
    if (ws->stream != stream) { ws->drop_graphs(); ws->stream = stream; }
    const bool dev_s = is_device_ptr(sources), dev_t = is_device_ptr(taus);
    const int K = ws->K;
    for (int i = 0; i < 2 * K; ++i) ws->h_io[i] = -1;
    if (!dev_s || !dev_t) {
        for (int i = 0; i < k; ++i) {
            if (!dev_s) {
                if (sources[i] < 0 || sources[i] >= g->n) {
                    iso::set_error("iso_submit: source %d of query %d outside [0,%d)", sources[i], i, g->n);
                    return ISO_E_INVAL;
                }
                ws->h_io[i] = sources[i];
            }
            if (!dev_t) {
                if (taus[i] < 0 || taus[i] > g->tau_max) {
                    iso::set_error("iso_submit: limit %d of query %d outside [0,%d]", taus[i], i, g->tau_max);
                    return ISO_E_INVAL;
                }
                ws->h_io[K + i] = taus[i];
            }
        }
    }
    for (int i = k; i < K; ++i) ws->h_io[K + i] = 0;  // idle lanes: src -1, tau 0
    ISO_CK(cudaMemcpyAsync(ws->io, ws->h_io, 2 * (size_t)K * 4, cudaMemcpyHostToDevice, stream));
    if (dev_s && k) ISO_CK(cudaMemcpyAsync(ws->io, sources, (size_t)k * 4, cudaMemcpyDeviceToDevice, stream));
    if (dev_t && k) ISO_CK(cudaMemcpyAsync(ws->io + K, taus, (size_t)k * 4, cudaMemcpyDeviceToDevice, stream));
    ws->k = k;
    ws->want_dist = want_dist;
    ws->collected = false;
    // the batch's kernels start once the sweep last submitted on `after` is done
    if (after && after != ws && after->submitted) ISO_CK(cudaStreamWaitEvent(stream, after->ev_swept, 0));
    int rc = launch_batch(ws, want_dist);
    if (rc) return rc;
    ws->submitted = true;
    return ISO_OK;
}

int collect_impl(iso_workspace* ws, int64_t* out_offsets, int32_t* out_arcs, int64_t cap, int32_t* out_dist) {
    if (!ws->submitted) { iso::set_error("iso_collect: nothing submitted"); return ISO_E_INVAL; }
    if (!out_offsets) { iso::set_error("iso_collect: out_offsets is NULL"); return ISO_E_INVAL; }
    if (out_dist && !ws->want_dist) { iso::set_error("iso_collect: distances were not requested at submit"); return ISO_E_INVAL; }
    for (int attempt = 0;; ++attempt) {
        ISO_CK(cudaEventSynchronize(ws->ev[5]));
        const int st = ws->h_ctl[0];
        ws->skipped = ws->h_ctl[1];
        if (st != kStOk) ws->stale_flags = true;
        if (st == kStTimeout) { ws->submitted = false; iso::set_error("sweep: a grid barrier timed out"); return ISO_E_TIMEOUT; }
        if (st == kStBadInput) { ws->submitted = false; iso::set_error("query: a source or limit failed validation"); return ISO_E_INVAL; }
        int grow_up = st == kStUpOverflow;
        int need = 0;
        for (int i = 0; i < ws->K; ++i) need = std::max(need, ws->h_ctl[8 + i]);
        const bool grow_emit = need > ws->ecap;
        if (!grow_up && !grow_emit) break;
        if (attempt > 8) { iso::set_error("collect: buffers kept overflowing"); return ISO_E_NOMEM; }
        ws->drop_graphs();
        if (grow_up) {
            ws->release(*(void**)&ws->pairs);
            ws->release(*(void**)&ws->gtab);
            ws->gcap *= 4;
            if (int rc = alloc_up(ws)) return rc;
        }
        if (grow_emit) {
            ws->release(*(void**)&ws->ebuf);
            ws->release(*(void**)&ws->tmp);
            ws->release(*(void**)&ws->out);
            while (ws->ecap < need) ws->ecap *= 2;
            if (int rc = alloc_emit(ws)) return rc;
        }
        if (int rc = launch_batch(ws, ws->want_dist)) return rc;
    }
    if (ws->trace)
        ISO_CK(cudaMemcpy(ws->h_trace.data(), ws->trace, ws->h_trace.size() * 8, cudaMemcpyDeviceToHost));
    float t[4] = {};
    for (int i = 0; i < 4; ++i) cudaEventElapsedTime(&t[i], ws->ev[i], ws->ev[i + 1]);
    for (int i = 0; i < 4; ++i) ws->phase_ms[i] = t[i];
    std::vector<int64_t> off(ws->k + 1, 0);
    for (int i = 0; i < ws->k; ++i) off[i + 1] = off[i] + ws->h_ctl[8 + i];
    const int64_t total = off[ws->k];
    cudaStream_t s = ws->stream;
    if (int rc = copy_out(out_offsets, off.data(), off.size() * 8, s)) return rc;
    int rc = ISO_OK;
    if (total > cap) {
        iso::set_error("iso_collect: %lld arcs do not fit capacity %lld", (long long)total, (long long)cap);
        rc = ISO_E_OVERFLOW;
    } else if (total > 0) {
        if (!out_arcs) { iso::set_error("iso_collect: out_arcs is NULL"); return ISO_E_INVAL; }
        if (int r2 = copy_out(out_arcs, ws->out, (size_t)total * 4, s)) return r2;
    }
    if (out_dist && rc == ISO_OK)
        if (int r2 = copy_out(out_dist, ws->dist, (size_t)ws->k * ws->g->n * 4, s)) return r2;
    ISO_CK(cudaStreamSynchronize(s));
    ws->collected = rc == ISO_OK || rc == ISO_E_OVERFLOW;
    return rc;
}

int range_impl(iso_workspace* ws, uint32_t* out_bits, int64_t words) {
    if (!ws->collected) { iso::set_error("iso_collect_range: no collected batch"); return ISO_E_INVAL; }
    const int n = ws->g->n;
    const int64_t need = ((int64_t)n + 31) / 32;
    if (!out_bits && ws->k > 0) { iso::set_error("iso_collect_range: out_bits is NULL"); return ISO_E_INVAL; }
    if (words < need) { iso::set_error("iso_collect_range: %lld words per query, %lld needed", (long long)words, (long long)need); return ISO_E_INVAL; }
    if (ws->k == 0) return ISO_OK;
    cudaStream_t s = ws->stream;
    const bool dev = is_device_ptr(out_bits);
    uint32_t* dst = out_bits;
    if (!dev) {
        if (!ws->range) {
            ws->range = (uint32_t*)ws->alloc((size_t)ws->K * need * 4);
            if (!ws->range) { iso::set_error("iso_collect_range: device allocation failed"); return ISO_E_NOMEM; }
        }
        dst = ws->range;
    }
    RangeParams rp{};
    rp.pos = ws->g->pos; rp.mask = ws->mask; rp.out = dst; rp.words = dev ? words : need; rp.n = n; rp.k = ws->k;
    ISO_CK(iso_launch_range(rp, ws->K, s));
    if (!dev) {
        // query i's bitset to out_bits[i * words], words beyond the need untouched
        ISO_CK(cudaMemcpy2DAsync(out_bits, (size_t)words * 4, dst, (size_t)need * 4, (size_t)need * 4, ws->k,
                                 cudaMemcpyDeviceToHost, s));
    }
    ISO_CK(cudaStreamSynchronize(s));
    return ISO_OK;
}
}  // namespace

extern "C" int iso_submit(iso_workspace* ws, int32_t k, const int32_t* sources, const int32_t* taus, int32_t flags,
                          void* stream) {
    iso::clear_error();
    if (!ws) { iso::set_error("iso_submit: NULL workspace"); return ISO_E_INVAL; }
    if (flags & ~ISO_SUBMIT_DIST) { iso::set_error("iso_submit: unknown flags"); return ISO_E_INVAL; }
    return submit_impl(ws, k, sources, taus, (flags & ISO_SUBMIT_DIST) != 0, (cudaStream_t)stream);
}

extern "C" int iso_submit_after(iso_workspace* ws, const iso_workspace* after, int32_t k, const int32_t* sources,
                                const int32_t* taus, int32_t flags, void* stream) {
    iso::clear_error();
    if (!ws) { iso::set_error("iso_submit_after: NULL workspace"); return ISO_E_INVAL; }
    if (after && after->g != ws->g) { iso::set_error("iso_submit_after: workspaces of different graphs"); return ISO_E_INVAL; }
    if (flags & ~ISO_SUBMIT_DIST) { iso::set_error("iso_submit_after: unknown flags"); return ISO_E_INVAL; }
    return submit_impl(ws, k, sources, taus, (flags & ISO_SUBMIT_DIST) != 0, (cudaStream_t)stream, after);
}

extern "C" int iso_collect(iso_workspace* ws, int64_t* out_offsets, int32_t* out_arcs, int64_t cap,
                           int32_t* out_dist) {
    iso::clear_error();
    if (!ws) { iso::set_error("iso_collect: NULL workspace"); return ISO_E_INVAL; }
    return collect_impl(ws, out_offsets, out_arcs, cap, out_dist);
}

extern "C" int iso_collect_range(iso_workspace* ws, uint32_t* out_bits, int64_t words_per_query) {
    iso::clear_error();
    if (!ws) { iso::set_error("iso_collect_range: NULL workspace"); return ISO_E_INVAL; }
    return range_impl(ws, out_bits, words_per_query);
}

extern "C" int32_t iso_workspace_trace(const iso_workspace* ws, int32_t* steps4, int64_t* ns, int32_t cap) {
    iso::clear_error();
    if (!ws) { iso::set_error("iso_workspace_trace: NULL workspace"); return -1; }
    if (!ws->trace) {
        iso::set_error("iso_workspace_trace: workspace created without record_trace or with the plain sweep");
        return -1;
    }
    const int L = ws->g->L;
    const long long walk0 = ws->h_trace[(size_t)L + 1];
    for (int32_t i = 0; i <= L && i < cap; ++i) {
        if (i < L) {
            if (steps4) { steps4[4 * i] = 0; steps4[4 * i + 1] = i; steps4[4 * i + 2] = i + 1; steps4[4 * i + 3] = 0; }
            if (ns) ns[i] = ws->h_trace[(size_t)i + 1] - walk0;
        } else {
            if (steps4) { steps4[4 * i] = 2; steps4[4 * i + 1] = 0; steps4[4 * i + 2] = 0; steps4[4 * i + 3] = 0; }
            if (ns) ns[i] = walk0 - ws->h_trace[0];
        }
    }
    return L + 1;
}

extern "C" int iso_workspace_sweep_info(const iso_workspace* ws, iso_sweep_info* out) {
    iso::clear_error();
    if (!ws || !out) { iso::set_error("iso_workspace_sweep_info: NULL argument"); return ISO_E_INVAL; }
    *out = ws->info;
    return ISO_OK;
}

extern "C" int iso_workspace_skipped_chunks(const iso_workspace* ws, int64_t* out) {
    iso::clear_error();
    if (!ws || !out) { iso::set_error("iso_workspace_skipped_chunks: NULL argument"); return ISO_E_INVAL; }
    *out = ws->skipped;
    return ISO_OK;
}

extern "C" int iso_graph_add_landmarks(iso_graph* g, const iso_ch* ch, int32_t count) {
    iso::clear_error();
    if (!g || !ch) { iso::set_error("iso_graph_add_landmarks: NULL argument"); return ISO_E_INVAL; }
    if (count < 1 || count > ISO_MAX_LANDMARKS) {
        iso::set_error("iso_graph_add_landmarks: count %d outside 1..%d", count, ISO_MAX_LANDMARKS);
        return ISO_E_INVAL;
    }
    if (ch->n != g->n || (int64_t)ch->down_off.back() != g->m_down) {
        iso::set_error("iso_graph_add_landmarks: the hierarchy is not the one uploaded as this graph");
        return ISO_E_INVAL;
    }
    std::lock_guard<std::mutex> lock(g->mu);
    // workspaces with restricted sweeps hold per-chunk bounds of the current
    // landmarks and use their device arrays (also from captured CUDA graphs):
    // iso_query's own are dropped, a caller's must be freed first
    for (auto*& w : g->query_ws)
        if (w && w->restrict_sweep) { iso_free_workspace(w); w = nullptr; }
    if (g->restricted_ws.load() > 0) {
        iso::set_error("iso_graph_add_landmarks: %d workspaces with restricted sweeps still use the landmarks; "
                       "free them first", g->restricted_ws.load());
        return ISO_E_INVAL;
    }
    LandmarkSet lm;
    try {
        if (iso_landmarks_compute(*ch, count, &lm) != 0) { iso::set_error("iso_graph_add_landmarks: bad input"); return ISO_E_INVAL; }
    } catch (const std::bad_alloc&) {
        iso::set_error("iso_graph_add_landmarks: out of host memory");
        return ISO_E_NOMEM;
    }
    uint32_t *f = nullptr, *b = nullptr;
    int rc = ISO_OK;
    if ((rc = g->upload(&f, lm.fwd.data(), lm.fwd.size())) || (rc = g->upload(&b, lm.bwd.data(), lm.bwd.size())))
        return rc;  // a buffer already made stays owned by the graph
    ISO_CK(cudaStreamSynchronize(g->stream));
    if (g->lm_fwd) { g->owned.erase(std::remove(g->owned.begin(), g->owned.end(), (void*)g->lm_fwd), g->owned.end()); g->A.put(g->lm_fwd, g->stream); }
    if (g->lm_bwd) { g->owned.erase(std::remove(g->owned.begin(), g->owned.end(), (void*)g->lm_bwd), g->owned.end()); g->A.put(g->lm_bwd, g->stream); }
    g->lm_fwd = f;
    g->lm_bwd = b;
    g->lm = std::move(lm);
    return ISO_OK;
}

extern "C" int iso_workspace_timings(const iso_workspace* ws, float* ms4) {
    iso::clear_error();
    if (!ws || !ms4) { iso::set_error("iso_workspace_timings: NULL argument"); return ISO_E_INVAL; }
    std::memcpy(ms4, ws->phase_ms, sizeof(ws->phase_ms));
    return ISO_OK;
}

namespace {
// Does workspace ws run with the settings that options o ask for?
bool same_config(const iso_workspace* ws, const iso_query_opts& o) {
    int kernel = 0, tpv = 0, occ = 0, vpb = 0;
    if (!sweep_shape(ws->K, o, &kernel, &tpv, &occ, &vpb)) return false;
    const int per_sm = o.ctas_per_sm ? std::min<int>(o.ctas_per_sm, occ) : occ;
    const int fuse = o.fuse_width == 0 ? vpb : (o.fuse_width < 0 ? 0 : o.fuse_width);
    const long long timeout = o.barrier_timeout_ns ? o.barrier_timeout_ns : 2000000000LL;
    return ws->kernel == kernel && ws->tpv == tpv && ws->grid == ws->g->num_sms * per_sm &&
           ws->fuse_width == fuse && ws->use_graph == (o.use_cuda_graph != 0) && ws->timeout_ns == timeout &&
           ws->bar_extra == o.debug_barrier_extra && ws->record_trace == (o.record_trace != 0 && kernel == 1) &&
           ws->sched_delay == (o.schedule_delay > 0 ? o.schedule_delay : 3 * ws->g->num_sms * per_sm) &&
           ws->solo_width == (o.solo_width < 0 ? 0 : (o.solo_width > 0 ? o.solo_width : kSoloWidth)) &&
           ws->chunk_span == o.chunk_span && ws->core_limit == core_limit_of(o, ws->g->n) &&
           ws->stage_arc_cap == o.debug_stage_arcs && ws->stage_pred_cap == o.debug_stage_deps &&
           ws->restrict_sweep == (o.restrict_sweep != 0) && ws->fused_emit == (o.fused_emission != 0);
}
}  // namespace

extern "C" int iso_query(iso_graph* g, int32_t k, const int32_t* sources, const int32_t* taus, int64_t* out_offsets,
                         int32_t* out_arcs, int64_t cap, int32_t* out_dist, const iso_query_opts* opts,
                         void* stream) {
    iso::clear_error();
    if (!g || !out_offsets) { iso::set_error("iso_query: NULL argument"); return ISO_E_INVAL; }
    if (k < 0) { iso::set_error("iso_query: k < 0"); return ISO_E_INVAL; }
    if (k > 0 && (!sources || !taus)) { iso::set_error("iso_query: NULL sources or taus"); return ISO_E_INVAL; }
    if (int rc = check_opts(opts)) return rc;
    std::lock_guard<std::mutex> lock(g->mu);
    const bool dev_off = is_device_ptr(out_offsets);
    const bool dev_src = is_device_ptr(sources), dev_tau = is_device_ptr(taus);
    std::vector<int64_t> offs((size_t)k + 1, 0);
    int64_t used = 0;
    int result = ISO_OK;
    const int chunk = kMaxLanes;
    for (int b = 0; b < k || (k == 0 && b == 0); b += chunk) {
        const int kb = std::min(chunk, k - b);
        if (kb <= 0) break;
        const int K = lanes_class(kb);
        int ci = 0;
        while ((1 << ci) < K) ++ci;
        iso_workspace*& ws = g->query_ws[ci];
        iso_query_opts o = opts ? *opts : iso_query_opts{};
        if (!opts) o.use_cuda_graph = 1;
        if (ws && !same_config(ws, o)) {
            iso_free_workspace(ws);
            ws = nullptr;
        }
        if (!ws) {
            if (int rc = iso_workspace_create(g, K, &o, stream, &ws)) return rc;
        }
        if (int rc = submit_impl(ws, kb, dev_src ? sources + b : sources + b, dev_tau ? taus + b : taus + b,
                                 out_dist != nullptr, (cudaStream_t)stream))
            return rc;
        std::vector<int64_t> lo(kb + 1);
        const int64_t room = result == ISO_OK ? std::max<int64_t>(0, cap - used) : 0;
        int32_t* dst = out_arcs ? out_arcs + used : nullptr;
        int32_t* ddst = out_dist ? out_dist + (size_t)b * g->n : nullptr;
        int rc = collect_impl(ws, lo.data(), dst, room, ddst);
        if (rc == ISO_E_OVERFLOW) result = ISO_E_OVERFLOW;
        else if (rc) return rc;
        for (int i = 0; i < kb; ++i) offs[b + i + 1] = used + lo[i + 1];
        used += lo[kb];
    }
    if (dev_off) ISO_CK(cudaMemcpyAsync(out_offsets, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    else std::memcpy(out_offsets, offs.data(), offs.size() * 8);
    ISO_CK(cudaStreamSynchronize((cudaStream_t)stream));
    if (result == ISO_E_OVERFLOW)
        iso::set_error("iso_query: %lld arcs do not fit capacity %lld", (long long)used, (long long)cap);
    return result;
}

int iso_graph_view_of(const iso_graph* g, iso_graph_view* v) {
    if (!g || !v) return ISO_E_INVAL;
    v->n = g->n; v->L = g->L; v->tau_max = g->tau_max; v->num_sms = g->num_sms; v->m = g->m;
    v->device = g->device;
    v->down_off = g->down_off; v->up_off = g->up_off; v->orig_off = g->orig_off;
    v->down_arc = g->down_arc; v->up_arc = g->up_arc;
    v->orig_head = g->orig_head; v->orig_id = g->orig_id; v->pos = g->pos; v->level_off = g->level_off;
    v->emit_tail = g->emit_tail;
    v->h_level_off = g->h_level_off.data();
    return ISO_OK;
}
