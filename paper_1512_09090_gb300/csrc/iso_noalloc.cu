// iso_query_noalloc: the query path with every scratch buffer in one
// file-scope device array instead of memory obtained from an allocator.
//
// Some callers cannot allocate device memory while they answer a query: a
// process whose device memory is fully reserved by another framework's pool,
// a latency-critical thread that must not wait on allocator locks or on the
// device-wide synchronisation a cudaFree can imply, or an embedding host that
// forbids allocation after start-up.  For them this entry point runs the same
// kernels (upward search, sweep, emission, sort) on slices of g_scratch, a
// static __device__ array of fixed size.  Every GPU that loads the library holds
// that array until the process exits.
//
// Limits (checked; larger requests return ISO_E_INVAL): graphs of at most
// kMaxVertices vertices and kMaxLevels CH levels, at most kMaxLanes queries per
// call, at most kMaxUpward upward-search vertices and kMaxArcs isochrone edges
// per query.
//
// The host code never uses the symbol g_scratch as a device address (in host
// code it names a host-side stand-in): on the first call on each device, with
// that device current, cudaGetSymbolAddress gives the device address, which is
// cached and passed to the kernels.  That first call must therefore come before
// any stream capture on the device.  All calls share the array and it keeps the
// last call's contents; each call clears what must start at zero.  Calls that
// overlap on the GPU (two streams, or two host threads) race on the array, so
// callers must serialise them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "ch_internal.h"
#include "graph_view.h"
#include "iso_device.cuh"
#include "../../include/iso.h"

namespace {

using namespace isod;

constexpr int kMaxVertices = ISO_NOALLOC_MAX_VERTICES;
constexpr int kMaxLanes = ISO_NOALLOC_MAX_QUERIES;  // one lane class: K = 4
constexpr int kLanes = 4;
constexpr int kMaxLevels = 4096;
constexpr int kUpCap = 16384;                        // global table slots per lane
constexpr int kMaxUpward = kUpCap / 2;
constexpr int kMaxArcs = ISO_NOALLOC_MAX_ARCS;       // isochrone edges per query

// Byte offsets of the slices (each 256-byte aligned).
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffD = 0;
constexpr size_t kOffMask = al(kOffD + (size_t)kMaxVertices * kLanes * 4);
constexpr size_t kOffFlag = al(kOffMask + (size_t)kMaxVertices);
constexpr size_t kOffIo = al(kOffFlag + (size_t)kMaxVertices);
constexpr size_t kOffCtl = al(kOffIo + 2 * kLanes * 4);
constexpr size_t kCtlWords = 8 + 2 * kLanes;
constexpr size_t kOffPairs = al(kOffCtl + kCtlWords * 4);
constexpr size_t kOffTab = al(kOffPairs + (size_t)kLanes * kUpCap * 8);
constexpr size_t kOffEbuf = al(kOffTab + (size_t)kLanes * 5 * kUpCap * 4);
constexpr size_t kOffTmp = al(kOffEbuf + (size_t)kLanes * kMaxArcs * 4);
constexpr size_t kOffOut = al(kOffTmp + (size_t)kLanes * kMaxArcs * 4);
constexpr size_t kOffOutOff = al(kOffOut + (size_t)kLanes * kMaxArcs * 4);
constexpr size_t kOffSched = al(kOffOutOff + (kLanes + 1) * 8);
constexpr size_t kScratchBytes = al(kOffSched + (size_t)kMaxLevels * sizeof(int4));
static_assert(kScratchBytes == ISO_NOALLOC_SCRATCH_BYTES, "iso.h states the scratch size");

std::mutex g_mu;
unsigned char* g_base[64] = {};   // device address of g_scratch, per device
int4 g_sched[kMaxLevels];         // host staging of the level schedule (static, not allocated)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int fail(int code, const char* what, cudaError_t e) {
    iso::set_error("iso_query_noalloc: %s: %s", what, cudaGetErrorString(e));
    return code;
}

// The same, for failures after work was enqueued on `stream`: waits for that
// work first (ignoring the result), so the next call never reuses the array
// while this call's kernels or copies still run on it.
int fail_enqueued(int code, const char* what, cudaError_t e, cudaStream_t stream) {
    cudaStreamSynchronize(stream);
    cudaGetLastError();
    return fail(code, what, e);
}

}  // namespace

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

extern "C" int iso_query_noalloc(iso_graph* g, int32_t k, const int32_t* sources, const int32_t* taus,
                                 int64_t* out_offsets, int32_t* out_arcs, int64_t cap, void* stream_) {
    iso::clear_error();
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!g || !out_offsets) { iso::set_error("iso_query_noalloc: NULL argument"); return ISO_E_INVAL; }
    if (k < 0 || k > kMaxLanes) {
        iso::set_error("iso_query_noalloc: k=%d outside 0..%d", k, kMaxLanes);
        return ISO_E_INVAL;
    }
    if (k > 0 && (!sources || !taus)) { iso::set_error("iso_query_noalloc: NULL sources or taus"); return ISO_E_INVAL; }
    iso_graph_view gv;
    if (iso_graph_view_of(g, &gv) != ISO_OK) { iso::set_error("iso_query_noalloc: bad graph"); return ISO_E_INVAL; }
    if (gv.n > kMaxVertices) {
        iso::set_error("iso_query_noalloc: graph has %d vertices, the limit is %d", gv.n, kMaxVertices);
        return ISO_E_INVAL;
    }
    if (gv.L > kMaxLevels) {
        iso::set_error("iso_query_noalloc: graph has %d CH levels, the limit is %d", gv.L, kMaxLevels);
        return ISO_E_INVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(ISO_E_CUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= 64) { iso::set_error("iso_query_noalloc: device id %d unsupported", dev); return ISO_E_INVAL; }
    if (dev != gv.device) {
        // the kernels would get another GPU's graph pointers and scratch
        iso::set_error("iso_query_noalloc: the graph lives on device %d but device %d is current", gv.device, dev);
        return ISO_E_INVAL;
    }
    if (!g_base[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return fail(ISO_E_CUDA, "cudaGetSymbolAddress", e);
        g_base[dev] = (unsigned char*)p;
    }
    unsigned char* base = g_base[dev];
    int32_t* io = (int32_t*)(base + kOffIo);
    int32_t* ctl = (int32_t*)(base + kOffCtl);

    // inputs: idle lanes have source -1
    int32_t h_io[2 * kLanes];
    for (int i = 0; i < kLanes; ++i) { h_io[i] = -1; h_io[kLanes + i] = 0; }
    const bool dev_s = is_device_ptr(sources), dev_t = is_device_ptr(taus);
    for (int i = 0; i < k; ++i) {
        if (!dev_s) {
            if (sources[i] < 0 || sources[i] >= gv.n) {
                iso::set_error("iso_query_noalloc: source %d of query %d outside [0,%d)", sources[i], i, gv.n);
                return ISO_E_INVAL;
            }
            h_io[i] = sources[i];
        }
        if (!dev_t) {
            if (taus[i] < 0 || taus[i] > gv.tau_max) {
                iso::set_error("iso_query_noalloc: limit %d of query %d outside [0,%d]", taus[i], i, gv.tau_max);
                return ISO_E_INVAL;
            }
            h_io[kLanes + i] = taus[i];
        }
    }
    if ((e = cudaMemcpyAsync(io, h_io, sizeof h_io, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        return fail_enqueued(ISO_E_CUDA, "input copy", e, stream);
    if (dev_s && k && (e = cudaMemcpyAsync(io, sources, (size_t)k * 4, cudaMemcpyDeviceToDevice, stream)))
        return fail_enqueued(ISO_E_CUDA, "input copy", e, stream);
    if (dev_t && k && (e = cudaMemcpyAsync(io + kLanes, taus, (size_t)k * 4, cudaMemcpyDeviceToDevice, stream)))
        return fail_enqueued(ISO_E_CUDA, "input copy", e, stream);
    // state that must start at zero: control block (status, barrier, counters) and flags
    if ((e = cudaMemsetAsync(ctl, 0, kCtlWords * 4, stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(base + kOffFlag, 0, (size_t)gv.n, stream)) != cudaSuccess)
        return fail_enqueued(ISO_E_CUDA, "clearing scratch", e, stream);
    // one grid-wide step per level
    for (int j = 0; j < gv.L; ++j) g_sched[j] = make_int4(kStepWide, j, j + 1, 0);
    if ((e = cudaMemcpyAsync(base + kOffSched, g_sched, (size_t)gv.L * sizeof(int4), cudaMemcpyHostToDevice,
                             stream)) != cudaSuccess)
        return fail_enqueued(ISO_E_CUDA, "schedule copy", e, stream);

    UpParams up{};
    up.up_off = gv.up_off; up.up_arc = gv.up_arc; up.pos = gv.pos; up.src = io; up.tau = io + kLanes;
    up.pairs = (int2*)(base + kOffPairs); up.cnt = ctl + 8 + kLanes; up.gtab = (uint32_t*)(base + kOffTab);
    up.status = ctl; up.n = gv.n; up.cap = kUpCap; up.gcap = kUpCap; up.tau_max = gv.tau_max;
    if ((e = iso_launch_upward(up, kLanes, stream)) != cudaSuccess) return fail_enqueued(ISO_E_CUDA, "upward launch", e, stream);

    SweepParams sw{};
    sw.down_off = gv.down_off; sw.down_arc = gv.down_arc; sw.level_off = gv.level_off;
    sw.sched = (const int4*)(base + kOffSched); sw.pairs = up.pairs; sw.cnt = up.cnt; sw.tau = io + kLanes;
    sw.d = (uint32_t*)(base + kOffD); sw.mask = base + kOffMask; sw.upflag = base + kOffFlag;
    sw.bar = (uint32_t*)(ctl + 4); sw.status = ctl; sw.timeout_ns = 2000000000LL; sw.n = gv.n; sw.L = gv.L;
    sw.nsched = gv.L; sw.cap = kUpCap; sw.last_level_block = gv.L - 1; sw.write_all = 0; sw.bar_extra = 0;
    int block = 0;
    const int occ = iso_sweep_occupancy(kLanes, 1, &block);
    if (occ <= 0) return fail_enqueued(ISO_E_CUDA, "sweep kernel cannot be resident", cudaGetLastError(), stream);
    if ((e = iso_launch_sweep(sw, kLanes, 1, gv.num_sms * occ, stream)) != cudaSuccess)
        return fail_enqueued(ISO_E_CUDA, "sweep launch", e, stream);

    EmitParams em{};
    em.orig_off = gv.orig_off; em.orig_head = gv.orig_head; em.orig_id = gv.orig_id; em.mask = sw.mask;
    em.tail_of = gv.emit_tail;
    em.status = ctl;
    em.ecnt = ctl + 8; em.ebuf = (int32_t*)(base + kOffEbuf); em.n = gv.n; em.ecap = kMaxArcs;
    if ((e = iso_launch_emit(em, kLanes, gv.num_sms * 8, stream)) != cudaSuccess)
        return fail_enqueued(ISO_E_CUDA, "emit launch", e, stream);
    GatherParams ga{};
    ga.ebuf = em.ebuf; ga.ecnt = em.ecnt; ga.tmp = (int32_t*)(base + kOffTmp); ga.out = (int32_t*)(base + kOffOut);
    ga.out_off = (int64_t*)(base + kOffOutOff); ga.k = kLanes; ga.ecap = kMaxArcs;
    ga.status = ctl;
    ga.key_bits = 1;
    while (ga.key_bits < 31 && (int64_t(1) << ga.key_bits) < gv.m) ++ga.key_bits;
    ga.m = gv.m;
    if ((e = iso_launch_sort_gather(ga, kLanes, stream)) != cudaSuccess)
        return fail_enqueued(ISO_E_CUDA, "sort launch", e, stream);

    int32_t h_ctl[kCtlWords];
    if ((e = cudaMemcpyAsync(h_ctl, ctl, sizeof h_ctl, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(stream)) != cudaSuccess)
        return fail_enqueued(ISO_E_CUDA, "kernels", e, stream);
    if (h_ctl[0] == kStTimeout) { iso::set_error("iso_query_noalloc: a grid barrier timed out"); return ISO_E_TIMEOUT; }
    if (h_ctl[0] == kStBadInput) { iso::set_error("iso_query_noalloc: a source or limit failed validation"); return ISO_E_INVAL; }
    if (h_ctl[0] == kStUpOverflow) {
        iso::set_error("iso_query_noalloc: an upward search exceeds %d vertices", kMaxUpward);
        return ISO_E_INVAL;
    }
    int64_t off[kLanes + 1] = {0};
    for (int i = 0; i < k; ++i) {
        if (h_ctl[8 + i] > kMaxArcs) {
            iso::set_error("iso_query_noalloc: query %d has %d isochrone edges, the limit is %d", i, h_ctl[8 + i],
                           kMaxArcs);
            return ISO_E_INVAL;
        }
        off[i + 1] = off[i] + h_ctl[8 + i];
    }
    const int64_t total = off[k];
    if (total > 0 && total <= cap && !out_arcs) { iso::set_error("iso_query_noalloc: out_arcs is NULL"); return ISO_E_INVAL; }
    if ((e = cudaMemcpyAsync(out_offsets, off, (size_t)(k + 1) * 8, cudaMemcpyDefault, stream)) != cudaSuccess)
        return fail_enqueued(ISO_E_CUDA, "offset copy", e, stream);
    int rc = ISO_OK;
    if (total > cap) {
        iso::set_error("iso_query_noalloc: %lld arcs do not fit capacity %lld", (long long)total, (long long)cap);
        rc = ISO_E_OVERFLOW;
    } else if (total > 0) {
        if ((e = cudaMemcpyAsync(out_arcs, base + kOffOut, (size_t)total * 4, cudaMemcpyDefault, stream)) !=
            cudaSuccess)
            return fail_enqueued(ISO_E_CUDA, "result copy", e, stream);
    }
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) return fail_enqueued(ISO_E_CUDA, "result copy", e, stream);
    return rc;
}
