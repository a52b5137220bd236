// Upward search of PHAST (Section 2): from each source s, distances in the
// upward graph G_up = (V, {(u,v) in E u E+ : rank(u) < rank(v)}), pruned at the
// query's limit tau.
//
// One CTA per lane.  Every upward arc ends at a strictly higher CH level, so
// G_up is a DAG and a frontier-based Bellman-Ford over it converges after as
// many rounds as the longest shortest upward path has arcs: each round relaxes
// the out-arcs of every vertex whose label improved in the previous round.  A
// warp takes one frontier vertex at a time and spreads its arcs over its 32
// threads.  Labels live in an open-addressing hash table in shared memory
// (vertex -> label) with a bitmap of the vertices queued for the next round; a
// search space too large for it is redone with the same structures in global
// memory.  Dropping labels above tau is exact because lengths are
// non-negative: every prefix of a path of length <= tau is itself <= tau.
#include "iso_device.cuh"

namespace {

using namespace isod;

constexpr int kThreads = 1024;
constexpr int kSmemSlots = 16384;  // power of two; at most half of them occupied

struct Table {
    int32_t* key;      // vertex or -1
    uint32_t* dist;    // label
    uint32_t* queued;  // bitmap: slot is in the next frontier
    int32_t* fr[2];    // frontier slot lists, capacity = limit
    uint32_t mask;     // slots - 1
    int limit;         // maximum occupied slots
};

__host__ __device__ constexpr size_t table_words(size_t slots) {
    return slots + slots + slots / 32 + slots;  // key, dist, queued bits, two half-size frontiers
}

__device__ __forceinline__ int find_or_insert(const Table& t, int32_t v, int* s_used) {
    uint32_t s = ((uint32_t)v * 0x9E3779B1u) & t.mask;
    for (uint32_t probe = 0; probe <= t.mask; ++probe) {
        const int32_t k = atomicCAS(&t.key[s], -1, v);
        if (k == v) return (int)s;
        if (k == -1) return atomicAdd(s_used, 1) < t.limit ? (int)s : -1;
        s = (s + 1) & t.mask;
    }
    return -1;
}

__device__ __forceinline__ Table carve(uint32_t* base, uint32_t slots) {
    Table t;
    t.key = (int32_t*)base;
    t.dist = base + slots;
    t.queued = base + 2 * slots;
    t.fr[0] = (int32_t*)(base + 2 * slots + slots / 32);
    t.fr[1] = t.fr[0] + slots / 2;
    t.mask = slots - 1;
    t.limit = (int)(slots / 2);
    return t;
}

// Runs the search with table t.  Returns false if the table overflowed.
__device__ bool search(const Table& t, const UpParams& p, int32_t s, uint32_t tau, int lane) {
    __shared__ int s_used, s_nfr, s_next, s_over, s_out, s_core;
    const uint32_t slots = t.mask + 1;
    const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
        t.key[i] = -1;
        t.dist[i] = kInf;
    }
    for (uint32_t i = threadIdx.x; i < slots / 32; i += blockDim.x) t.queued[i] = 0;
    if (threadIdx.x == 0) { s_used = 0; s_over = 0; s_out = 0; s_core = 0; }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int sl = find_or_insert(t, s, &s_used);
        t.dist[sl] = 0;
        t.fr[0][0] = sl;
        s_nfr = 1;
    }
    __syncthreads();
    for (int r = 0; s_nfr > 0; ++r) {
        const int32_t* cur = t.fr[r & 1];
        int32_t* nxt = t.fr[(r + 1) & 1];
        const int nfr = s_nfr;
        // a vertex leaves the queue when its round starts; a later improvement re-queues it
        for (int i = threadIdx.x; i < nfr; i += blockDim.x) atomicAnd(&t.queued[cur[i] >> 5], ~(1u << (cur[i] & 31)));
        if (threadIdx.x == 0) s_next = 0;
        __syncthreads();
        for (int f = warp; f < nfr; f += nwarps) {
            const int su = cur[f];
            const int32_t u = t.key[su];
            const uint32_t du = *((volatile uint32_t*)&t.dist[su]);
            const uint32_t a1 = __ldg(p.up_off + u + 1);
            for (uint32_t a = __ldg(p.up_off + u) + wl; a < a1; a += 32) {
                const int2 arc = __ldg(&p.up_arc[a]);
                const uint32_t nd = du + (uint32_t)arc.y;
                if (nd > tau) continue;
                const int sx = find_or_insert(t, arc.x, &s_used);
                if (sx < 0) { s_over = 1; continue; }
                if (nd < atomicMin(&t.dist[sx], nd)) {
                    const uint32_t bit = 1u << (sx & 31);
                    if (!(atomicOr(&t.queued[sx >> 5], bit) & bit)) nxt[atomicAdd(&s_next, 1)] = sx;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_nfr = s_over ? 0 : s_next;
        __syncthreads();
    }
    if (s_over) return false;
    if (p.direct) {
        // labels go straight into their row slots (other lanes own the other
        // slots); those of the top core [0, core_n), which the sweep resolves
        // per lane, go to the lane's pair list instead
        int2* core = p.pairs + (size_t)lane * p.cap;
        for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
            const int32_t v = t.key[i];
            if (v >= 0) {
                if (v < p.core_n) {
                    core[atomicAdd(&s_core, 1)] = make_int2(v, (int)t.dist[i]);
                } else {
                    p.d[(size_t)v * p.K + lane] = t.dist[i];
                    atomicOr(p.upmask + v, 1ull << lane);
                    p.upflag[v] = 1;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_out = s_core;
    } else {
        int2* out = p.pairs + (size_t)lane * p.cap;
        for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
            const int32_t v = t.key[i];
            if (v >= 0) out[atomicAdd(&s_out, 1)] = make_int2(v, (int)t.dist[i]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) p.cnt[lane] = s_out;
    return true;
}

__global__ void __launch_bounds__(kThreads) k_upward(UpParams p) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = blockIdx.x;
    const int32_t src = p.src[lane];
    const int32_t tau = p.tau[lane];
    if (src < 0) {                                   // idle lane
        if (threadIdx.x == 0) p.cnt[lane] = 0;
        return;
    }
    if (src >= p.n || tau < 0 || tau > p.tau_max) {
        if (threadIdx.x == 0) { p.cnt[lane] = 0; atomicCAS(p.status, kStOk, kStBadInput); }
        return;
    }
    const int32_t s = p.pos[src];
    const bool small_cap = !p.direct && p.cap < kSmemSlots / 2;   // pairs must hold every label
    if (!small_cap && search(carve(smem, kSmemSlots), p, s, (uint32_t)tau, lane)) return;
    // Too large for shared memory: the same search on this lane's global table.
    __syncthreads();
    uint32_t* base = p.gtab + (size_t)lane * table_words((size_t)p.gcap);
    if (!search(carve(base, (uint32_t)p.gcap), p, s, (uint32_t)tau, lane)) {
        if (threadIdx.x == 0) { p.cnt[lane] = 0; atomicCAS(p.status, kStOk, kStUpOverflow); }
    }
}

}  // namespace

size_t iso_upward_table_words(size_t gcap) { return table_words(gcap); }

cudaError_t iso_launch_upward(const isod::UpParams& p, int K, cudaStream_t s) {
    const size_t smem = table_words(kSmemSlots) * 4;  // 194 KB
    static std::atomic<unsigned long long> attr{0};
    if (cudaError_t e = iso_smem_attr_once(k_upward, (int)smem, attr)) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(K);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = iso_high_priority();
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_upward, p);
}
