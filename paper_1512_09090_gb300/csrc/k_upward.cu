// Upward search of PHAST (Section 2): from each source s, distances in the
// upward graph G_up = (V, {(u,v) in E u E+ : rank(u) < rank(v)}), pruned at the
// query's limit tau.
//
// One CTA per lane.  Every upward arc ends at a strictly higher CH level, so
// G_up is a DAG and a frontier-based Bellman-Ford over it converges after as
// many rounds as the longest shortest upward path has arcs: each round relaxes
// the out-arcs of every vertex whose label improved in the previous round.
// Labels live in an open-addressing hash table in shared memory (vertex ->
// label); a search space too large for it is redone with a table in global
// memory.  Dropping labels above tau is exact because lengths are non-negative:
// every prefix of a path of length <= tau is itself <= tau.
#include "iso_device.cuh"

namespace {

using namespace isod;

constexpr int kThreads = 512;
constexpr int kSmemSlots = 8192;  // power of two

struct Table {
    int32_t* key;     // vertex or -1
    uint32_t* dist;   // label
    int32_t* stamp;   // last round in which the slot was queued
    int32_t* fr[2];   // frontier slot lists
    uint32_t mask;    // slots - 1
    int limit;        // maximum occupied slots before giving up
};

__device__ __forceinline__ int find_or_insert(const Table& t, int32_t v, int* s_used) {
    uint32_t s = ((uint32_t)v * 0x9E3779B1u) & t.mask;
    for (uint32_t probe = 0; probe <= t.mask; ++probe) {
        int32_t k = atomicCAS(&t.key[s], -1, v);
        if (k == v) return (int)s;
        if (k == -1) {
            if (atomicAdd(s_used, 1) >= t.limit) return -1;
            return (int)s;
        }
        s = (s + 1) & t.mask;
    }
    return -1;
}

// Runs the search with table t.  Returns false if the table overflowed.
__device__ bool search(const Table& t, const UpParams& p, int32_t s, uint32_t tau, int lane) {
    __shared__ int s_used, s_nfr, s_next, s_over, s_out;
    const uint32_t slots = t.mask + 1;
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
        t.key[i] = -1;
        t.dist[i] = kInf;
        t.stamp[i] = -1;
    }
    if (threadIdx.x == 0) { s_used = 0; s_over = 0; s_out = 0; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int sl = find_or_insert(t, s, &s_used);
        t.dist[sl] = 0;
        t.stamp[sl] = 0;
        t.fr[0][0] = sl;
        s_nfr = 1;
    }
    __syncthreads();
    for (int r = 0; s_nfr > 0; ++r) {
        const int32_t* cur = t.fr[r & 1];
        int32_t* nxt = t.fr[(r + 1) & 1];
        const int nfr = s_nfr;
        if (threadIdx.x == 0) s_next = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < nfr; i += blockDim.x) {
            const int su = cur[i];
            const int32_t u = t.key[su];
            const uint32_t du = *((volatile uint32_t*)&t.dist[su]);
            for (uint32_t a = p.up_off[u], e = p.up_off[u + 1]; a < e; ++a) {
                const int2 arc = __ldg(&p.up_arc[a]);
                const uint32_t nd = du + (uint32_t)arc.y;
                if (nd > tau) continue;
                const int sx = find_or_insert(t, arc.x, &s_used);
                if (sx < 0) { s_over = 1; continue; }
                if (nd < atomicMin(&t.dist[sx], nd)) {
                    if (atomicExch(&t.stamp[sx], r + 1) != r + 1) {
                        int q = atomicAdd(&s_next, 1);
                        if (q < t.limit) nxt[q] = sx;
                        else s_over = 1;
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_nfr = s_over ? 0 : s_next;
        __syncthreads();
    }
    if (s_over) return false;
    int2* out = p.pairs + (size_t)lane * p.cap;
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
        const int32_t v = t.key[i];
        if (v >= 0) {
            int q = atomicAdd(&s_out, 1);
            out[q] = make_int2(v, (int)t.dist[i]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) p.cnt[lane] = s_out;
    return true;
}

__global__ void __launch_bounds__(kThreads) k_upward(UpParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
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
    Table t;
    t.key = (int32_t*)smem;
    t.dist = (uint32_t*)(t.key + kSmemSlots);
    t.stamp = (int32_t*)(t.dist + kSmemSlots);
    t.fr[0] = t.stamp + kSmemSlots;
    t.fr[1] = t.fr[0] + kSmemSlots / 2;
    t.mask = kSmemSlots - 1;
    t.limit = kSmemSlots / 2;
    if (search(t, p, s, (uint32_t)tau, lane)) return;
    // Too large for shared memory: same search on this lane's global table.
    const size_t g = (size_t)p.gcap;
    uint32_t* base = p.gtab + (size_t)lane * 5 * g;
    t.key = (int32_t*)base;
    t.dist = base + g;
    t.stamp = (int32_t*)(base + 2 * g);
    t.fr[0] = (int32_t*)(base + 3 * g);
    t.fr[1] = (int32_t*)(base + 4 * g);
    t.mask = (uint32_t)g - 1;
    t.limit = (int)(g / 2);
    __syncthreads();
    if (!search(t, p, s, (uint32_t)tau, lane)) {
        if (threadIdx.x == 0) { p.cnt[lane] = 0; atomicCAS(p.status, kStOk, kStUpOverflow); }
    }
}

}  // namespace

cudaError_t iso_launch_upward(const isod::UpParams& p, int K, cudaStream_t s) {
    const size_t smem = (size_t)kSmemSlots * 4 * 4;  // key, dist, stamp, two half frontiers
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_upward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_upward<<<K, kThreads, smem, s>>>(p);
    return cudaGetLastError();
}
