// The top core of the hierarchy, swept for each lane by one CTA (first part of
// PHAST's scanning phase, Section 2).
//
// The top level blocks of a contraction hierarchy hold few vertices but form a
// long chain of dependent levels.  Section 5 of the paper sweeps the topmost
// vertices as a separate small graph before the rest; here that graph is small
// enough (at most kCoreMaxVertices vertices) for one lane's labels to sit in a
// CTA's shared memory, so each level of the chain costs a CTA barrier instead
// of a round trip between SMs.  CTA i handles lane i:
//   - labels start at kInf, then take the lane's upward labels of core
//     vertices (the upward search leaves those as (vertex, label) pairs);
//   - level blocks 0 .. core_levels-1 in order: every thread takes arcs of the
//     level (coalesced 8-byte records {src | head << 16, len}, eight loads in
//     flight per thread) and lowers the head's label with a shared-memory
//     atomicMin; the first arcs of the next two levels are read ahead, since
//     they do not depend on labels;
//   - the final labels, clamped to kInf above tau, go to row i of a lane-major
//     array (coalesced); the sweep kernel transposes them into the label rows.
// Labels above tau are not pruned before the end: a value above tau only ever
// produces values above tau, and a uint32 sum of a label <= 0x7FFFFFFF and a
// length <= 0x7FFFFFFE cannot wrap, so the clamped result is PHAST's.
//
// This is a separate kernel, not a phase of k_sweep_tma, because its shared
// memory (up to 212 KB) would shrink the L1 that the sweep's gathers need.
// It has no waits on other CTAs.  The sweep kernel that follows writes the
// label rows and in-range masks of these vertices.
#include "iso_device.cuh"

namespace {

using namespace isod;

constexpr int kThreads = 1024;
constexpr int kBatch = 8;  // arc loads in flight per thread

__device__ __forceinline__ void relax(uint32_t* lab, uint2 a) {
    const uint32_t x = lab[a.x & 0xFFFFu] + a.y;
    if (x < kInf) atomicMin(lab + (a.x >> 16), x);
}

__global__ void __launch_bounds__(kThreads, 1) k_core(SweepParams p) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* lab = smem;                      // [core_n]
    uint32_t* larc = smem + kCoreMaxVertices;  // [core_levels + 1]
    const int tid = threadIdx.x, b = blockIdx.x;
    const int cn = p.core_n, C = p.core_levels;
    if (p.trace && b == 0 && tid == 0) p.trace[0] = p.trace[p.L + 1] = (long long)global_ns();
    for (int v = tid; v < cn; v += kThreads) lab[v] = kInf;
    for (int j = tid; j <= C; j += kThreads) larc[j] = __ldg(p.level_arc + j);
    __syncthreads();
    const int np = p.cnt[b];
    const int2* pr = p.pairs + (size_t)b * p.cap;
    for (int i = tid; i < np; i += kThreads) {
        const int2 q = pr[i];
        lab[q.x] = (uint32_t)q.y;
    }
    __syncthreads();
    // first arcs of levels j (pre0) and j + 1 (pre1), read two levels ahead
    auto first = [&](int j, bool& has) {
        has = j < C && larc[j] + tid < larc[j + 1];
        return has ? __ldg(p.core_arc + larc[j] + tid) : make_uint2(0u, 0u);
    };
    bool h0, h1, h2;
    uint2 pre0 = first(0, h0), pre1 = first(1, h1);
    for (int j = 0; j < C; ++j) {
        const uint2 pre2 = first(j + 2, h2);
        if (h0) relax(lab, pre0);
        const uint32_t a1 = larc[j + 1];
        for (uint32_t a = larc[j] + tid + kThreads; a < a1; a += kBatch * kThreads) {
            uint2 q[kBatch];
#pragma unroll
            for (int r = 0; r < kBatch; ++r)
                q[r] = a + r * kThreads < a1 ? __ldg(p.core_arc + a + r * kThreads) : make_uint2(0u, 0u);
            // all label reads first (sources lie in earlier levels, so no
            // update of this level can change them), then the updates
            uint32_t x[kBatch];
#pragma unroll
            for (int r = 0; r < kBatch; ++r)
                x[r] = a + r * kThreads < a1 ? lab[q[r].x & 0xFFFFu] + q[r].y : kInf;
#pragma unroll
            for (int r = 0; r < kBatch; ++r)
                if (x[r] < kInf) atomicMin(lab + (q[r].x >> 16), x[r]);
        }
        __syncthreads();
        if (p.trace && b == 0 && tid == 0) atomicMax((unsigned long long*)p.trace + 1 + j, global_ns());
        pre0 = pre1; h0 = h1; pre1 = pre2; h1 = h2;
    }
    const uint32_t tau = p.tau[b] < 0 ? 0u : (uint32_t)p.tau[b];
    uint32_t* out = p.core_out + (size_t)b * cn;
    for (int v = tid; v < cn; v += kThreads) {
        const uint32_t x = lab[v];
        out[v] = x > tau ? kInf : x;
    }
}

constexpr int kCoreSmem = (kCoreMaxVertices + kCoreMaxLevels + 1) * 4;

}  // namespace

cudaError_t iso_launch_core(const isod::SweepParams& p, int K, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    if (cudaError_t e = iso_smem_attr_once(k_core, kCoreSmem, attr)) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(K);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kCoreSmem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = iso_high_priority();  // ahead of the previous batch's emission and sort
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_core, p);
}
