// PHAST scanning phase (Section 2) for K queries at once, pruned at tau.
//
// Vertices are stored in descending CH level; level block j (sweep positions
// level_off[j] .. level_off[j+1]) depends only on blocks < j, and vertices of
// one block are independent.  For every vertex v and lane i:
//     d[v,i] = min( up_i(v), min over downward arcs (u,v) of d[u,i] + len(u,v) )
// and d[v,i] becomes 0x7FFFFFFF when it exceeds tau_i, which is exact because
// lengths are non-negative (a path within tau has every prefix within tau).
// Arithmetic is uint32: labels are <= 0x7FFFFFFF and lengths <= 0x7FFFFFFE, so
// d + len never wraps, and a path through an out-of-range label stays > tau.
//
// The kernel is persistent: one cooperative grid walks all levels, with a
// grid-wide barrier between steps.  Runs of narrow levels are done by CTA 0
// alone with block barriers (one grid barrier per run).  A group of TPV threads
// owns a vertex; each thread owns K/TPV consecutive lanes, so a row of K int32
// labels is read and written as contiguous 16-byte vectors.  Labels written
// earlier in the same launch are read with ld.global.cg so no SM can hit a stale
// L1 line.  Every barrier wait is bounded by a time limit after which the
// kernel records kStTimeout and returns.
#include <cooperative_groups.h>

#include "iso_device.cuh"

namespace {

using namespace isod;

constexpr int kThreads = 512;

template <int K> struct MaskOf { using T = uint8_t; };
template <> struct MaskOf<16> { using T = uint16_t; };
template <> struct MaskOf<32> { using T = uint32_t; };
template <> struct MaskOf<64> { using T = unsigned long long; };

__device__ bool grid_sync(const SweepParams& p) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile int32_t* st = p.status;
        volatile uint32_t* gen = p.bar + 1;
        if (*st != kStOk) {
            ok = 0;
        } else {
            const uint32_t g0 = *gen;
            __threadfence();
            const uint32_t want = gridDim.x + (uint32_t)p.bar_extra;
            if (atomicAdd(p.bar, 1u) + 1u == want) {
                atomicExch(p.bar, 0u);
                __threadfence();
                atomicAdd(p.bar + 1, 1u);
            } else {
                const unsigned long long t0 = global_ns();
                const unsigned long long max_iter = (unsigned long long)p.timeout_ns / 16 + 4096;
                for (unsigned long long it = 0; *gen == g0; ++it) {
                    if (*st != kStOk) { ok = 0; break; }
                    if (global_ns() - t0 > (unsigned long long)p.timeout_ns || it > max_iter) {
                        atomicCAS(p.status, kStOk, kStTimeout);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <int LPT> struct Row { uint32_t x[LPT]; };

template <int LPT>
__device__ __forceinline__ Row<LPT> load_row(const uint32_t* ptr) {
    Row<LPT> r;
    if constexpr (LPT >= 4) {
#pragma unroll
        for (int q = 0; q < LPT / 4; ++q) {
            uint4 v = __ldcg(reinterpret_cast<const uint4*>(ptr) + q);
            r.x[4 * q] = v.x; r.x[4 * q + 1] = v.y; r.x[4 * q + 2] = v.z; r.x[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < LPT; ++q) r.x[q] = __ldcg(ptr + q);
    }
    return r;
}

template <int LPT>
__device__ __forceinline__ void store_row(uint32_t* ptr, const Row<LPT>& r) {
    if constexpr (LPT >= 4) {
#pragma unroll
        for (int q = 0; q < LPT / 4; ++q)
            reinterpret_cast<uint4*>(ptr)[q] = make_uint4(r.x[4 * q], r.x[4 * q + 1], r.x[4 * q + 2], r.x[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < LPT; ++q) ptr[q] = r.x[q];
    }
}

template <int LPT>
__device__ __forceinline__ Row<LPT> load_row_if(const uint32_t* ptr, bool ok) {
    Row<LPT> r;
    if (ok) {
        r = load_row<LPT>(ptr);
    } else {
#pragma unroll
        for (int i = 0; i < LPT; ++i) r.x[i] = kInf;
    }
    return r;
}

// One vertex slot: all TPV threads of a group call this with the same v.
// valid == false keeps the thread in the shuffles without touching memory.
template <int K, int TPV>
__device__ __forceinline__ void scan_vertex(const SweepParams& p, int v, bool valid, bool store_d,
                                            const uint32_t (&tau)[K / TPV], int sub) {
    constexpr int LPT = K / TPV;
    using MaskT = typename MaskOf<K>::T;
    Row<LPT> acc;
#pragma unroll
    for (int i = 0; i < LPT; ++i) acc.x[i] = kInf;
    uint32_t a = 0, e = 0, flagged = 0;
    if (valid) flagged = __ldcg(p.upflag + v);
    __syncwarp();  // every thread of the group has read the flag before it is cleared
    if (flagged) {
        acc = load_row<LPT>(p.d + (size_t)v * K + sub * LPT);
        if (sub == 0) p.upflag[v] = 0;
    }
    if (valid) {
        a = __ldg(p.down_off + v);
        e = __ldg(p.down_off + v + 1);
    }
    // four rows in flight per round, the last round predicated, so a vertex
    // with n arcs waits for ceil(n/4) round trips; a predicated-off row is
    // kInf with length 0 and never lowers the minimum
    for (; a < e; a += 4) {
        const bool o1 = a + 1 < e, o2 = a + 2 < e, o3 = a + 3 < e;
        const int2 a0 = __ldg(p.down_arc + a);
        const int2 a1 = o1 ? __ldg(p.down_arc + a + 1) : make_int2(0, 0);
        const int2 a2 = o2 ? __ldg(p.down_arc + a + 2) : make_int2(0, 0);
        const int2 a3 = o3 ? __ldg(p.down_arc + a + 3) : make_int2(0, 0);
        const Row<LPT> r0 = load_row<LPT>(p.d + (size_t)a0.x * K + sub * LPT);
        const Row<LPT> r1 = load_row_if<LPT>(p.d + (size_t)a1.x * K + sub * LPT, o1);
        const Row<LPT> r2 = load_row_if<LPT>(p.d + (size_t)a2.x * K + sub * LPT, o2);
        const Row<LPT> r3 = load_row_if<LPT>(p.d + (size_t)a3.x * K + sub * LPT, o3);
#pragma unroll
        for (int i = 0; i < LPT; ++i) {
            const uint32_t m01 = min(r0.x[i] + (uint32_t)a0.y, r1.x[i] + (uint32_t)a1.y);
            const uint32_t m23 = min(r2.x[i] + (uint32_t)a2.y, r3.x[i] + (uint32_t)a3.y);
            acc.x[i] = min(acc.x[i], min(m01, m23));
        }
    }
    unsigned long long bits = 0;
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        if (acc.x[i] > tau[i]) acc.x[i] = kInf;
        else bits |= 1ull << i;
    }
    if (valid && store_d) store_row<LPT>(p.d + (size_t)v * K + sub * LPT, acc);
    bits <<= sub * LPT;
#pragma unroll
    for (int o = 1; o < TPV; o <<= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
    if (valid && sub == 0) static_cast<MaskT*>(p.mask)[v] = (MaskT)bits;
}

template <int K, int TPV>
__global__ void __launch_bounds__(kThreads) k_sweep(SweepParams p) {
    constexpr int LPT = K / TPV;
    static_assert(LPT >= 4 || K < 4, "a thread owns at least one 16-byte vector");
    const int tid = threadIdx.x;
    const int sub = tid % TPV;
    const int slot = tid / TPV;
    const int vpb = kThreads / TPV;

    uint32_t tau[LPT];
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        const int32_t t = p.tau[sub * LPT + i];
        tau[i] = t < 0 ? 0u : (uint32_t)t;
    }

    // Upward labels: clear the rows they touch, flag them, then min them in.
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + tid;
    const size_t gsz = (size_t)gridDim.x * blockDim.x;
    for (int lane = 0; lane < K; ++lane) {
        const int c = p.cnt[lane];
        const int2* pr = p.pairs + (size_t)lane * p.cap;
        for (size_t j = gtid; j < (size_t)c; j += gsz) {
            const int v = pr[j].x;
            uint32_t* row = p.d + (size_t)v * K;
            if constexpr (K >= 4) {
#pragma unroll
                for (int q = 0; q < K / 4; ++q) reinterpret_cast<uint4*>(row)[q] = make_uint4(kInf, kInf, kInf, kInf);
            } else {
                row[0] = kInf;
            }
            p.upflag[v] = 1;
        }
    }
    if (!grid_sync(p)) return;
    for (int lane = 0; lane < K; ++lane) {
        const int c = p.cnt[lane];
        const int2* pr = p.pairs + (size_t)lane * p.cap;
        for (size_t j = gtid; j < (size_t)c; j += gsz) {
            const int2 q = pr[j];
            atomicMin(p.d + (size_t)q.x * K + lane, (uint32_t)q.y);
        }
    }
    if (!grid_sync(p)) return;

    for (int s = 0; s < p.nsched; ++s) {
        const int4 st = p.sched[s];
        if (st.x == kStepFused) {
            if (blockIdx.x == 0) {
                for (int j = st.y; j < st.z; ++j) {
                    const int lo = p.level_off[j], hi = p.level_off[j + 1];
                    const bool store = p.write_all || j != p.last_level_block;
                    for (int base = lo; base < hi; base += vpb) {
                        const int v = base + slot;
                        scan_vertex<K, TPV>(p, v, v < hi, store, tau, sub);
                    }
                    __syncthreads();
                }
            }
        } else {
            const int j = st.y;
            const int lo = p.level_off[j], hi = p.level_off[j + 1];
            const bool store = p.write_all || j != p.last_level_block;
            for (int base = lo + blockIdx.x * vpb; base < hi; base += gridDim.x * vpb) {
                const int v = base + slot;
                scan_vertex<K, TPV>(p, v, v < hi, store, tau, sub);
            }
        }
        if (s + 1 < p.nsched && !grid_sync(p)) return;
    }
}

template <int K, int TPV>
cudaError_t launch(const SweepParams& p, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_sweep<K, TPV>, p);
}

template <int K, int TPV>
int occupancy() {
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_sweep<K, TPV>, kThreads, 0) != cudaSuccess)
        return 0;
    return blocks;
}

#define ISO_SWEEP_CASES(X) \
    X(1, 1) X(4, 1) X(8, 1) X(8, 2) X(16, 1) X(16, 2) X(16, 4) X(32, 1) X(32, 2) X(32, 4) X(32, 8) \
    X(64, 1) X(64, 2) X(64, 4) X(64, 8) X(64, 16)

}  // namespace

bool iso_sweep_supported(int K, int tpv) {
#define X(k, t) if (K == k && tpv == t) return true;
    ISO_SWEEP_CASES(X)
#undef X
    return false;
}

cudaError_t iso_launch_sweep(const isod::SweepParams& p, int K, int tpv, int grid, cudaStream_t s) {
#define X(k, t) if (K == k && tpv == t) return launch<k, t>(p, grid, s);
    ISO_SWEEP_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

int iso_sweep_occupancy(int K, int tpv, int* block) {
    *block = kThreads;
#define X(k, t) if (K == k && tpv == t) return occupancy<k, t>();
    ISO_SWEEP_CASES(X)
#undef X
    return 0;
}
