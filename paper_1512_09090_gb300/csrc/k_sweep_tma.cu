// PHAST scanning phase (Section 2) for K queries at once, pruned at tau, with
// the downward-arc blocks staged through shared memory by TMA bulk copies.
//
// Same computation as k_sweep.cu: for every vertex v (descending CH level) and
// lane i, d[v,i] = min(up_i(v), min over downward arcs (u,v) of d[u,i] +
// len(u,v)), and 0x7FFFFFFF when that exceeds tau_i (exact for non-negative
// lengths); uint32 arithmetic never wraps because labels are <= 0x7FFFFFFF and
// lengths <= 0x7FFFFFFE.
//
// The upward search has already written each lane's labels into the rows
// (upmask[v] says which lanes), so the walk starts at once.
//
// Work is cut into chunks of VPB consecutive vertices of one level and run in
// the order of a host-built schedule (schedule.cpp) that interleaves levels
// region by region for L2 reuse; schedule position q belongs to CTA q mod G.
// Each CTA (1024 threads, one per SM) has 31 consumer warps and one producer
// warp.
// The producer walks the CTA's chunks and copies each chunk's CSR offsets and
// its contiguous block of incoming downward arcs into one of kStages shared-
// memory buffers with cp.async.bulk, completing on the buffer's "full"
// mbarrier; consumers release a buffer on its "empty" mbarrier, and the last
// consumer warp to finish a chunk marks its position complete.  There are no
// grid barriers: after starting the copy of chunk q (read-only graph data) the
// producer warp waits until every position q depends on is complete and posts
// that in shared memory; only then do the consumers gather the label rows d[u]
// of q, with ld.global.cg.  Narrow levels use a warp per vertex: its groups of TPV
// threads take every (32/TPV)-th arc, so a vertex with many arcs needs one
// round of gathers, and chunks are 31 vertices so more CTAs share the level.
//
// Every wait (mbarrier, dependency flags) is bounded: past the limit
// the kernel records kStTimeout, stops issuing copies, waits (bounded) for the
// copies it already issued, and returns.
#include "iso_device.cuh"

namespace {

using namespace isod;

constexpr int kThreads = 1024;
constexpr int kConsumers = 992;          // warps 0..30; warp 31 produces
constexpr int kStages = 3;
constexpr int kArcCap = 4096;            // arcs per stage buffer
constexpr int kOffCap = 1024;            // offsets per stage buffer (>= VPB + 5)

template <int K> struct MaskOf { using T = uint8_t; };
template <> struct MaskOf<16> { using T = uint16_t; };
template <> struct MaskOf<32> { using T = uint32_t; };
template <> struct MaskOf<64> { using T = unsigned long long; };

struct Meta {
    int v0, v1;   // vertices [v0, v1)
    int abase;    // first arc index held in the stage buffer
    int flags;    // bit 0: arcs did not fit (read them from global memory); bit 1: warp per vertex
    int q, level; // schedule position and level block
    int pad[2];
};

struct Smem {
    int2 arcs[kStages][kArcCap];
    uint32_t tau[64];
    uint32_t offs[kStages][kOffCap];
    Meta meta[kStages];
    unsigned long long full[kStages];
    unsigned long long empty[kStages];
    int finished[kStages];  // consumer warps done with the chunk in each stage
    int ready_it[kStages];  // chunk (CTA-local index + 1) whose dependencies were seen complete
    int ok;
};

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, uint32_t tx) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(tx) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(sa(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sa(dst)),
                 "l"(src), "r"(bytes), "r"(sa(b))
                 : "memory");
}

// Bounded wait for phase `parity` of barrier b.  false = gave up (status set).
__device__ bool mbar_wait(unsigned long long* b, uint32_t parity, const SweepParams& p) {
    if (mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(b, parity)) return true;
        if ((it & 63) == 0) {
            if (*(volatile int32_t*)p.status != kStOk) return false;
            if (global_ns() - t0 > (unsigned long long)p.timeout_ns || it > (1u << 28)) {
                atomicCAS(p.status, kStOk, kStTimeout);
                return false;
            }
        }
    }
}

template <int LPT> struct Row { uint32_t x[LPT]; };

// Lane layout of a row: the K labels form K/4 quads of 16 bytes; thread `sub`
// of a vertex's group owns quads sub, sub+TPV, sub+2*TPV, ..., so every warp-wide
// vector load or store covers whole contiguous segments of the row.  Element i
// of a thread's Row is lane 4*(sub + TPV*(i/4)) + i%4.
template <int LPT, int TPV>
__device__ __forceinline__ Row<LPT> load_row(const uint32_t* row, int sub) {
    Row<LPT> r;
    if constexpr (LPT >= 4) {
#pragma unroll
        for (int q = 0; q < LPT / 4; ++q) {
            const uint4 v = __ldcg(reinterpret_cast<const uint4*>(row) + sub + TPV * q);
            r.x[4 * q] = v.x; r.x[4 * q + 1] = v.y; r.x[4 * q + 2] = v.z; r.x[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < LPT; ++q) r.x[q] = __ldcg(row + sub * LPT + q);
    }
    return r;
}

template <int LPT, int TPV>
__device__ __forceinline__ void store_row(uint32_t* row, int sub, const Row<LPT>& r) {
    if constexpr (LPT >= 4) {
#pragma unroll
        for (int q = 0; q < LPT / 4; ++q)
            reinterpret_cast<uint4*>(row)[sub + TPV * q] =
                make_uint4(r.x[4 * q], r.x[4 * q + 1], r.x[4 * q + 2], r.x[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < LPT; ++q) row[sub * LPT + q] = r.x[q];
    }
}

// Lane of element i of thread `sub`'s Row.
template <int LPT, int TPV>
__device__ __forceinline__ int lane_of(int sub, int i) {
    if constexpr (LPT >= 4) return 4 * (sub + TPV * (i / 4)) + (i & 3);
    else return sub * LPT + i;
}

// The CTA's chunks: schedule position q belongs to CTA q mod G, and every CTA
// takes its positions in increasing order.  Both warp roles walk this order.
struct ChunkWalk {
    const SweepParams& p;
    int q;
    __device__ explicit ChunkWalk(const SweepParams& pp) : p(pp), q(blockIdx.x) {}
    // Next chunk: vertices [v0, v1) of level block blk at position pos, with a
    // thread group (mode 0) or a warp (mode 1) per vertex.  false at the end.
    __device__ bool next(int& v0, int& v1, int& blk, int& mode, int& pos) {
        if (q >= p.Q) return false;
        const int4 c = p.sched_info[q];
        v0 = c.x; v1 = c.y; blk = c.z; mode = c.w; pos = q;
        q += gridDim.x;
        return true;
    }
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* a) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

// Bounded wait, by a whole warp, until every position schedule position q
// depends on is complete (plus bar_extra flags that never come when a test asks
// for a timeout).  Returns false, the same on every lane, if it gave up.
__device__ bool wait_deps(const SweepParams& p, int q, int lane) {
    const int a = p.pred_off[q], b_real = p.pred_off[q + 1], b = b_real + p.bar_extra;
    const unsigned long long t0 = global_ns();
    for (int base = a; base < b; base += 128) {
        // up to four flags per lane, all loads in flight at once
        bool mine[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int i = base + lane + 32 * t;
            mine[t] = i >= b || (i < b_real && ld_acquire(reinterpret_cast<const uint32_t*>(p.done + p.pred[i])) != 0u);
        }
        uint32_t nap = 32;
        for (uint32_t it = 0; !__all_sync(0xffffffffu, mine[0] && mine[1] && mine[2] && mine[3]); ++it) {
            __nanosleep(nap);
            if (nap < 256) nap <<= 1;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int i = base + lane + 32 * t;
                if (!mine[t] && i < b_real)
                    mine[t] = ld_acquire(reinterpret_cast<const uint32_t*>(p.done + p.pred[i])) != 0u;
            }
            int give_up = 0;
            if (lane == 0 && (it & 15) == 15) {
                if (*(volatile int32_t*)p.status != kStOk) give_up = 1;
                else if (global_ns() - t0 > (unsigned long long)p.timeout_ns || it > (1u << 26)) {
                    atomicCAS(p.status, kStOk, kStTimeout);
                    give_up = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, give_up, 0)) return false;
        }
    }
    return true;
}

// Gathers rows d[u] + len(u,v) for arcs a, a+STEP, a+2*STEP, ... < e into acc.
template <int K, int LPT, int TPV, int STEP>
__device__ __forceinline__ void gather(Row<LPT>& acc, const uint32_t* d, const int2* arcs, uint32_t a, uint32_t e,
                                       int sub) {
    for (; a + 3 * STEP < e; a += 4 * STEP) {
        const int2 a0 = arcs[a], a1 = arcs[a + STEP], a2 = arcs[a + 2 * STEP], a3 = arcs[a + 3 * STEP];
        const Row<LPT> r0 = load_row<LPT, TPV>(d + (size_t)a0.x * K, sub);
        const Row<LPT> r1 = load_row<LPT, TPV>(d + (size_t)a1.x * K, sub);
        const Row<LPT> r2 = load_row<LPT, TPV>(d + (size_t)a2.x * K, sub);
        const Row<LPT> r3 = load_row<LPT, TPV>(d + (size_t)a3.x * K, sub);
#pragma unroll
        for (int i = 0; i < LPT; ++i) {
            const uint32_t m01 = min(r0.x[i] + (uint32_t)a0.y, r1.x[i] + (uint32_t)a1.y);
            const uint32_t m23 = min(r2.x[i] + (uint32_t)a2.y, r3.x[i] + (uint32_t)a3.y);
            acc.x[i] = min(acc.x[i], min(m01, m23));
        }
    }
    for (; a < e; a += STEP) {
        const int2 a0 = arcs[a];
        const Row<LPT> r0 = load_row<LPT, TPV>(d + (size_t)a0.x * K, sub);
#pragma unroll
        for (int i = 0; i < LPT; ++i) acc.x[i] = min(acc.x[i], r0.x[i] + (uint32_t)a0.y);
    }
}

// Starts pulling the rows of arcs a, a+step, ... < e into L2 (no registers, no
// shared memory: cp.async.bulk.prefetch).  Stale or not-yet-final rows are
// harmless there: every later store lands in L2 as well.
__device__ __forceinline__ void prefetch_rows(const uint32_t* d, int K, const int2* arcs, uint32_t a, uint32_t e,
                                              uint32_t step) {
    const uint32_t bytes = (uint32_t)K * 4u;
    for (; a < e; a += step) {
        const uint32_t* row = d + (size_t)arcs[a].x * K;
        if (bytes >= 16)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(row), "r"(bytes) : "memory");
        else
            asm volatile("prefetch.global.L2 [%0];" ::"l"(row) : "memory");
    }
}

template <int K, int TPV>
__global__ void __launch_bounds__(kThreads, 1) k_sweep_tma(SweepParams p) {
    constexpr int LPT = K / TPV;
    constexpr int VPB = kConsumers / TPV;
    static_assert(VPB + 5 <= kOffCap, "offset buffer");
    using MaskT = typename MaskOf<K>::T;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&sm.full[i], 1);
            mbar_init(&sm.empty[i], kConsumers / 32);
            sm.finished[i] = 0;
            sm.ready_it[i] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp == kConsumers / 32) {
        // ---------------- producer warp: checks dependencies, copies chunks ----------------
        ChunkWalk walk(p);
        int it = 0;
        int v0, v1, blk, mode, pos;
        while (walk.next(v0, v1, blk, mode, pos)) {
            const int stage = it % kStages;
            const uint32_t round = (uint32_t)(it / kStages);
            int fine = 1;
            if (lane == 0) fine = mbar_wait(&sm.empty[stage], (round & 1u) ^ 1u, p);
            fine = __shfl_sync(0xffffffffu, fine, 0);
            if (!fine) break;
            if (lane == 0) {
                const uint32_t off0 = __ldg(p.down_off + v0), off1 = __ldg(p.down_off + v1);
                const int ob = v0 & ~3;
                const uint32_t obytes = (uint32_t)(((v1 + 1 - ob) * 4 + 15) & ~15);
                const uint32_t ab = off0 & ~1u;
                const uint32_t na = off1 - ab;
                const bool big = na > (uint32_t)kArcCap;
                const uint32_t abytes = big ? 0u : ((na * 8u + 15u) & ~15u);
                sm.meta[stage] = Meta{v0, v1, (int)ab, (big ? 1 : 0) | (mode ? 2 : 0), pos, blk, {0, 0}};
                mbar_expect_tx(&sm.full[stage], obytes + abytes);
                bulk_load(sm.offs[stage], p.down_off + ob, obytes, &sm.full[stage]);
                if (abytes) bulk_load(sm.arcs[stage], p.down_arc + ab, abytes, &sm.full[stage]);
            }
            __syncwarp();
            ++it;
            // the copy is in flight; meanwhile wait for the chunk's dependencies
            // and tell the consumers when its rows may be gathered
            if (!wait_deps(p, pos, lane)) break;
            __threadfence_block();
            if (lane == 0) *(volatile int*)&sm.ready_it[stage] = it;
        }
        // every issued copy must land before the CTA exits
        if (lane == 0)
            for (int i = it > kStages ? it - kStages : 0; i < it; ++i)
                mbar_wait(&sm.full[i % kStages], (uint32_t)(i / kStages) & 1u, p);
        __syncthreads();
        return;
    }

    // ---------------- consumer warps ----------------
    // mode 0: a group of TPV threads per vertex; mode 1: a warp per vertex whose
    // GPV groups take every GPV-th arc and then combine with shuffles
    constexpr int GPV = 32 / TPV;
    const int sub = tid % TPV;
    if (tid < K) {
        const int32_t t = p.tau[tid];
        sm.tau[tid] = t < 0 ? 0u : (uint32_t)t;
    }
    if (tid == 0) sm.ok = 0;  // positions below sm.ok are known complete
    asm volatile("bar.sync 1, 992;" ::: "memory");
    if (p.trace && tid == 0 && blockIdx.x == 0) p.trace[0] = p.trace[p.L + 1] = (long long)global_ns();

    ChunkWalk walk(p);
    bool alive = true;
    int it = 0;
    int v0, v1, j, mode, pos;
    while (walk.next(v0, v1, j, mode, pos)) {
        const int stage = it % kStages;
        const uint32_t round = (uint32_t)(it / kStages);
        ++it;
        // the producer posts ready_it once every position the chunk depends on is
        // complete; only then may its rows be gathered
        if (alive && lane == 0) {
            const unsigned long long t0 = global_ns();
            for (uint32_t n = 0; *(volatile int*)&sm.ready_it[stage] != it; ++n) {
                __nanosleep(32);
                if ((n & 255) == 255 && (*(volatile int32_t*)p.status != kStOk ||
                                         global_ns() - t0 > (unsigned long long)p.timeout_ns)) {
                    atomicCAS(p.status, kStOk, kStTimeout);
                    alive = false;
                    break;
                }
            }
        }
        alive = __shfl_sync(0xffffffffu, alive, 0);
        __threadfence_block();
        const bool ready = __all_sync(0xffffffffu, alive && mbar_wait(&sm.full[stage], round & 1u, p));
        if (ready) {
            const Meta mt = sm.meta[stage];
            const int ob = mt.v0 & ~3;
            const int g = mode ? lane / TPV : 0;         // arc group within the vertex
            const int v = mode ? v0 + warp : v0 + tid / TPV;
            const bool valid = v < v1;
            const bool store = p.write_all || j != p.last_level_block;
            Row<LPT> acc;
#pragma unroll
            for (int i = 0; i < LPT; ++i) acc.x[i] = kInf;
            uint32_t a = 0, e = 0, flagged = 0;
            if (valid) {
                flagged = __ldcg(p.upflag + v);
                a = sm.offs[stage][v - ob] + g;
                e = sm.offs[stage][v + 1 - ob];
            }
            const int2* arcs = (mt.flags & 1) ? p.down_arc : sm.arcs[stage] - mt.abase;
            // the CTA's next chunk is usually staged already: warm L2 with its rows
            if (sub == 0 && mbar_try_wait(&sm.full[it % kStages], (uint32_t)(it / kStages) & 1u)) {
                const Meta nx = sm.meta[it % kStages];
                const int nm = (nx.flags >> 1) & 1;
                const int nv = nm ? nx.v0 + warp : nx.v0 + tid / TPV;
                if (nv < nx.v1 && !(nx.flags & 1)) {
                    const int nob = nx.v0 & ~3;
                    const uint32_t* noffs = sm.offs[it % kStages];
                    prefetch_rows(p.d, K, sm.arcs[it % kStages] - nx.abase, noffs[nv - nob] + (nm ? lane / TPV : 0),
                                  noffs[nv + 1 - nob], nm ? GPV : 1);
                }
            }
            if (mode) gather<K, LPT, TPV, GPV>(acc, p.d, arcs, a, e, sub);
            else gather<K, LPT, TPV, 1>(acc, p.d, arcs, a, e, sub);
            if (mode) {
#pragma unroll
                for (int o = TPV; o < 32; o <<= 1) {
#pragma unroll
                    for (int i = 0; i < LPT; ++i) acc.x[i] = min(acc.x[i], __shfl_xor_sync(0xffffffffu, acc.x[i], o));
                }
            }
            if (flagged) {
                // upward labels: only the lanes marked in upmask hold this batch's values
                const unsigned long long um = __ldcg(p.upmask + v);
                const Row<LPT> own = load_row<LPT, TPV>(p.d + (size_t)v * K, sub);
#pragma unroll
                for (int i = 0; i < LPT; ++i)
                    if ((um >> lane_of<LPT, TPV>(sub, i)) & 1ull) acc.x[i] = min(acc.x[i], own.x[i]);
            }
            __syncwarp();  // every thread of the vertex has read flag and mask before they are cleared
            if (flagged && g == 0 && sub == 0) { p.upflag[v] = 0; p.upmask[v] = 0ull; }
            unsigned long long bits = 0;
#pragma unroll
            for (int i = 0; i < LPT; ++i) {
                const int ln = lane_of<LPT, TPV>(sub, i);
                if (acc.x[i] > sm.tau[ln]) acc.x[i] = kInf;
                else bits |= 1ull << ln;
            }
            if (valid && store && g == 0) store_row<LPT, TPV>(p.d + (size_t)v * K, sub, acc);
#pragma unroll
            for (int o = 1; o < TPV; o <<= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
            if (valid && sub == 0 && g == 0) static_cast<MaskT*>(p.mask)[v] = (MaskT)bits;
        }
        __syncwarp();
        if (lane == 0) {
            // the last warp to finish the chunk publishes it to the other CTAs
            __threadfence_block();
            if (atomicAdd(&sm.finished[stage], 1) == kConsumers / 32 - 1) {
                __threadfence_block();
                sm.finished[stage] = 0;
                __threadfence();
                *(volatile int32_t*)(p.done + pos) = 1;
                if (p.trace) atomicMax((unsigned long long*)p.trace + 1 + j, global_ns());
            }
            mbar_arrive(&sm.empty[stage]);
        }
    }
    __syncthreads();
}

template <int K, int TPV>
cudaError_t launch(const SweepParams& p, int grid, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep_tma<K, TPV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(Smem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = sizeof(Smem);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_sweep_tma<K, TPV>, p);
}

template <int K, int TPV>
int occupancy() {
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_sweep_tma<K, TPV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(Smem)) != cudaSuccess)
            return 0;
        attr = true;
    }
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_sweep_tma<K, TPV>, kThreads, sizeof(Smem)) !=
        cudaSuccess)
        return 0;
    return blocks;
}

#define ISO_TMA_CASES(X) X(1, 1) X(4, 1) X(8, 1) X(16, 2) X(16, 4) X(32, 4) X(32, 8) X(64, 8) X(64, 16)

}  // namespace

bool iso_sweep_tma_supported(int K, int tpv) {
#define X(k, t) if (K == k && tpv == t) return true;
    ISO_TMA_CASES(X)
#undef X
    return false;
}

cudaError_t iso_launch_sweep_tma(const isod::SweepParams& p, int K, int tpv, int grid, cudaStream_t s) {
#define X(k, t) if (K == k && tpv == t) return launch<k, t>(p, grid, s);
    ISO_TMA_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

int iso_sweep_tma_occupancy(int K, int tpv, int* block, int* vpb) {
    *block = kThreads;
    *vpb = kConsumers / tpv;
#define X(k, t) if (K == k && tpv == t) return occupancy<k, t>();
    ISO_TMA_CASES(X)
#undef X
    return 0;
}
