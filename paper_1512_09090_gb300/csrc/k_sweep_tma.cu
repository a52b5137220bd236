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
// (upmask[v] says which lanes), so the walk starts at once.  One persistent
// kernel, launched cooperatively (every CTA resident), in two phases.
//
// Leading levels.  The top of the hierarchy is a long chain of small levels.
// CTA 0 alone sweeps those of at most solo_width vertices (a warp per vertex,
// a CTA barrier per level); then all CTAs sweep the following narrow ones with
// a bounded grid barrier per level, each thread reading its next vertex's arc
// range and first arcs before the barrier that ends the level in front.
//
// Chunk schedule.  Every later level is cut into chunks of VPB consecutive
// vertices (kRounds per thread group) and run in the order of a host-built
// schedule (schedule.cpp) that interleaves levels region by region for L2
// reuse; schedule position q belongs to CTA q mod G.  (Handing positions out
// dynamically from a global counter was measured slower: a CTA then holds
// positions it cannot start for a whole window.)  Each CTA (1024 threads, one
// per SM) has 31 consumer warps and one producer warp and holds up to kStages
// chunks at once.  Lane s of the producer owns stage s: once the buffer is
// free it copies the chunk's CSR offsets, its contiguous block of incoming
// downward arcs and its dependency list (the schedule positions holding
// sources of its arcs) in with cp.async.bulk, completing on the stage's "full"
// mbarrier.  It never blocks: each pass it fills every free buffer, then reads
// the completion flags of all staged chunks in one batch of relaxed loads and
// posts every chunk whose dependencies are all complete as ready.  Each
// consumer warp works on any ready chunk among the oldest kStages it has not
// done (oldest first), gathering rows d[u] with ld.global.cg, so one chunk
// waiting for another CTA does not hold up the chunks behind it.  A warp
// releases the buffer on the "empty" mbarrier; the last of the 31 to finish a
// chunk marks its position complete.  A narrow level further down uses a warp
// per vertex: its groups of TPV threads take every (32/TPV)-th arc, and chunks
// are 31 vertices so more CTAs share the level.
//
// Every wait (mbarrier, dependency flag, grid barrier) is bounded: past the
// limit the kernel records kStTimeout, stops issuing copies, waits (bounded)
// for the copies it already issued, and returns.
#include "iso_device.cuh"

namespace {

using namespace isod;

constexpr int kThreads = 1024;           // per CTA; 1024 / kThreads CTAs per SM
constexpr int kConsumers = kThreads - 32;  // all warps but the last consume; the last produces
constexpr int kStages = 3;               // chunks a CTA holds at once; warps take any ready one
constexpr int kArcCap = 3072;            // arcs per stage buffer (larger chunks read arcs from HBM)
constexpr int kOffCap = 1024;            // offsets per stage buffer (>= VPB + 5)
constexpr int kPredCap = 128;            // dependency list held per stage (longer lists stay in HBM)
constexpr int kRounds = 2;               // vertices per thread group in a chunk of a wide level

// Rounds per chunk for a group size: kRounds where the chunk's offsets fit the
// stage buffer, else one.
template <int TPV>
__host__ __device__ constexpr int rounds_of() { return kRounds * (kConsumers / TPV) + 5 <= kOffCap ? kRounds : 1; }

template <int K> struct MaskOf { using T = uint8_t; };
template <> struct MaskOf<16> { using T = uint16_t; };
template <> struct MaskOf<32> { using T = uint32_t; };
template <> struct MaskOf<64> { using T = unsigned long long; };

struct Meta {
    int v0, v1;   // vertices [v0, v1)
    int abase;    // first arc index held in the stage buffer
    int flags;    // bit 0: arcs did not fit (read them from global memory); bit 1: a warp per vertex;
                  // bit 2: out of range for every lane (restricted sweep): nothing staged
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
    int32_t preds[kStages][kPredCap];  // positions the staged chunk depends on
    int finished[kStages];  // consumer warps done with the chunk in each stage
    int ready_it[kStages];  // chunk (CTA-local index + 1) whose dependencies were seen complete
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
// Non-blocking probe of phase `parity` (try_wait may suspend the thread for a
// while; a polling loop that also watches other things must not).
__device__ __forceinline__ bool mbar_test_wait(unsigned long long* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
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

// The same through L1 (for rows nobody else writes meanwhile).
template <int LPT, int TPV>
__device__ __forceinline__ Row<LPT> load_row_l1(const uint32_t* row, int sub) {
    Row<LPT> r;
    if constexpr (LPT >= 4) {
#pragma unroll
        for (int q = 0; q < LPT / 4; ++q) {
            const uint4 v = __ldca(reinterpret_cast<const uint4*>(row) + sub + TPV * q);
            r.x[4 * q] = v.x; r.x[4 * q + 1] = v.y; r.x[4 * q + 2] = v.z; r.x[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < LPT; ++q) r.x[q] = __ldca(row + sub * LPT + q);
    }
    return r;
}

// Starts pulling `bytes` (a multiple of 4) from p into L1.
__device__ __forceinline__ void prefetch_l1(const uint32_t* p, int bytes) {
    for (int o = 0; o < bytes; o += 128)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(p + o / 4));
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

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Polling load of a completion flag.  Flags are read relaxed, so that all of a
// pass's loads are in flight at once; the reader fences (acquire) once after
// seeing every flag it needs set.
__device__ __forceinline__ uint32_t ld_relaxed(const int32_t* a) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a));
    return v;
}

// Row of a predicated gather: the label row, or all kInf when `ok` is false
// (no memory access then).
template <int LPT, int TPV>
__device__ __forceinline__ Row<LPT> load_row_if(const uint32_t* row, int sub, bool ok) {
    Row<LPT> r;
    if (ok) {
        r = load_row<LPT, TPV>(row, sub);
    } else {
#pragma unroll
        for (int i = 0; i < LPT; ++i) r.x[i] = kInf;
    }
    return r;
}

// Gathers rows d[u] + len(u,v) for arcs a, a+STEP, a+2*STEP, ... < e into acc,
// four rows in flight per round and every round four wide (the last one
// predicated), so a vertex with n arcs waits for ceil(n/4) round trips.
// A predicated-off row is kInf with length 0, which never lowers the minimum
// (kInf + len cannot wrap: kInf + 0x7FFFFFFE < 2^32).
// One round: rows of arcs q[0..3] (q[i] taken only if on[i]; q[0] always).
template <int K, int LPT, int TPV>
__device__ __forceinline__ void gather_round(Row<LPT>& acc, const uint32_t* d, const int2 (&q)[4], bool o1, bool o2,
                                             bool o3, int sub) {
    const Row<LPT> r0 = load_row<LPT, TPV>(d + (size_t)q[0].x * K, sub);
    const Row<LPT> r1 = load_row_if<LPT, TPV>(d + (size_t)q[1].x * K, sub, o1);
    const Row<LPT> r2 = load_row_if<LPT, TPV>(d + (size_t)q[2].x * K, sub, o2);
    const Row<LPT> r3 = load_row_if<LPT, TPV>(d + (size_t)q[3].x * K, sub, o3);
#pragma unroll
    for (int i = 0; i < LPT; ++i) {
        const uint32_t m01 = min(r0.x[i] + (uint32_t)q[0].y, r1.x[i] + (uint32_t)q[1].y);
        const uint32_t m23 = min(r2.x[i] + (uint32_t)q[2].y, r3.x[i] + (uint32_t)q[3].y);
        acc.x[i] = min(acc.x[i], min(m01, m23));
    }
}

// The arcs a, a+STEP, a+2*STEP, a+3*STEP (those below e; zero beyond).
template <int STEP>
__device__ __forceinline__ void arcs_of_round(int2 (&q)[4], const int2* arcs, uint32_t a, uint32_t e) {
#pragma unroll
    for (int r = 0; r < 4; ++r) q[r] = a + r * STEP < e ? arcs[a + r * STEP] : make_int2(0, 0);
}

template <int K, int LPT, int TPV, int STEP>
__device__ __forceinline__ void gather(Row<LPT>& acc, const uint32_t* d, const int2* arcs, uint32_t a, uint32_t e,
                                       int sub) {
    for (; a < e; a += 4 * STEP) {
        int2 q[4];
        arcs_of_round<STEP>(q, arcs, a, e);
        gather_round<K, LPT, TPV>(acc, d, q, a + STEP < e, a + 2 * STEP < e, a + 3 * STEP < e, sub);
    }
}

// A vertex's first round of arcs, read ahead (before a barrier) by the
// level-synchronous sweep of narrow levels.
struct FirstRound {
    bool on;      // q holds the arcs of the first round
    int2 q[4];
};

// True (on every lane) if every position in pred[pa .. pa+np) is complete right
// now (plus bar_extra flags that never come when a test asks for a timeout).
// Relaxed reads: the caller fences before relying on the result.
__device__ bool deps_done_now(const SweepParams& p, int pa, int np, int lane) {
    const int b_real = pa + np, b = b_real + p.bar_extra;
    for (int i = pa + lane;; i += 32) {
        const bool mine = i >= b || (i < b_real && ld_relaxed(p.done + p.pred[i]) != 0u);
        if (!__all_sync(0xffffffffu, mine)) return false;
        if (__all_sync(0xffffffffu, i + 32 >= b)) return true;
    }
}

// New label row of vertex v: min(upward labels, min over its downward arcs
// [a, e) of d[u] + len), pruned at tau; stored as a row (if `store`) and as an
// in-range mask.  WPV: the whole warp works on v, its 32/TPV groups of TPV
// threads taking every (32/TPV)-th arc; otherwise v belongs to one group.  With
// a warp per vertex (narrow levels, where the sweep waits on latency) the
// vertex's own state is read before the gathers instead of after them.
template <int K, int TPV, bool WPV>
__device__ __forceinline__ void vertex_update(const SweepParams& p, const Smem& sm, int v, bool valid, uint32_t a,
                                              uint32_t e, const int2* arcs, bool store, int tid,
                                              const FirstRound& pre = FirstRound{false, {}}) {
    constexpr int LPT = K / TPV;
    constexpr int GPV = 32 / TPV;
    using MaskT = typename MaskOf<K>::T;
    const int lane = tid & 31;
    const int sub = tid % TPV;
    const int g = WPV ? lane / TPV : 0;
    Row<LPT> acc;
#pragma unroll
    for (int i = 0; i < LPT; ++i) acc.x[i] = kInf;
    unsigned long long um = 0;
    bool hit = false;
    if (WPV) {
        // the row of v is written by nobody but this update during the sweep,
        // so an L1 copy of it cannot be stale
        if (valid && g == 0) {
            um = __ldcg(p.upmask + v);
            prefetch_l1(p.d + (size_t)v * K, K * 4);
        }
        if (valid) {
            uint32_t b = a + g;
            if (pre.on) {  // pre holds the arcs of this thread's group
                if (b < e) gather_round<K, LPT, TPV>(acc, p.d, pre.q, b + GPV < e, b + 2 * GPV < e, b + 3 * GPV < e, sub);
                b += 4 * GPV;
            }
            gather<K, LPT, TPV, GPV>(acc, p.d, arcs, b, e, sub);
        }
#pragma unroll
        for (int o = TPV; o < 32; o <<= 1) {
#pragma unroll
            for (int i = 0; i < LPT; ++i) acc.x[i] = min(acc.x[i], __shfl_xor_sync(0xffffffffu, acc.x[i], o));
        }
        hit = um != 0ull;
    } else if (valid) {
        hit = __ldcg(p.upflag + v) != 0;
        uint32_t b = a;
        if (pre.on) {
            if (b < e) gather_round<K, LPT, TPV>(acc, p.d, pre.q, b + 1 < e, b + 2 < e, b + 3 < e, sub);
            b += 4;
        }
        gather<K, LPT, TPV, 1>(acc, p.d, arcs, b, e, sub);
        if (hit) um = __ldcg(p.upmask + v);
    }
    if (hit) {
        // upward labels: only the lanes marked in upmask hold this batch's values
        const Row<LPT> own = WPV ? load_row_l1<LPT, TPV>(p.d + (size_t)v * K, sub)
                                 : load_row<LPT, TPV>(p.d + (size_t)v * K, sub);
#pragma unroll
        for (int i = 0; i < LPT; ++i)
            if ((um >> lane_of<LPT, TPV>(sub, i)) & 1ull) acc.x[i] = min(acc.x[i], own.x[i]);
    }
    __syncwarp();  // every thread of the vertex has read flag and mask before they are cleared
    if (hit && g == 0 && sub == 0) { p.upflag[v] = 0; p.upmask[v] = 0ull; }
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

// Levels lo_level .. hi_level-1, swept by this CTA alone (all 32 warps), a
// warp per vertex, with a CTA barrier after each level.
template <int K, int TPV>
__device__ void sweep_levels_cta(const SweepParams& p, const Smem& sm, int lo_level, int hi_level, int warp, int tid) {
    for (int j = lo_level; j < hi_level; ++j) {
        const int lo = __ldg(p.level_off + j), hi = __ldg(p.level_off + j + 1);
        const bool store = p.write_all || j != p.last_level_block;
        for (int v = lo + warp; v < hi; v += kThreads / 32)
            vertex_update<K, TPV, true>(p, sm, v, true, __ldg(p.down_off + v), __ldg(p.down_off + v + 1), p.down_arc,
                                        store, tid);
        __syncthreads();
        if (p.trace && tid == 0) atomicMax((unsigned long long*)p.trace + 1 + j, global_ns());
    }
}

// Level j, swept by all CTAs together: a warp per vertex if the level has no
// more vertices than the grid has warps, else a group of TPV threads per
// vertex, in as many passes over the grid's groups as the level needs.
// plan_level reads what does not depend on the labels -- the arc range and
// first round of arcs of the thread's first vertex -- so that it can run
// before the barrier that ends the previous level; finish_level gathers.
struct LevelPlan {
    int v, hi;
    bool valid, wpv;
    uint32_t a, e;
    FirstRound pre;
};

template <int TPV>
__device__ __forceinline__ LevelPlan plan_level(const SweepParams& p, int j, int warp, int tid) {
    constexpr int GPV = 32 / TPV;
    LevelPlan pl;
    const int lo = __ldg(p.level_off + j), hi = __ldg(p.level_off + j + 1);
    const int warps = (int)gridDim.x * (kThreads / 32);
    pl.wpv = hi - lo <= warps;
    pl.hi = hi;
    pl.v = pl.wpv ? lo + (int)blockIdx.x * (kThreads / 32) + warp : lo + (int)blockIdx.x * (kThreads / TPV) + tid / TPV;
    pl.valid = pl.v < hi;
    pl.a = pl.valid ? __ldg(p.down_off + pl.v) : 0u;
    pl.e = pl.valid ? __ldg(p.down_off + pl.v + 1) : 0u;
    pl.pre.on = true;
    if (pl.wpv) arcs_of_round<GPV>(pl.pre.q, p.down_arc, pl.a + (uint32_t)((tid & 31) / TPV), pl.e);
    else arcs_of_round<1>(pl.pre.q, p.down_arc, pl.a, pl.e);
    return pl;
}

template <int K, int TPV>
__device__ __forceinline__ void finish_level(const SweepParams& p, const Smem& sm, int j, const LevelPlan& pl, int tid) {
    const bool store = p.write_all || j != p.last_level_block;
    if (pl.wpv) {
        if (pl.valid)  // warp-uniform
            vertex_update<K, TPV, true>(p, sm, pl.v, true, pl.a, pl.e, p.down_arc, store, tid, pl.pre);
    } else {
        vertex_update<K, TPV, false>(p, sm, pl.v, pl.valid, pl.a, pl.e, p.down_arc, store, tid, pl.pre);
        // further passes (uniform bounds: every thread takes part in the shuffles)
        const int groups = (int)gridDim.x * (kThreads / TPV);
        for (int v = pl.v + groups; v - (tid / TPV) < pl.hi; v += groups) {
            const bool valid = v < pl.hi;
            vertex_update<K, TPV, false>(p, sm, v, valid, valid ? __ldg(p.down_off + v) : 0u,
                                         valid ? __ldg(p.down_off + v + 1) : 0u, p.down_arc, store, tid);
        }
    }
}

// Label rows and in-range masks of the core vertices from k_core's lane-major
// output (final, clamped labels): thread t of a warp takes vertex v0 + t,
// reading lane i's label from row i of the lane-major array (coalesced over
// the warp) and writing its own label row; bit i of the mask is set iff lane
// i's label is not kInf.
template <int K>
__device__ void core_rows(const SweepParams& p, int warp, int lane) {
    using MaskT = typename MaskOf<K>::T;
    const int cn = p.core_n;
    for (int v0 = ((int)blockIdx.x * (kThreads / 32) + warp) * 32; v0 < cn; v0 += (int)gridDim.x * kThreads) {
        const int v = v0 + lane;
        if (v >= cn) continue;
        const uint32_t* src = p.core_out + v;
        unsigned long long bits = 0;
        if constexpr (K >= 4) {
#pragma unroll 4
            for (int i = 0; i < K; i += 4) {
                uint4 x;
                x.x = __ldcg(src + (size_t)i * cn);
                x.y = __ldcg(src + (size_t)(i + 1) * cn);
                x.z = __ldcg(src + (size_t)(i + 2) * cn);
                x.w = __ldcg(src + (size_t)(i + 3) * cn);
                bits |= (unsigned long long)(x.x != kInf) << i | (unsigned long long)(x.y != kInf) << (i + 1) |
                        (unsigned long long)(x.z != kInf) << (i + 2) | (unsigned long long)(x.w != kInf) << (i + 3);
                reinterpret_cast<uint4*>(p.d + (size_t)v * K)[i / 4] = x;
            }
        } else {
            for (int i = 0; i < K; ++i) {
                const uint32_t x = __ldcg(src + (size_t)i * cn);
                bits |= (unsigned long long)(x != kInf) << i;
                p.d[(size_t)v * K + i] = x;
            }
        }
        static_cast<MaskT*>(p.mask)[v] = (MaskT)bits;
    }
}

// Fused emission (Section 5: isochrone edges found by a second look at the
// arcs of a vertex once its label is final).  Input arc e = (a, b) is checked
// at its later-swept endpoint v against the other one, h, which is final
// because a downward arc h -> v (a real or a dummy one) makes v's chunk wait
// for h: e is an isochrone edge for lane i iff bit i of mask[v] XOR mask[h]
// is set.  `nv` vertices per warp (a power of two <= 32), lane l taking
// vertex l / (32 / nv) and every (32 / nv)-th of its entries; per lane the
// ids are appended with one atomicAdd per warp, as in k_emit.  v's mask was
// written by this warp (ordered by __syncwarp) or before a grid barrier.
template <int K>
__device__ void emit_vertices(const SweepParams& p, int v_first, int v_stride, int nv, int v_end, int lane) {
    using MaskT = typename MaskOf<K>::T;
    constexpr unsigned long long kLanes = K >= 64 ? ~0ull : ((1ull << K) - 1ull);
    const MaskT* mask = static_cast<const MaskT*>(p.mask);
    const int lpv = 32 / nv;
    const int j = lane / lpv, o = lane % lpv;
    const int v = v_first + j * v_stride;
    const bool valid = v < v_end;
    const uint32_t e0 = valid ? __ldg(p.emit_off + v) : 0u, e1 = valid ? __ldg(p.emit_off + v + 1) : 0u;
    const unsigned long long mv = valid ? (unsigned long long)__ldcg(mask + v) : 0ull;
    const unsigned lt = (1u << lane) - 1u;
    // rounds over the entries, as many as the vertex with the most needs
    const int rounds = __reduce_max_sync(0xffffffffu, valid ? (int)((e1 - e0 + lpv - 1) / lpv) : 0);
    for (int r = 0; r < rounds; ++r) {
        const uint32_t e = e0 + o + (uint32_t)r * lpv;
        unsigned long long x = 0;
        int id = 0;
        if (e < e1) {
            const int2 en = __ldg(p.emit_ent + e);
            x = (mv ^ (unsigned long long)__ldcg(mask + en.x)) & kLanes;
            id = en.y;
        }
        unsigned long long todo = __reduce_or_sync(0xffffffffu, (unsigned)x) |
                                  ((unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)(x >> 32)) << 32);
        while (todo) {
            const int i = __ffsll((long long)todo) - 1;
            todo &= todo - 1;
            const unsigned b = __ballot_sync(0xffffffffu, (x >> i) & 1ull);
            const int leader = __ffs(b) - 1;
            int at = 0;
            if (lane == leader) at = atomicAdd(p.ecnt + i, __popc(b));
            at = __shfl_sync(0xffffffffu, at, leader);
            if ((x >> i) & 1ull) {
                const int q = at + __popc(b & lt);
                if (q < p.ecap) p.ebuf[(size_t)i * p.ecap + q] = id;
            }
        }
    }
}

// Grid-wide barrier of the whole CTA (the launch is cooperative, so every CTA
// is resident): an arrival counter that the last arriver resets before it
// advances a generation word the others poll.  (A barrier on one ever-growing
// counter, one release-add to arrive and acquire-polling to wait, passed the
// grid-synchronous levels about 70 us sooner on the 18M graph but left the
// chunk phase that follows it 0.6 ms slower, with relaxed polling as well;
// this one is kept.)  Bounded: gives up, recording kStTimeout, after the
// timeout (bar_extra adds arrivals that never come, for the tests).  Returns
// false, the same on every thread of the CTA, if the kernel has failed.
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
            fence_acq_rel_gpu();
            const uint32_t want = gridDim.x + (uint32_t)p.bar_extra;
            if (atomicAdd(p.bar, 1u) + 1u == want) {
                atomicExch(p.bar, 0u);
                fence_acq_rel_gpu();
                atomicAdd(p.bar + 1, 1u);
            } else {
                const unsigned long long t0 = global_ns();
                for (uint32_t it = 0; *gen == g0; ++it) {
                    if ((it & 15) == 15) {
                        if (*st != kStOk) { ok = 0; break; }
                        if (global_ns() - t0 > (unsigned long long)p.timeout_ns || it > (1u << 28)) {
                            atomicCAS(p.status, kStOk, kStTimeout);
                            ok = 0;
                            break;
                        }
                    }
                }
            }
            fence_acq_rel_gpu();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The chunk held in `stage`, by one consumer warp (its share of the vertices).
template <int K, int TPV>
__device__ __forceinline__ void process_chunk(const SweepParams& p, const Smem& sm, int stage, int warp, int tid) {
    const Meta mt = sm.meta[stage];
    const int mode = (mt.flags >> 1) & 1;
    const int ob = mt.v0 & ~3;
    const bool store = p.write_all || mt.level != p.last_level_block;
    const int2* arcs = (mt.flags & 1) ? p.down_arc : sm.arcs[stage] - mt.abase;
    if (mt.flags & 4) {
        // out of range for every lane: kInf rows, empty masks, no gathers, a
        // thread per vertex (the bounds exclude upward labels here; a flag is
        // cleared regardless)
        using MaskT = typename MaskOf<K>::T;
        for (int v = mt.v0 + tid; v < mt.v1; v += kConsumers) {
            if (store) {
                if constexpr (K >= 4) {
#pragma unroll
                    for (int i = 0; i < K / 4; ++i)
                        reinterpret_cast<uint4*>(p.d + (size_t)v * K)[i] = make_uint4(kInf, kInf, kInf, kInf);
                } else {
                    for (int i = 0; i < K; ++i) p.d[(size_t)v * K + i] = kInf;
                }
            }
            static_cast<MaskT*>(p.mask)[v] = (MaskT)0;
            if (__ldcg(p.upflag + v)) { p.upflag[v] = 0; p.upmask[v] = 0ull; }
        }
        return;
    }
    if (mode) {
        const int v = mt.v0 + warp;
        const bool valid = v < mt.v1;
        const uint32_t a = valid ? sm.offs[stage][v - ob] : 0u, e = valid ? sm.offs[stage][v + 1 - ob] : 0u;
        vertex_update<K, TPV, true>(p, sm, v, valid, a, e, arcs, store, tid);
        return;
    }
    // kRounds vertices per thread group, one after the other
#pragma unroll 1
    for (int r = 0; r < rounds_of<TPV>(); ++r) {
        const int v = mt.v0 + r * (kConsumers / TPV) + tid / TPV;
        const bool valid = v < mt.v1;
        const uint32_t a = valid ? sm.offs[stage][v - ob] : 0u, e = valid ? sm.offs[stage][v + 1 - ob] : 0u;
        vertex_update<K, TPV, false>(p, sm, v, valid, a, e, arcs, store, tid);
    }
}

// Bookkeeping of a polling loop that found nothing to do (lane 0 decides):
// true once the kernel has failed elsewhere or this warp has been idle for
// longer than the timeout (then the status records the timeout).  The clock is
// read only while idle.
__device__ __forceinline__ bool idle_too_long(const SweepParams& p, unsigned long long& idle_since, int lane) {
    if (lane != 0) return false;
    if (*(volatile int32_t*)p.status != kStOk) return true;
    const unsigned long long now = global_ns();
    if (idle_since == 0) {
        idle_since = now;
        return false;
    }
    if (now - idle_since > (unsigned long long)p.timeout_ns) {
        atomicCAS(p.status, kStOk, kStTimeout);
        return true;
    }
    return false;
}

// A consumer warp is done with the chunk in `stage` (schedule position q, level
// block `level`): the last of the consumer warps to get here publishes the
// position as complete to every CTA; each warp releases the buffer.
__device__ __forceinline__ void release_chunk(const SweepParams& p, Smem& sm, int stage, int q, int level, int lane) {
    __syncwarp();
    if (lane == 0) {
        __threadfence_block();
        if (atomicAdd(&sm.finished[stage], 1) == kConsumers / 32 - 1) {
            __threadfence_block();
            sm.finished[stage] = 0;
            fence_acq_rel_gpu();  // release: the CTA's rows before the flag
            *(volatile int32_t*)(p.done + q) = 1;
            if (p.trace) atomicMax((unsigned long long*)p.trace + 1 + level, global_ns());
        }
        mbar_arrive(&sm.empty[stage]);
    }
}

// FUSED: the instantiation with fused emission (a separate one, so that the
// plain kernel's code is not shaped by the emission paths).
template <int K, int TPV, bool FUSED>
__global__ void __launch_bounds__(kThreads, 1024 / kThreads) k_sweep_tma(SweepParams p) {
    constexpr int VPB = rounds_of<TPV>() * (kConsumers / TPV);
    static_assert(VPB + 5 <= kOffCap, "offset buffer");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    // chunks of this CTA: positions blockIdx.x, blockIdx.x + G, ...
    const int G = (int)gridDim.x;
    const int n_mine = (int)blockIdx.x < p.Q ? (p.Q - (int)blockIdx.x + G - 1) / G : 0;

    // (with a per-lane core, k_core has recorded the start of the sweep step)
    if (p.trace && tid == 0 && blockIdx.x == 0 && p.core_levels == 0)
        p.trace[0] = p.trace[p.L + 1] = (long long)global_ns();
    // The per-lane core (k_core, launched just before) has left the final
    // labels of its vertices lane-major; they become label rows and masks here,
    // complete for every CTA after a grid barrier.
    if (p.core_levels > 0) {
        core_rows<K>(p, warp, lane);
        if (!grid_sync(p)) return;  // the same in every thread of the CTA
    }
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&sm.full[i], 1);
            mbar_init(&sm.empty[i], kConsumers / 32);
            sm.finished[i] = 0;
            sm.ready_it[i] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < K) {
        const int32_t t = p.tau[tid];
        sm.tau[tid] = t < 0 ? 0u : (uint32_t)t;
    }
    __syncthreads();

    // ---------------- the leading levels, level by level ----------------
    // The top of the hierarchy is a long chain of small levels: CTA 0 sweeps
    // the smallest alone (a CTA barrier per level), then all CTAs sweep the
    // other narrow ones (a grid barrier per level).  The schedule holds no
    // chunks of these levels and no dependencies on them.
    if (p.sync_levels > p.core_levels) {
        bool ok = true;
        // plans read graph data only, so each is made before the barrier that
        // ends the level in front of it
        const bool grid_levels = p.solo_levels < p.sync_levels;
        LevelPlan pl{};
        if (grid_levels) pl = plan_level<TPV>(p, p.solo_levels, warp, tid);
        if (p.solo_levels > p.core_levels) {
            if (blockIdx.x == 0) sweep_levels_cta<K, TPV>(p, sm, p.core_levels, p.solo_levels, warp, tid);
            ok = grid_sync(p);
        }
        for (int j = p.solo_levels; ok && j < p.sync_levels; ++j) {
            finish_level<K, TPV>(p, sm, j, pl, tid);
            if (j + 1 < p.sync_levels) pl = plan_level<TPV>(p, j + 1, warp, tid);
            ok = grid_sync(p);
            if (ok && p.trace && tid == 0 && blockIdx.x == 0)
                atomicMax((unsigned long long*)p.trace + 1 + j, global_ns());
        }
        if (!ok) return;  // the same in every thread of the CTA
    }
    // fused emission of the vertices swept so far (complete after the last
    // grid barrier), a warp per 32 of them
    if constexpr (FUSED)
        for (int v0 = ((int)blockIdx.x * (kThreads / 32) + warp) * 32; v0 < p.sync_n; v0 += (int)gridDim.x * kThreads)
            emit_vertices<K>(p, v0, 1, 32, p.sync_n, lane);

    if (warp == kConsumers / 32) {
        // ---------------- producer warp ----------------
        // Lane s < kStages runs stage s, whose chunks are s, s + kStages, ...:
        // once the stage is free it copies the next one's offsets, arcs and
        // dependency list in, and once those have landed and every position
        // the chunk depends on is complete it posts the chunk as ready.  No
        // lane ever blocks, so the stages' latencies overlap.
        int t = lane;             // next chunk of my stage
        int cur = -1;             // chunk in my stage not posted yet, or -1
        int cur_pa = 0, cur_np = 0;
        bool cur_held = false;    // its dependency list was copied to shared memory
        // staging limits (the buffer sizes, or lower ones a test asks for)
        const int arc_cap = p.stage_arc_cap > 0 && p.stage_arc_cap < kArcCap ? p.stage_arc_cap : kArcCap;
        const int pred_cap = p.stage_pred_cap > 0 && p.stage_pred_cap < kPredCap ? p.stage_pred_cap : kPredCap;
        int posted = 0;
        // schedule record of chunk t, loaded one chunk ahead so that issuing
        // never waits for it
        int4 n0 = make_int4(0, 0, 0, 0), n1 = n0;
        if (lane < kStages && t < n_mine) {
            n0 = __ldg(p.sched_info + 2 * ((size_t)blockIdx.x + (size_t)t * G));
            n1 = __ldg(p.sched_info + 2 * ((size_t)blockIdx.x + (size_t)t * G) + 1);
        }
        unsigned long long idle_since = 0;
        uint32_t nap = 32;
        while (posted < n_mine) {
            // (1) copy the next chunk into every free stage
            const bool issue = lane < kStages && cur < 0 && t < n_mine &&
                               (t < kStages || mbar_test_wait(&sm.empty[lane], ((uint32_t)(t / kStages) & 1u) ^ 1u));
            if (issue) {
                const int pos = (int)blockIdx.x + t * G;
                const int4 c0 = n0;  // v0, v1, level, mode
                const int4 c1 = n1;  // arc base, arcs, deps start, deps
                const int ob = c0.x & ~3;
                // a skipped chunk needs neither its graph data nor its dependencies
                const bool skip = p.skip && __ldg(p.skip + pos);
                const uint32_t obytes = skip ? 0u : (uint32_t)(((c0.y + 1 - ob) * 4 + 15) & ~15);
                const int big = c1.y > arc_cap;
                const uint32_t abytes = big || skip ? 0u : (uint32_t)((c1.y * 8 + 15) & ~15);
                cur_held = skip || (c1.w <= pred_cap && p.bar_extra == 0);
                const uint32_t pbytes = cur_held && !skip ? (uint32_t)(((c1.w + 3) & ~3) * 4) : 0u;
                sm.meta[lane] = Meta{c0.x, c0.y, c1.x, big | (c0.w ? 2 : 0) | (skip ? 4 : 0), pos, c0.z, {0, 0}};
                mbar_expect_tx(&sm.full[lane], obytes + abytes + pbytes);
                if (obytes) bulk_load(sm.offs[lane], p.down_off + ob, obytes, &sm.full[lane]);
                if (abytes) bulk_load(sm.arcs[lane], p.down_arc + c1.x, abytes, &sm.full[lane]);
                if (pbytes) bulk_load(sm.preds[lane], p.pred + c1.z, pbytes, &sm.full[lane]);
                cur = t;
                cur_pa = c1.z;
                cur_np = skip ? 0 : c1.w;
                t += kStages;
                if (t < n_mine) {
                    n0 = __ldg(p.sched_info + 2 * ((size_t)blockIdx.x + (size_t)t * G));
                    n1 = __ldg(p.sched_info + 2 * ((size_t)blockIdx.x + (size_t)t * G) + 1);
                }
            }
            bool progress = __any_sync(0xffffffffu, issue);
            // (2) post the staged chunks whose copies have landed and whose
            // dependencies are complete: one pass reads the flags of all of
            // them, every load in flight at once
            const bool landed =
                lane < kStages && cur >= 0 && mbar_test_wait(&sm.full[lane], (uint32_t)(cur / kStages) & 1u);
            const uint32_t cand = __ballot_sync(0xffffffffu, landed);
            if (cand) {
                uint32_t notdone = 0;
#pragma unroll
                for (int st = 0; st < kStages; ++st) {
                    if (!((cand >> st) & 1u)) continue;
                    const int cst = __shfl_sync(0xffffffffu, cur, st);
                    const int np = __shfl_sync(0xffffffffu, cur_np, st);
                    const int pa = __shfl_sync(0xffffffffu, cur_pa, st);
                    if (!__shfl_sync(0xffffffffu, (int)cur_held, st)) {
                        if (!deps_done_now(p, pa, np, lane)) notdone |= 1u << st;
                        continue;
                    }
                    // this lane's view of the landed copy (the phase cannot move on yet)
                    (void)mbar_test_wait(&sm.full[st], (uint32_t)(cst / kStages) & 1u);
#pragma unroll
                    for (int r = 0; r < kPredCap / 32; ++r) {
                        const int i = lane + 32 * r;
                        if (i < np && ld_relaxed(p.done + sm.preds[st][i]) == 0u) notdone |= 1u << st;
                    }
                }
                notdone = __reduce_or_sync(0xffffffffu, notdone);
                const uint32_t now_ready = cand & ~notdone;
                if (now_ready) {
                    fence_acq_rel_gpu();  // acquire: the flags seen set order the label rows behind them
                    if ((now_ready >> lane) & 1u) {
                        *(volatile int*)&sm.ready_it[lane] = cur + 1;
                        cur = -1;
                    }
                    posted += __popc(now_ready);
                    progress = true;
                }
            }
            if (progress) {
                nap = 32;
                idle_since = 0;
                continue;
            }
            __nanosleep(nap);
            if (nap < 256) nap <<= 1;
            if (__shfl_sync(0xffffffffu, (int)idle_too_long(p, idle_since, lane), 0)) break;
        }
        // every issued copy must land before the CTA exits
        if (lane < kStages && t >= kStages) {
            const int last = t - kStages;
            mbar_wait(&sm.full[lane], (uint32_t)(last / kStages) & 1u, p);
        }
        __syncthreads();
        return;
    }

    // ---------------- consumer warps ----------------
    // Each warp takes, among the oldest kStages chunks it has not done yet, any
    // one that is copied and ready (oldest first), does its part of it, and
    // releases the buffer; the last warp to finish a chunk publishes it.
    int base = 0;            // oldest chunk this warp has not done
    uint32_t done_bits = 0;  // bit d: chunk base + d done by this warp
    unsigned long long idle_since = 0;
    uint32_t nap = 32;
    while (base < n_mine) {
        // lane d looks at chunk base + d of the window
        bool cand = false;
        if (lane < kStages && base + lane < n_mine && !((done_bits >> lane) & 1u)) {
            const int t = base + lane;
            const int stage = t % kStages;
            cand = *(volatile int*)&sm.ready_it[stage] == t + 1 &&
                   mbar_test_wait(&sm.full[stage], (uint32_t)(t / kStages) & 1u);
        }
        const uint32_t ready = __ballot_sync(0xffffffffu, cand);
        if (!ready) {
            __nanosleep(nap);
            if (nap < 256) nap <<= 1;
            if (__shfl_sync(0xffffffffu, (int)idle_too_long(p, idle_since, lane), 0)) break;
            continue;
        }
        nap = 32;
        idle_since = 0;
        const int pick = __ffs(ready) - 1;
        const int t = base + pick;
        const int stage = t % kStages;
        // every lane acquires the copied data (the phase is complete and cannot
        // move on before this warp releases the buffer) and the ready flag
        mbar_wait(&sm.full[stage], (uint32_t)(t / kStages) & 1u, p);
        __threadfence_block();
        if constexpr (!FUSED) {
            process_chunk<K, TPV>(p, sm, stage, warp, tid);
            release_chunk(p, sm, stage, sm.meta[stage].q, sm.meta[stage].level, lane);
        } else {
        const Meta mt = sm.meta[stage];  // the buffer may be refilled once released
        process_chunk<K, TPV>(p, sm, stage, warp, tid);
        release_chunk(p, sm, stage, mt.q, mt.level, lane);
        // fused emission of this warp's vertices of the chunk, after the chunk
        // is published, so that no dependent waits for it
        {
            if (mt.flags & 4) {  // skipped: a thread per vertex
                for (int v = mt.v0 + warp * 32; v < mt.v1; v += kConsumers) emit_vertices<K>(p, v, 1, 32, mt.v1, lane);
            } else if (mt.flags & 2) {  // a warp per vertex
                emit_vertices<K>(p, mt.v0 + warp, 1, 1, mt.v1, lane);
            } else {
#pragma unroll 1
                for (int r = 0; r < rounds_of<TPV>(); ++r)
                    emit_vertices<K>(p, mt.v0 + r * (kConsumers / TPV) + warp * (32 / TPV), 1, 32 / TPV, mt.v1, lane);
            }
        }
        }
        done_bits |= 1u << pick;
        while (done_bits & 1u) { done_bits >>= 1; ++base; }
    }
    __syncthreads();
}

// Dynamic shared memory of a CTA.  Kept to the chunk phase's buffers: the
// shared memory a CTA takes comes out of the SM's L1, which also holds the
// gathers in flight (a larger carve-out measurably slowed the chunk phase).
constexpr size_t kSmemBytes = sizeof(Smem);

template <int K, int TPV, bool FUSED>
cudaError_t launch(const SweepParams& p, int grid, cudaStream_t s) {
    static std::atomic<unsigned long long> attr{0};
    if (cudaError_t e = iso_smem_attr_once(k_sweep_tma<K, TPV, FUSED>, (int)kSmemBytes, attr)) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_sweep_tma<K, TPV, FUSED>, p);
}

template <int K, int TPV>
int occupancy() {
    static std::atomic<unsigned long long> attr{0};
    if (iso_smem_attr_once(k_sweep_tma<K, TPV, false>, (int)kSmemBytes, attr) != cudaSuccess) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_sweep_tma<K, TPV, false>, kThreads, kSmemBytes) !=
        cudaSuccess)
        return 0;
    return blocks;
}

#define ISO_TMA_CASES(X) X(1, 1) X(4, 1) X(8, 1) X(16, 2) X(16, 4) X(32, 4) X(32, 8) X(64, 8) X(64, 16)

}  // namespace

void iso_sweep_tma_stage_caps(int* arcs, int* deps) {
    *arcs = kArcCap;
    *deps = kPredCap;
}

bool iso_sweep_tma_supported(int K, int tpv) {
#define X(k, t) if (K == k && tpv == t) return true;
    ISO_TMA_CASES(X)
#undef X
    return false;
}

cudaError_t iso_launch_sweep_tma(const isod::SweepParams& p, int K, int tpv, int grid, cudaStream_t s) {
#define X(k, t) \
    if (K == k && tpv == t) return p.fused_emit ? launch<k, t, true>(p, grid, s) : launch<k, t, false>(p, grid, s);
    ISO_TMA_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

int iso_sweep_tma_occupancy(int K, int tpv, int* block, int* vpb) {
    *block = kThreads;
#define X(k, t) if (K == k && tpv == t) { *vpb = rounds_of<t>() * (kConsumers / t); return occupancy<k, t>(); }
    ISO_TMA_CASES(X)
#undef X
    return 0;
}
