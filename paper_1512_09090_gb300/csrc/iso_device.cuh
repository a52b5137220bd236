// Device-side types shared by the isochrone kernels and their launchers.
//
// Layouts (all in HBM, sweep order = descending CH level):
//   d[v*K + i]      uint32 label of vertex v for lane i (query i of the batch);
//                   0x7FFFFFFF = out of range.  K lanes per row, K in {1,4,...,64}.
//   mask[v]         K-bit word, bit i set iff v is in range for lane i.
//   upflag[v]       1 while d[v*K..] holds upward-search labels not yet consumed
//                   by the sweep (the sweep clears it).
//   upmask[v]       lanes whose slot of d[v*K..] holds an upward label (TMA sweep).
//   down arcs       int2 {src, len} grouped by head, heads in sweep order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace isod {

constexpr uint32_t kInf = 0x7FFFFFFFu;

// Per-lane core of the TMA-staged sweep: at most this many vertices (one
// lane's labels in a CTA's shared memory; heads and sources fit 16 bits) in at
// most this many level blocks.
constexpr int kCoreMaxVertices = 53248;
constexpr int kCoreMaxLevels = 1023;

// Device status word values (status[0]); the host maps them to ISO_E_*.
enum : int {
    kStOk = 0,
    kStTimeout = 1,      // a grid barrier gave up
    kStBadInput = 2,     // a source or limit failed validation on the device
    kStUpOverflow = 3,   // upward search space exceeded the global table
};

// Sweep schedule step: x = kind (0 wide level, 1 run of narrow levels done by
// CTA 0), y = first level block, z = one past the last level block.
enum : int { kStepWide = 0, kStepFused = 1 };

struct UpParams {
    const uint32_t* up_off;   // [n+1]
    const int2* up_arc;       // {dst, len}, dst a sweep position
    const int32_t* pos;       // original id -> sweep position
    const int32_t* src;       // [K] original ids, -1 = idle lane
    const int32_t* tau;       // [K]
    int2* pairs;              // [K * cap] {vertex, label} per lane
    int32_t* cnt;             // [K]
    uint32_t* gtab;           // [K * iso_upward_table_words(gcap)] global fallback tables
    int32_t* status;
    int n;
    int cap;                  // entries per lane in pairs (== gcap)
    int gcap;                 // power of two
    int tau_max;
    // direct != 0: instead of pairs, write every label into its row slot d[v*K + lane],
    // set bit lane of upmask[v] and upflag[v] (the TMA sweep reads them there);
    // labels of vertices below core_n still go to pairs (cnt[lane] of them)
    int direct;
    int core_n;
    int K;
    uint32_t* d;
    unsigned long long* upmask;
    uint8_t* upflag;
};

struct SweepParams {
    const uint32_t* down_off;  // [n+1]
    const int2* down_arc;      // {src, len}
    const int32_t* level_off;  // [L+1]
    const int4* sched;         // [nsched]
    const int2* pairs;         // upward labels, [K * cap]
    const int32_t* cnt;        // [K]
    const int32_t* tau;        // [K]
    uint32_t* d;               // [n*K]
    void* mask;                // [n] K-bit words
    uint8_t* upflag;           // [n]
    uint32_t* bar;             // [2] arrival count, generation
    int32_t* status;
    long long timeout_ns;
    int n, L, nsched, cap;
    int last_level_block;      // index j of the lowest level (its d rows need no store)
    int write_all;             // store every d row (distances requested)
    int bar_extra;             // testing: extra arrivals a barrier waits for
    long long* trace;          // nullable: global ns; layout depends on the kernel (see iso_api.cu)
    // TMA kernel: chunk schedule (see schedule.cpp) and its progress
    const int4* sched_info;    // [2Q] per schedule position {v0, v1, level block, mode},
                               //      {first staged arc, arcs, dependency list start, its length}
    const int32_t* pred;       // dependency lists (positions), each 16-byte aligned
    int32_t* done;             // [Q] 1 once a position is complete; zeroed per batch
    int solo_levels;           // TMA kernel: levels 0 .. solo_levels-1 are swept by CTA 0 alone,
    int sync_levels;           // then levels .. sync_levels-1 by all CTAs, a grid barrier per level
    int Q;
    unsigned long long* upmask;// [n] lanes with an upward label (TMA kernel)
    // TMA kernel, per-lane core: levels 0 .. core_levels-1 (vertices [0, core_n))
    // are swept by CTA i for lane i alone, labels in shared memory, starting
    // from the lane's upward labels in pairs[i*cap .. + cnt[i]]
    int core_levels, core_n;
    const uint2* core_arc;     // downward arcs into [0, core_n): {src | head << 16, len}
    const uint32_t* level_arc; // [L+1] first downward arc of each level block
    uint32_t* core_out;        // [K * core_n] final core labels, lane-major (k_core -> sweep)
    // testing: stage at most this many arcs / dependency-list entries per chunk
    // (0 = the buffer sizes); larger chunks take the global-memory paths
    int stage_arc_cap, stage_pred_cap;
    // restricted sweep: skip[q] != 0 = chunk at position q is out of range for
    // every lane (k_skip); its rows are written kInf without gathers (nullable)
    const uint8_t* skip;
    // fused emission (fused_emit != 0): the input arcs at their later-swept
    // endpoint v, emit_ent[emit_off[v] .. emit_off[v+1]) = {other endpoint, arc
    // id}, are emitted by the sweep itself into ebuf / ecnt (as k_emit would)
    int fused_emit;
    const uint32_t* emit_off;
    const int2* emit_ent;
    int32_t* ecnt;             // [K]
    int32_t* ebuf;             // [K * ecap]
    int ecap;
    int sync_n;                // vertices swept before the chunk schedule (core + leading levels)
};

// Restricted sweep: which chunks are out of range for every lane of a batch,
// from landmark lower bounds (landmarks.h).
struct SkipParams {
    const int32_t* src;        // [K] original ids (-1 = idle lane)
    const int32_t* tau;        // [K]
    const int32_t* pos;        // [n] original id -> sweep position
    const uint32_t* lm_fwd;    // [count * n] d(L_i, v)
    const uint32_t* lm_bwd;    // [count * n] d(v, L_i)
    const uint32_t* chunk_lo;  // [Q * count] min over the chunk of d(L_i, v)
    const uint32_t* chunk_hi;  // [Q * count] max over the chunk of d(v, L_i)
    uint8_t* skip;             // [Q]
    int32_t* skipped;          // chunks skipped (counter)
    int n, K, Q, count;
};

struct EmitParams {
    const uint32_t* orig_off;  // [n+1] input arcs grouped by tail, by emission index
    const int32_t* orig_head;  // sweep positions
    const int32_t* orig_id;
    const int32_t* tail_of;    // [n] sweep position of the tail at each emission index
    const int32_t* status;     // batch status: emission is skipped once it is not kStOk
    const void* mask;
    int32_t* ecnt;             // [K]
    int32_t* ebuf;             // [K * ecap]
    int n, ecap;
};

struct GatherParams {
    int32_t* ebuf;             // sorted per-lane segments [K * ecap]
    const int32_t* ecnt;       // [K]
    int32_t* tmp;              // [K * ecap] scratch for large sorts
    int32_t* out;              // contiguous lists
    int64_t* out_off;          // [K+1]
    int k, ecap;
    int key_bits;              // bits needed for arc ids
    int64_t m;                 // arc ids are in [0, m)
    const int32_t* status;     // batch status: nothing is written once it is not kStOk
};

struct RangeParams {
    const int32_t* pos;        // [n] original id -> sweep position
    const void* mask;          // [n] K-bit in-range words (sweep order)
    uint32_t* out;             // [k * words] bitsets over original ids, query-major
    int64_t words;             // 32-bit words per query (>= ceil(n / 32))
    int n, k;
};

struct DistParams {
    const uint32_t* d;
    const int32_t* perm;
    int32_t* out;              // [k * n], query-major, original vertex order
    int n, k, K;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace isod

// Raises kernel f's dynamic shared-memory limit to `bytes` on the current
// device.  Function attributes belong to a device's context, so this is done
// once per device: bit d of `done` records device d (devices beyond 63 set it
// on every call).  Concurrent first calls may both set it, which is harmless.
template <class F>
cudaError_t iso_smem_attr_once(F* f, int bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// The highest scheduling priority of the current device (lower numbers are
// higher), for launches that should be placed ahead of other streams' pending
// work: a batch's upward search and core run while the previous batch's
// emission and sort still occupy the GPU, and are placed first.
inline int iso_high_priority() {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return greatest;
}

// Launchers (one translation unit each); return the launch's cudaError_t.
cudaError_t iso_launch_upward(const isod::UpParams& p, int K, cudaStream_t s);
size_t iso_upward_table_words(size_t gcap);  // 32-bit words of one lane's global table
cudaError_t iso_launch_sweep(const isod::SweepParams& p, int K, int tpv, int grid, cudaStream_t s);
int iso_sweep_occupancy(int K, int tpv, int* block);
bool iso_sweep_supported(int K, int tpv);
cudaError_t iso_launch_sweep_tma(const isod::SweepParams& p, int K, int tpv, int grid, cudaStream_t s);
// Per-lane core (k_core.cu): K CTAs; runs before iso_launch_sweep_tma when p.core_levels > 0.
cudaError_t iso_launch_core(const isod::SweepParams& p, int K, cudaStream_t s);
int iso_sweep_tma_occupancy(int K, int tpv, int* block, int* vpb);
bool iso_sweep_tma_supported(int K, int tpv);
void iso_sweep_tma_stage_caps(int* arcs, int* deps);  // stage buffer sizes (arcs, dependency entries)
cudaError_t iso_launch_emit(const isod::EmitParams& p, int K, int grid, cudaStream_t s);
cudaError_t iso_launch_sort_gather(const isod::GatherParams& p, int K, cudaStream_t s);
cudaError_t iso_launch_dist(const isod::DistParams& p, cudaStream_t s);
cudaError_t iso_launch_range(const isod::RangeParams& p, int K, cudaStream_t s);
cudaError_t iso_launch_skip(const isod::SkipParams& p, int grid, cudaStream_t s);
