// Isochrone edge emission (Section 3): arc (u,v) of the input graph is an
// isochrone edge for lane i iff exactly one of u, v is in range, i.e. iff bit i
// of mask[u] XOR mask[v] is set.  Arcs are visited grouped by tail, tails in
// BFS order of the input graph: neighbouring warps then read the masks of
// neighbouring vertices, which sit in a few short stretches of each level's
// part of the mask array and stay in L2, instead of scattered sectors.  Per lane, ids are appended with one
// atomicAdd per warp: __ballot_sync gives the warp's members for that lane and
// __popc of the lower lanes gives each member's slot.
//
// Then k_sort_gather sorts each lane's ids ascending (bucket sort in shared
// memory, four CTAs per lane) and writes them to the contiguous output at the
// lane's offset; CTA 0 also writes the offsets.
#include "iso_device.cuh"

namespace {

using namespace isod;

template <int K> struct MaskOf { using T = uint8_t; };
template <> struct MaskOf<16> { using T = uint16_t; };
template <> struct MaskOf<32> { using T = uint32_t; };
template <> struct MaskOf<64> { using T = unsigned long long; };

constexpr int kEmitThreads = 256;
constexpr int kEmitBatch = 4;     // rounds of 32 arcs whose loads a warp has in flight together
constexpr int kSortThreads = 1024;
constexpr int kSortSmem = 16384;  // ids bucketed in shared memory (64 KB): two sorting CTAs fit an SM

__device__ __forceinline__ unsigned long long warp_or(unsigned long long x) {
    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)x);
    const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(x >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

template <int K>
__global__ void __launch_bounds__(kEmitThreads) k_emit(EmitParams p) {
    using MaskT = typename MaskOf<K>::T;
    // bits of lanes that exist: a mask word holds at least 8 bits, and after a
    // failed sweep it may hold anything
    constexpr unsigned long long kLanes = K >= 64 ? ~0ull : ((1ull << K) - 1ull);
    // a failed batch (bad input, upward overflow, timeout) is reported by the
    // host; its masks may be stale, so nothing is emitted
    if (*(volatile const int32_t*)p.status != kStOk) return;
    const MaskT* mask = static_cast<const MaskT*>(p.mask);
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int warps = (int)(gridDim.x * blockDim.x) >> 5;
    // a warp takes 32 consecutive tails (emission indices); their arcs are one
    // contiguous range
    for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w * 32 < p.n; w += warps) {
        const int u0 = w * 32;
        const int u = min(u0 + (int)lane, p.n);
        const uint32_t my_off = __ldg(p.orig_off + u);           // start of tail u0+lane's arcs
        const uint32_t a0 = __shfl_sync(0xffffffffu, my_off, 0);
        const uint32_t a1 = __ldg(p.orig_off + min(u0 + 32, p.n));
        const unsigned long long mu_lane = u < p.n ? (unsigned long long)mask[__ldg(p.tail_of + u)] : 0ull;
        // kEmitBatch rounds of 32 arcs at a time: all their heads, then all the
        // heads' masks are in flight together (two dependent round trips for up
        // to 32 * kEmitBatch arcs instead of two per 32)
        for (uint32_t base0 = a0; base0 < a1; base0 += 32 * kEmitBatch) {
            unsigned long long mh[kEmitBatch];
            {
                int32_t hd[kEmitBatch];
#pragma unroll
                for (int r = 0; r < kEmitBatch; ++r) {
                    const uint32_t a = base0 + 32 * r + lane;
                    hd[r] = a < a1 ? __ldg(p.orig_head + a) : -1;
                }
#pragma unroll
                for (int r = 0; r < kEmitBatch; ++r) mh[r] = hd[r] >= 0 ? (unsigned long long)mask[hd[r]] : 0ull;
            }
#pragma unroll
            for (int r = 0; r < kEmitBatch; ++r) {
            const uint32_t base = base0 + 32 * r;
            if (base >= a1) break;  // warp-uniform
            const uint32_t a = base + lane;
            unsigned long long x = 0;
            int id = 0;
            // tail of arc a: the last lane t whose first arc is <= a
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t o = __shfl_sync(0xffffffffu, my_off, lo + step);
                if (lo + step < 32 && o <= a) lo += step;
            }
            const unsigned long long mu = __shfl_sync(0xffffffffu, mu_lane, lo);
            if (a < a1) {
                x = (mu ^ mh[r]) & kLanes;
                if (x) id = __ldg(p.orig_id + a);
            }
            if (!__any_sync(0xffffffffu, x != 0)) continue;
            unsigned long long todo = warp_or(x);
            while (todo) {
                const int i = __ffsll((long long)todo) - 1;
                todo &= todo - 1;
                const unsigned b = __ballot_sync(0xffffffffu, (x >> i) & 1ull);
                const int leader = __ffs(b) - 1;
                int at = 0;
                if ((int)lane == leader) at = atomicAdd(p.ecnt + i, __popc(b));
                at = __shfl_sync(0xffffffffu, at, leader);
                if ((x >> i) & 1ull) {
                    const int q = at + __popc(b & lt);
                    if (q < p.ecap) p.ebuf[(size_t)i * p.ecap + q] = id;
                }
            }
            }
        }
    }
}

// kParts CTAs per lane.  Ids are distinct and in [0, m); CTA (lane, part)
// takes the ids of the part-th of kParts equal slices of [0, m) (their count
// and the counts of the slices before it come from one pass over the lane's
// list), so the parts' sorted lists are consecutive pieces of the lane's
// sorted list.  A part is split into about cnt/4 equal buckets of its slice
// (histogram, scan, scatter into shared memory); buckets are then sorted on
// their own: small ones by one thread each (insertion sort), any bucket above
// kSmallBucket ids by the whole CTA (every id's rank by counting the smaller
// ones in its bucket, written straight to its place).  CTA 0 also writes the
// offsets of all lanes.  A lane one of whose parts would not fit shared memory
// is sorted by its part-0 CTA alone with the list in global memory (the other
// parts of that lane return).
constexpr int kMaxBuckets = 4096;
constexpr int kSmallBucket = 64;
constexpr int kMaxBigBuckets = 256;  // big buckets listed for the whole-CTA ranking
constexpr int kParts = 4;

// Sorts the ids x of src[0..src_cnt) with lo <= x < hi (cnt of them) into
// out[0..cnt): bucketed into B[0..cnt) by equal slices of [lo, hi) (about four
// ids per bucket), small buckets sorted in place and copied, big buckets
// ranked straight into out.
__device__ void bucket_sort(const int32_t* src, int src_cnt, int32_t* B, int cnt, int32_t* out, int64_t lo,
                            int64_t hi, int32_t* s_hist, int32_t* s_cur) {
    __shared__ int s_part[kSortThreads];
    __shared__ int s_nbig, s_big[kMaxBigBuckets];
    int lg = 0;
    while ((1 << lg) < kMaxBuckets && (4 << lg) < cnt) ++lg;
    const int nb = 1 << lg;
    const uint64_t span = (uint64_t)(hi - lo);
    auto bucket_of = [&](int32_t x) { return (int)((uint64_t)(x - lo) * (uint64_t)nb / span); };
    auto mine = [&](int32_t x) { return x >= lo && x < hi; };
    for (int bb = threadIdx.x; bb <= nb; bb += blockDim.x) s_hist[bb] = 0;
    if (threadIdx.x == 0) s_nbig = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < src_cnt; i += blockDim.x) {
        const int32_t x = src[i];
        if (mine(x)) atomicAdd(&s_hist[bucket_of(x)], 1);
    }
    __syncthreads();
    // exclusive scan of the nb counts (nb <= kMaxBuckets, a few per thread)
    {
        const int per = (nb + blockDim.x - 1) / blockDim.x;
        const int b0 = threadIdx.x * per;
        int sum = 0;
        for (int bb = b0; bb < min(b0 + per, nb); ++bb) sum += s_hist[bb];
        s_part[threadIdx.x] = sum;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const int v = threadIdx.x >= (unsigned)o ? s_part[threadIdx.x - o] : 0;
            __syncthreads();
            s_part[threadIdx.x] += v;
            __syncthreads();
        }
        int acc = s_part[threadIdx.x] - sum;
        for (int bb = b0; bb < min(b0 + per, nb); ++bb) {
            const int c = s_hist[bb];
            s_hist[bb] = acc;
            s_cur[bb] = acc;
            acc += c;
        }
        if (threadIdx.x == 0) s_hist[nb] = cnt;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < src_cnt; i += blockDim.x) {
        const int32_t x = src[i];
        if (mine(x)) B[atomicAdd(&s_cur[bucket_of(x)], 1)] = x;
    }
    __syncthreads();
    for (int bb = threadIdx.x; bb < nb; bb += blockDim.x) {
        const int blo = s_hist[bb], bhi = s_hist[bb + 1];
        if (bhi - blo > kSmallBucket) {
            const int q = atomicAdd(&s_nbig, 1);
            if (q < kMaxBigBuckets) s_big[q] = bb;
            continue;
        }
        for (int i = blo + 1; i < bhi; ++i) {
            const int32_t x = B[i];
            int j = i - 1;
            while (j >= blo && B[j] > x) { B[j + 1] = B[j]; --j; }
            B[j + 1] = x;
        }
        for (int i = blo; i < bhi; ++i) out[i] = B[i];
    }
    __syncthreads();
    // big buckets: the whole CTA, each id's place is the count of smaller ids
    // (the list of them, or every bucket if it overflowed)
    const int nbig = s_nbig;
    for (int t = 0; t < (nbig <= kMaxBigBuckets ? nbig : nb); ++t) {
        const int bb = nbig <= kMaxBigBuckets ? s_big[t] : t;
        const int blo = s_hist[bb], bhi = s_hist[bb + 1];
        if (bhi - blo <= kSmallBucket) continue;
        for (int i = blo + threadIdx.x; i < bhi; i += blockDim.x) {
            const int32_t x = B[i];
            int r = 0;
            for (int j = blo; j < bhi; ++j) r += B[j] < x;
            out[blo + r] = x;
        }
    }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_gather(GatherParams p) {
    extern __shared__ int32_t sbuf[];
    int32_t* s_hist = sbuf + kSortSmem;           // [kMaxBuckets + 1]
    int32_t* s_cur = s_hist + kMaxBuckets + 1;    // [kMaxBuckets]
    __shared__ long long s_off;
    __shared__ int s_pc[kParts];
    const int lane = blockIdx.x / kParts, part = blockIdx.x % kParts;
    if (*(volatile const int32_t*)p.status != kStOk) return;  // failed batch: the host reports it
    if (threadIdx.x == 0) {
        long long off = 0;
        for (int i = 0; i < lane; ++i) off += min(p.ecnt[i], p.ecap);
        s_off = off;
        if (blockIdx.x == 0) {
            long long o = 0;
            p.out_off[0] = 0;
            for (int i = 0; i < p.k; ++i) { o += min(p.ecnt[i], p.ecap); p.out_off[i + 1] = o; }
        }
    }
    if (threadIdx.x < kParts) s_pc[threadIdx.x] = 0;
    __syncthreads();
    if (lane >= p.k) return;
    const int cnt = min(p.ecnt[lane], p.ecap);
    if (cnt == 0) return;
    const int32_t* seg = p.ebuf + (size_t)lane * p.ecap;
    int32_t* out = p.out + s_off;
    const int64_t m = p.m > 0 ? p.m : 1;
    // part q holds [slice(q), slice(q + 1)), i.e. exactly the ids x with x * kParts / m == q
    auto slice = [&](int q) { return (m * q + kParts - 1) / kParts; };
    {
        int c[kParts] = {0, 0, 0, 0};
        for (int i = threadIdx.x; i < cnt; i += blockDim.x)
            c[min((int)((int64_t)seg[i] * kParts / m), kParts - 1)]++;
        for (int q = 0; q < kParts; ++q)
            if (c[q]) atomicAdd(&s_pc[q], c[q]);
    }
    __syncthreads();
    bool lane_mode = false;
    int below = 0;
    for (int q = 0; q < kParts; ++q) {
        lane_mode = lane_mode || s_pc[q] > kSortSmem;
        if (q < part) below += s_pc[q];
    }
    if (!lane_mode) {
        const int my = s_pc[part];
        if (my > 0) bucket_sort(seg, cnt, sbuf, my, out + below, slice(part), slice(part + 1), s_hist, s_cur);
        return;
    }
    if (part != 0) return;
    // the whole lane in one CTA, bucketed in global scratch
    bucket_sort(seg, cnt, p.tmp + (size_t)lane * p.ecap, cnt, out, 0, m, s_hist, s_cur);
}

__global__ void k_dist(DistParams p) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += gridDim.x * blockDim.x) {
        const int o = p.perm[v];
        const uint32_t* row = p.d + (size_t)v * p.K;
        for (int i = 0; i < p.k; ++i) p.out[(size_t)i * p.n + o] = (int32_t)row[i];
    }
}

// Vertices in range (Section 3's other output: the set of vertices in range),
// as one bitset over original vertex ids per query: a warp takes 32
// consecutive original ids, reads each one's in-range mask through its sweep
// position, and for every query i writes the 32-bit word whose bit t is bit i
// of vertex (v0 + t)'s mask (one ballot per query; lane i % 32 stores it).
template <int K>
__global__ void k_range(RangeParams p) {
    using MaskT = typename MaskOf<K>::T;
    const MaskT* mask = static_cast<const MaskT*>(p.mask);
    const int lane = threadIdx.x & 31;
    const int warps = (int)(gridDim.x * blockDim.x) >> 5;
    for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); (int64_t)w * 32 < p.n; w += warps) {
        const int v = w * 32 + lane;
        const unsigned long long m = v < p.n ? (unsigned long long)mask[__ldg(p.pos + v)] : 0ull;
        for (int i = 0; i < p.k; ++i) {
            const unsigned word = __ballot_sync(0xffffffffu, (m >> i) & 1ull);
            if (lane == (i & 31)) p.out[(size_t)i * p.words + w] = word;
        }
    }
}

}  // namespace

cudaError_t iso_launch_range(const isod::RangeParams& p, int K, cudaStream_t s) {
    const int grid = 1024;
    switch (K) {
        case 1: k_range<1><<<grid, 256, 0, s>>>(p); break;
        case 4: k_range<4><<<grid, 256, 0, s>>>(p); break;
        case 8: k_range<8><<<grid, 256, 0, s>>>(p); break;
        case 16: k_range<16><<<grid, 256, 0, s>>>(p); break;
        case 32: k_range<32><<<grid, 256, 0, s>>>(p); break;
        case 64: k_range<64><<<grid, 256, 0, s>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t iso_launch_emit(const isod::EmitParams& p, int K, int grid, cudaStream_t s) {
    switch (K) {
        case 1: k_emit<1><<<grid, kEmitThreads, 0, s>>>(p); break;
        case 4: k_emit<4><<<grid, kEmitThreads, 0, s>>>(p); break;
        case 8: k_emit<8><<<grid, kEmitThreads, 0, s>>>(p); break;
        case 16: k_emit<16><<<grid, kEmitThreads, 0, s>>>(p); break;
        case 32: k_emit<32><<<grid, kEmitThreads, 0, s>>>(p); break;
        case 64: k_emit<64><<<grid, kEmitThreads, 0, s>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t iso_launch_sort_gather(const isod::GatherParams& p, int K, cudaStream_t s) {
    const int smem = (kSortSmem + 2 * kMaxBuckets + 1) * 4;
    static std::atomic<unsigned long long> attr{0};
    if (cudaError_t e = iso_smem_attr_once(k_sort_gather, smem, attr)) return e;
    k_sort_gather<<<K * kParts, kSortThreads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t iso_launch_dist(const isod::DistParams& p, cudaStream_t s) {
    k_dist<<<1024, 256, 0, s>>>(p);
    return cudaGetLastError();
}
