// Isochrone edge emission (Section 3): arc (u,v) of the input graph is an
// isochrone edge for lane i iff exactly one of u, v is in range, i.e. iff bit i
// of mask[u] XOR mask[v] is set.  Arcs are visited grouped by tail (sweep
// order), so mask[u] is read once per vertex and mask[v] is a gather from a
// small array the sweep just wrote.  Per lane, ids are appended with one
// atomicAdd per warp: __ballot_sync gives the warp's members for that lane and
// __popc of the lower lanes gives each member's slot.
//
// Then one CTA per lane sorts its ids ascending (bitonic network, in shared
// memory when it fits, else in global memory) and writes them to the
// contiguous output at the lane's offset; CTA 0 also writes the offsets.
#include "iso_device.cuh"

namespace {

using namespace isod;

template <int K> struct MaskOf { using T = uint8_t; };
template <> struct MaskOf<16> { using T = uint16_t; };
template <> struct MaskOf<32> { using T = uint32_t; };
template <> struct MaskOf<64> { using T = unsigned long long; };

constexpr int kEmitThreads = 256;
constexpr int kSortThreads = 1024;
constexpr int kSortSmem = 32768;  // ids sorted in shared memory (128 KB)

__device__ __forceinline__ unsigned long long warp_or(unsigned long long x) {
    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)x);
    const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(x >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

template <int K>
__global__ void __launch_bounds__(kEmitThreads) k_emit(EmitParams p) {
    using MaskT = typename MaskOf<K>::T;
    const MaskT* mask = static_cast<const MaskT*>(p.mask);
    const unsigned lane_id = threadIdx.x & 31;
    const unsigned lt = (1u << lane_id) - 1u;
    for (int base = blockIdx.x * blockDim.x; base < p.n; base += gridDim.x * blockDim.x) {
        const int u = base + threadIdx.x;
        unsigned long long mu = 0;
        uint32_t a = 0, e = 0;
        if (u < p.n) {
            mu = mask[u];
            a = __ldg(p.orig_off + u);
            e = __ldg(p.orig_off + u + 1);
        }
        for (; __any_sync(0xffffffffu, a < e); ++a) {
            unsigned long long x = 0;
            int id = 0;
            if (a < e) {
                x = mu ^ (unsigned long long)mask[__ldg(p.orig_head + a)];
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
                if ((int)lane_id == leader) at = atomicAdd(p.ecnt + i, __popc(b));
                at = __shfl_sync(0xffffffffu, at, leader);
                if ((x >> i) & 1ull) {
                    const int q = at + __popc(b & lt);
                    if (q < p.ecap) p.ebuf[(size_t)i * p.ecap + q] = id;
                }
            }
        }
    }
}

// In-place ascending bitonic sort of s[0..n2), n2 a power of two, one CTA.
__device__ void bitonic(int32_t* s, int n2) {
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int ij = i ^ j;
                if (ij > i) {
                    const int32_t x = s[i], y = s[ij];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) { s[i] = y; s[ij] = x; }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_gather(GatherParams p) {
    extern __shared__ int32_t sbuf[];
    const int lane = blockIdx.x;
    __shared__ long long s_off;
    if (threadIdx.x == 0) {
        long long off = 0;
        for (int i = 0; i < lane; ++i) off += min(p.ecnt[i], p.ecap);
        s_off = off;
        if (lane == 0) {
            long long o = 0;
            p.out_off[0] = 0;
            for (int i = 0; i < p.k; ++i) { o += min(p.ecnt[i], p.ecap); p.out_off[i + 1] = o; }
        }
    }
    __syncthreads();
    if (lane >= p.k) return;
    const int cnt = min(p.ecnt[lane], p.ecap);
    if (cnt == 0) return;
    int n2 = 1;
    while (n2 < cnt) n2 <<= 1;
    const int32_t* seg = p.ebuf + (size_t)lane * p.ecap;
    int32_t* s = n2 <= kSortSmem ? sbuf : p.tmp + (size_t)lane * p.ecap;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) s[i] = i < cnt ? seg[i] : INT32_MAX;
    __syncthreads();
    bitonic(s, n2);
    int32_t* out = p.out + s_off;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) out[i] = s[i];
}

__global__ void k_dist(DistParams p) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += gridDim.x * blockDim.x) {
        const int o = p.perm[v];
        const uint32_t* row = p.d + (size_t)v * p.K;
        for (int i = 0; i < p.k; ++i) p.out[(size_t)i * p.n + o] = (int32_t)row[i];
    }
}

}  // namespace

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
    const int smem = kSortSmem * 4;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sort_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_sort_gather<<<K, kSortThreads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t iso_launch_dist(const isod::DistParams& p, cudaStream_t s) {
    k_dist<<<1024, 256, 0, s>>>(p);
    return cudaGetLastError();
}
