// Restricted sweep: the chunks of the schedule that are out of range for every
// lane of a batch (RPHAST's restricted scan, Section 2; isoPHAST's active
// cells, Section 5, decide the same with precomputed cell distances).
//
// For lane i with source s and landmark L, every vertex v of chunk c has
//     d(s,v) >= max(min_c d(L,.) - d(L,s),  d(s,L) - max_c d(.,L))
// (iso_lower_bound, landmarks.h); a chunk is skipped when, for every lane, the
// largest of these bounds over the landmarks exceeds the lane's limit.  Each
// CTA first gathers the lanes' distances to and from the landmarks into shared
// memory, then a thread decides one chunk at a time.  Idle lanes (source -1)
// need nothing; a source outside [0, n) keeps every chunk (the upward search
// reports the bad input).
#include "iso_device.cuh"
#include "landmarks.h"

namespace {

using namespace isod;

constexpr int kMaxLm = 16;

__global__ void __launch_bounds__(256) k_skip(SkipParams p) {
    __shared__ uint32_t a[64][kMaxLm], b[64][kMaxLm], tau[64];
    __shared__ int active[64];
    __shared__ int s_count;
    for (int t = threadIdx.x; t < p.K * p.count; t += blockDim.x) {
        const int i = t / p.count, l = t % p.count;
        const int32_t s = p.src[i];
        const bool ok = s >= 0 && s < p.n;
        const int32_t v = ok ? p.pos[s] : 0;
        a[i][l] = ok ? p.lm_fwd[(size_t)l * p.n + v] : 0u;
        b[i][l] = ok ? p.lm_bwd[(size_t)l * p.n + v] : 0u;
    }
    for (int i = threadIdx.x; i < p.K; i += blockDim.x) {
        const int32_t s = p.src[i];
        // 0: idle; 1: decide by bounds; 2: keep everything (bad source)
        active[i] = s < 0 ? 0 : (s < p.n ? 1 : 2);
        tau[i] = p.tau[i] < 0 ? 0u : (uint32_t)p.tau[i];
    }
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    int mine = 0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < p.Q; q += gridDim.x * blockDim.x) {
        const uint32_t* lo = p.chunk_lo + (size_t)q * p.count;
        const uint32_t* hi = p.chunk_hi + (size_t)q * p.count;
        bool need = false;
        for (int i = 0; i < p.K && !need; ++i) {
            if (active[i] == 0) continue;
            if (active[i] == 2) { need = true; break; }
            uint32_t bound = 0;
            for (int l = 0; l < p.count; ++l) bound = max(bound, iso_lower_bound(a[i][l], b[i][l], lo[l], hi[l]));
            need = bound <= tau[i];
        }
        p.skip[q] = need ? 0 : 1;
        mine += need ? 0 : 1;
    }
    if (mine) atomicAdd(&s_count, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_count) atomicAdd(p.skipped, s_count);
}

}  // namespace

cudaError_t iso_launch_skip(const isod::SkipParams& p, int grid, cudaStream_t s) {
    if (p.count <= 0 || p.count > kMaxLm || p.K > 64) return cudaErrorInvalidValue;
    k_skip<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}
