// Landmark distances for restricted sweeps (landmarks.cpp) and the lower
// bound they give (shared by the host and the device).
#pragma once

#include <cstdint>
#include <vector>

struct iso_ch;

// Distances are uint32: kUnreach = no path; a finite distance that does not
// fit is stored as kSat (a lower bound of the true one, see iso_lower_bound).
constexpr uint32_t kUnreach = 0xFFFFFFFFu;
constexpr uint32_t kSat = 0xFFFFFFFEu;

struct LandmarkSet {
    int count = 0;
    std::vector<int32_t> vertex;   // [count] sweep positions
    std::vector<uint32_t> fwd;     // [count * n] d(L_i, v), v a sweep position
    std::vector<uint32_t> bwd;     // [count * n] d(v, L_i)
};

// Picks `count` landmarks and computes both distance arrays.  0, or -1 on bad input.
int iso_landmarks_compute(const iso_ch& ch, int count, LandmarkSet* out);

// Per landmark i, for the sweep positions [v0, v1): lo_fwd[i] = min d(L_i, v),
// hi_bwd[i] = max d(v, L_i).
void iso_landmark_chunk_bounds(const LandmarkSet& lm, int n, int32_t v0, int32_t v1, uint32_t* lo_fwd,
                               uint32_t* hi_bwd);

// Lower bound on d(s, v) for every v of a chunk from one landmark, by the
// triangle inequality: a = d(L, s), b = d(s, L); lo = min over the chunk of
// d(L, v), hi = max of d(v, L).  Saturated and unreachable values are handled
// conservatively: a term is used only where every value it rests on is exact
// or errs towards a smaller bound.  Returns a value in [0, 2^32-1], where
// 2^32-1 means "no vertex of the chunk is reachable from s".
#if defined(__CUDACC__)
__host__ __device__
#endif
inline uint32_t iso_lower_bound(uint32_t a, uint32_t b, uint32_t lo, uint32_t hi) {
    uint32_t best = 0;
    // d(s,v) >= d(L,v) - d(L,s): needs d(L,s) exact
    if (a < kSat) {
        if (lo == kUnreach) return kUnreach;          // s reachable from L, no chunk vertex is
        if (lo > a) best = lo - a;
    }
    // d(s,v) >= d(s,L) - d(v,L): needs every d(v,L) exact (a saturated b only lowers the bound)
    if (hi < kSat) {
        if (b == kUnreach) return kUnreach;           // every chunk vertex reaches L, s does not
        if (b > hi && b - hi > best) best = b - hi;
    }
    return best;
}
