// Host-side contraction hierarchy shared by the CH builder, the file format and
// the device upload.  Everything is stored in sweep order: vertices sorted by
// descending CH level, so every downward arc goes from a smaller to a larger
// sweep position and PHAST's scanning phase (Section 2) is a linear pass.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <vector>

struct iso_ch {
    int32_t n = 0;          // vertices
    int64_t m = 0;          // original arcs
    int32_t L = 0;          // CH levels
    int32_t max_w = 0;      // largest original length
    int64_t shortcuts = 0;  // shortcut arcs created
    double build_seconds = 0;

    std::vector<int32_t> perm;       // sweep position -> original vertex id
    std::vector<int32_t> pos;        // original vertex id -> sweep position
    // level_off[j] .. level_off[j+1] are the sweep positions of level L-1-j
    std::vector<int32_t> level_off;  // [L+1]
    // BFS rank (in the undirected input graph) of every sweep position: a
    // spatial key that orders chunks of different levels for cache locality
    std::vector<int32_t> bfs;        // [n]
    // incoming downward arcs (u -> v, rank(u) > rank(v)) of each sweep position v,
    // u given as a sweep position (always < v)
    std::vector<int64_t> down_off;   // [n+1]
    std::vector<int32_t> down_src, down_w;
    // outgoing upward arcs (v -> x, rank(x) > rank(v)); x is a sweep position < v
    std::vector<int64_t> up_off;     // [n+1]
    std::vector<int32_t> up_dst, up_w;
    // original arcs grouped by tail sweep position: head sweep position + input arc id
    std::vector<int64_t> orig_off;   // [n+1]
    std::vector<int32_t> orig_head, orig_id;
};

namespace iso {
// Thread-local last-error message (iso_last_error()).
void set_error(const char* fmt, ...);
void clear_error();
// Largest accepted input length: shortcut lengths are clamped to 2^31 - 2,
// which stays above every valid limit tau <= 2^31 - 2 - max_w.
constexpr int32_t kMaxWeight = (1 << 30) - 1;
}  // namespace iso
