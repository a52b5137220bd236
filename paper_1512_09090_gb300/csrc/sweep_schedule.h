// Chunk schedule of the TMA-staged sweep, built on the host (schedule.cpp).
#pragma once

#include <cstdint>
#include <vector>

// Everything the sweep needs to start the chunk at one schedule position, in
// one 32-byte record (two int4 on the device).
struct SchedChunk {
    int32_t v0, v1;  // sweep positions [v0, v1)
    int32_t level;   // level block index (0 = top level)
    int32_t mode;    // 0: a thread group per vertex, 1: a warp per vertex
    int32_t abase;   // first downward arc to stage (even, so the copy starts 16-byte aligned)
    int32_t na;      // arcs to stage from abase
    int32_t pa;      // its dependency list: pred[pa .. pa + np), pa a multiple of 4
    int32_t np;
};

struct SweepSchedule {
    std::vector<SchedChunk> info;  // by schedule position
    // dependency lists by position, each padded with repeats to a multiple of
    // four entries so that it can be copied in 16-byte units
    std::vector<int32_t> pred;
    std::vector<int32_t> succ;     // scratch
    int Q = 0;
};

// Builds the schedule for chunks of `vpb` vertices (levels narrower than
// narrow_width: chunks of narrow_chunk vertices, a warp per vertex) of levels
// sync_levels .. L-1; the levels above are swept before the schedule starts.
// chunk_span > 0 also ends a chunk where the BFS rank of its next vertex is
// chunk_span or more above that of its first (bfs is non-decreasing within a
// level).  Returns 0, or -1 if the input is inconsistent.
int iso_make_schedule(int n, int L, const int32_t* level_off, const uint32_t* down_off, const int32_t* down_src,
                      const int32_t* bfs, int vpb, int narrow_chunk, int narrow_width, int sync_levels, int delay,
                      int chunk_span, SweepSchedule* out);
