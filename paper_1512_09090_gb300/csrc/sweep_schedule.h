// Chunk schedule of the TMA-staged sweep, built on the host (schedule.cpp).
#pragma once

#include <cstdint>
#include <vector>

struct SchedChunk {
    int32_t v0, v1;  // sweep positions [v0, v1), all in one level block
    int32_t level;   // level block index (0 = top level)
    int32_t mode;    // 0: a thread group per vertex, 1: a warp per vertex
};

struct SweepSchedule {
    std::vector<SchedChunk> info;  // by schedule position
    std::vector<int32_t> pred_off; // [Q+1] positions each position depends on: pred[pred_off[q]..]
    std::vector<int32_t> pred;
    std::vector<int32_t> succ;     // scratch
    int Q = 0;
};

// Builds the schedule for chunks of `vpb` vertices (levels narrower than
// narrow_width: chunks of narrow_chunk vertices, a warp per vertex).  Returns 0,
// or -1 if the input is inconsistent.
int iso_make_schedule(int n, int L, const int32_t* level_off, const uint32_t* down_off, const int32_t* down_src,
                      const int32_t* bfs, int vpb, int narrow_chunk, int narrow_width, int delay,
                      SweepSchedule* out);
