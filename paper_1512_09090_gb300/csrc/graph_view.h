// Read-only view of a device graph (iso_graph is defined in iso_api.cu), for
// code outside that file that launches the kernels on it: the
// allocation-free entry point.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "iso.h"

struct iso_graph_view {
    int n, L, tau_max, num_sms;
    int device;  // CUDA device the graph was uploaded to
    int64_t m;
    const uint32_t *down_off, *up_off, *orig_off;
    const int2 *down_arc, *up_arc;
    const int32_t *orig_head, *orig_id, *pos, *level_off, *emit_tail;
    const int32_t* h_level_off;
};

// Fills v from g.  ISO_E_INVAL if either is NULL.
int iso_graph_view_of(const iso_graph* g, iso_graph_view* v);
