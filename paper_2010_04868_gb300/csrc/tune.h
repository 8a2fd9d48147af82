// Plan selection (kernel family and its parameters) and the batched runner.
#pragma once
#include "internal.h"

namespace gbst {

struct Plan {
    int kernel;       // STENCIL_KERNEL_PLAIN / BLOCKED / WAVEFRONT / DIAMOND
    int tb;           // temporal block depth (blocked, diamond) or sweeps per warp (wavefront)
    int64_t tile[3];  // tile extents (blocked) or period lengths (diamond), slowest first
};

// The plan a run uses: the handle's fixed plan if set, else the tuned one.
Plan plan_for(const stencil_handle_s* h, const Geo& g, int64_t T, cudaStream_t caller);

// Batched execution of n problems (see stencil_run_batch).
int batch_run(const stencil_handle* h, const stencil_grid* g, const int64_t* T, int n, cudaStream_t st);

}  // namespace gbst
