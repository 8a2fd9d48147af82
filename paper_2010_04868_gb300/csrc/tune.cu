// Plan selection.
#include "tune.h"

namespace gbst {

Plan plan_for(const stencil_handle_s* h, const Geo& g, int64_t T)
{
    (void)g;
    (void)T;
    Plan p{STENCIL_KERNEL_PLAIN, 1, {0, 0, 0}};
    if (h->plan_kernel != STENCIL_KERNEL_AUTO) {
        p.kernel = h->plan_kernel;
        p.tb = h->plan_tb;
        for (int d = 0; d < 3; ++d) p.tile[d] = h->plan_tile[d];
    }
    return p;
}

int batch_run(const stencil_handle* h, const stencil_grid* g, const int64_t* T, int n, cudaStream_t st)
{
    for (int i = 0; i < n; ++i) {
        int rc = stencil_run(h[i], &g[i], T[i], st);
        if (rc) return rc;
    }
    return STENCIL_OK;
}

}  // namespace gbst
