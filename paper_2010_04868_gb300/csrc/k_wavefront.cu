// Time-skewed wavefront Gauss-Seidel (placeholder until the kernel lands).
#include "internal.h"

namespace gbst {
bool gs_wavefront_supported(const stencil_handle_s*, const Geo&) { return false; }
int gs_wavefront_run(const RunCtx&, double*, int64_t, int) { return STENCIL_EUNSUPPORTED; }
}  // namespace gbst
