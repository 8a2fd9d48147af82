// Allocation-free Jacobi entry point.
//
// stencil_run needs one grid of device workspace for Jacobi (the second
// buffer of the ping-pong) and, when the caller passes none, allocates it
// with cudaMallocAsync. Some callers cannot allow that: code that runs under
// a hard device-memory budget fixed up front, real-time loops that must not
// enter the CUDA allocator (it can synchronise or fail under fragmentation),
// and host code that runs where allocation is forbidden (inside a memory pool
// owned by another framework, or while an allocator lock is held). For them,
// stencil_run_noalloc takes its workspace from a fixed array that is part of
// this library's device image, and never allocates.
//
// The array holds NOALLOC_MAX_POINTS doubles (16 MiB). Every GPU that loads
// the library keeps it for the life of the process. All calls share it, and
// it keeps the contents of the last call: calls whose work overlaps on the GPU
// (different streams, or different handles at once) race on it and must be
// serialised by the caller. Nothing in it needs to start at zero, because
// every Jacobi step writes every point of its output before any is read.
//
// The host cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the device address is looked up with
// cudaGetSymbolAddress once per device, on the first call made with that
// device current. That first call should therefore come before any stream
// capture begins. The address found is kept for the life of the process: it
// does not survive cudaDeviceReset (or anything else that destroys the
// device's primary context), after which this entry point must not be called
// on that device again.
#include <mutex>

#include "internal.h"

namespace {

constexpr int64_t NOALLOC_MAX_POINTS = int64_t(1) << 21;  // 2^21 doubles = 16 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_MAX_POINTS];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the fixed workspace on the current device (nullptr on failure).
double* noalloc_scratch(int device)
{
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) return nullptr;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_noalloc_ptr[device] = (double*)p;
    }
    return g_noalloc_ptr[device];
}

}  // namespace

extern "C" int stencil_run_noalloc(stencil_handle h, const stencil_grid* g, int64_t T, void* cuda_stream)
{
    using namespace gbst;
    if (!h || !g || T < 0) return STENCIL_EINVAL;
    if (h->method != STENCIL_JACOBI) return STENCIL_EINVAL;
    // the library's own grid checks (extents, periodic minimum, field extents,
    // and a size whose product cannot overflow) come first
    int rc = check_grid(h, g);
    if (rc) return rc;
    int64_t n = 1;
    for (int d = 0; d < h->dim; ++d) {
        if (g->ext[d] > NOALLOC_MAX_POINTS / n) return STENCIL_EUNSUPPORTED;  // n * ext > the maximum
        n *= g->ext[d];
    }
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) return STENCIL_ECUDA;
    if (device != h->device) return STENCIL_EINVAL;
    double* scratch = noalloc_scratch(device);
    if (!scratch) return STENCIL_ECUDA;
    if (T == 0) return STENCIL_OK;

    RunCtx ctx;
    ctx.h = h;
    ctx.g = make_geo(h->dim, g->ext);
    ctx.st = (cudaStream_t)cuda_stream;
    ctx.sd = make_sd(h, n);
    double* a = g->data;
    double* b = scratch;
    for (int64_t t = 0; t < T; ++t) {
        rc = jacobi_plain_step(ctx, a, b);
        if (rc) return rc;
        double* tmp = a;
        a = b;
        b = tmp;
    }
    if (a != g->data)
        return cuda_rc(cudaMemcpyAsync(g->data, a, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, ctx.st));
    return STENCIL_OK;
}
