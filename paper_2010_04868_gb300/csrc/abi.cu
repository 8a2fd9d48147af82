// C ABI of the stencil library: argument checks, handle life cycle, and the
// choice of kernel family for each run.
#include <algorithm>
#include <cstring>
#include <new>

#include "internal.h"
#include "tune.h"

using namespace gbst;

namespace gbst {

Geo make_geo(int dim, const int64_t ext[3])
{
    Geo g{1, 1, 1};
    int64_t n[3] = {1, 1, 1};
    for (int d = 0; d < dim; ++d) n[3 - dim + d] = ext[d];
    g.n0 = n[0];
    g.n1 = n[1];
    g.n2 = n[2];
    return g;
}

// Argument checks shared by every entry point that takes a grid: extents >= 1
// (>= 2r+1 when periodic), the bound field's extents, and a byte size that
// fits in int64 (so no later product of the extents overflows).
int check_grid(const stencil_handle_s* h, const stencil_grid* g)
{
    if (!h || !g || !g->data) return STENCIL_EINVAL;
    for (int d = 0; d < h->dim; ++d) {
        if (g->ext[d] < 1) return STENCIL_EINVAL;
        if (h->bc == STENCIL_BC_PERIODIC && g->ext[d] < 2 * h->r + 1) return STENCIL_EINVAL;
        if (h->field && g->ext[d] != h->field_ext[d]) return STENCIL_EINVAL;
    }
    int64_t n = 1;
    for (int d = 0; d < h->dim; ++d) {
        if (n > INT64_MAX / g->ext[d] / 8) return STENCIL_EINVAL;
        n *= g->ext[d];
    }
    return STENCIL_OK;
}

#ifdef STENCIL_CHECKED
// The fault-word readers of the library's translation units (checked build); each unit adds its own
// while the library loads.
static std::vector<unsigned long long (*)()>& chk_readers()
{
    static std::vector<unsigned long long (*)()> v;
    return v;
}

void chk_register(unsigned long long (*take)()) { chk_readers().push_back(take); }

// Read and clear every unit's fault word; true if any index check failed since the last call.
static bool chk_take_all()
{
    bool any = false;
    for (auto f : chk_readers()) any |= f() != 0;
    return any;
}
#endif

__global__ void k_check_index(int64_t i, int64_t n)
{
    const bool ok = GBST_IN(i, n);
    (void)ok;
}

}  // namespace gbst

// Canonical offsets (lexicographic, slowest axis first), padded to 3 components.
static int canonical_offsets(int dim, int shape, int r, std::vector<int>& off)
{
    off.clear();
    int lo0 = dim >= 3 ? -r : 0, hi0 = dim >= 3 ? r : 0;
    int lo1 = dim >= 2 ? -r : 0, hi1 = dim >= 2 ? r : 0;
    for (int a = lo0; a <= hi0; ++a)
        for (int b = lo1; b <= hi1; ++b)
            for (int c = -r; c <= r; ++c) {
                int nz = (a != 0) + (b != 0) + (c != 0);
                if (shape == STENCIL_STAR && nz > 1) continue;
                off.push_back(a);
                off.push_back(b);
                off.push_back(c);
            }
    return (int)off.size() / 3;
}

static int64_t npoints(int dim, const int64_t ext[3])
{
    int64_t n = 1;
    for (int d = 0; d < dim; ++d) n *= ext[d];
    return n;
}

extern "C" {

int stencil_create(int dim, int shape, int radius, const double* coeffs, int ncoeffs, int method, int boundary,
                   double boundary_value, int arith, stencil_handle* out)
{
    if (!out) return STENCIL_EINVAL;
    *out = nullptr;
    if (shape != STENCIL_STAR && shape != STENCIL_BOX) return STENCIL_EINVAL;
    if (method != STENCIL_JACOBI && method != STENCIL_GAUSS_SEIDEL) return STENCIL_EINVAL;
    if (boundary != STENCIL_BC_CONSTANT && boundary != STENCIL_BC_PERIODIC) return STENCIL_EINVAL;
    if (arith != STENCIL_ARITH_FMA && arith != STENCIL_ARITH_UNFUSED) return STENCIL_EINVAL;
    if (dim < 1 || radius < 1) return dim < 1 || radius < 0 ? STENCIL_EINVAL : STENCIL_EUNSUPPORTED;
    if (dim > 3 || radius > 4) return STENCIL_EUNSUPPORTED;
    if (!coeffs) return STENCIL_EINVAL;
    std::vector<int> off;
    int K = canonical_offsets(dim, shape, radius, off);
    if (ncoeffs != K) return STENCIL_EINVAL;
    stencil_handle_s* h = new (std::nothrow) stencil_handle_s();
    if (!h) return STENCIL_ENOMEM;
    h->dim = dim;
    h->shape = dim == 1 ? STENCIL_STAR : shape;  // in 1D a box is a star
    h->r = radius;
    h->K = K;
    h->method = method;
    h->bc = boundary;
    h->arith = arith;
    h->c = boundary_value;
    h->w_desc.resize(K);
    h->off_desc.resize(3 * K);
    for (int q = 0; q < K; ++q) {
        h->w_desc[q] = coeffs[K - 1 - q];
        for (int d = 0; d < 3; ++d) h->off_desc[3 * q + d] = off[3 * (K - 1 - q) + d];
    }
    cudaGetDevice(&h->device);
    bool ok = cudaMalloc(&h->d_w, sizeof(double) * K) == cudaSuccess &&
              cudaMalloc(&h->d_off, sizeof(int) * 3 * K) == cudaSuccess &&
              cudaMalloc(&h->d_status, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMemcpy(h->d_w, h->w_desc.data(), sizeof(double) * K, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->d_off, h->off_desc.data(), sizeof(int) * 3 * K, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(h->d_status, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFree(h->d_w);
        cudaFree(h->d_off);
        cudaFree(h->d_status);
        delete h;
        return STENCIL_ENOMEM;
    }
    *out = h;
    return STENCIL_OK;
}

int stencil_set_plan(stencil_handle h, int kernel, int tb, const int64_t tile[3])
{
    if (!h || kernel < STENCIL_KERNEL_AUTO || kernel > STENCIL_KERNEL_STREAM || tb < 0) return STENCIL_EINVAL;
    if ((kernel == STENCIL_KERNEL_BLOCKED || kernel == STENCIL_KERNEL_DIAMOND || kernel == STENCIL_KERNEL_STREAM) &&
        h->method != STENCIL_JACOBI)
        return STENCIL_EINVAL;
    if (kernel == STENCIL_KERNEL_WAVEFRONT && (h->method != STENCIL_GAUSS_SEIDEL || tb > 32)) return STENCIL_EINVAL;
    h->plan_kernel = kernel;
    h->plan_tb = tb;
    for (int d = 0; d < 3; ++d) h->plan_tile[d] = tile ? std::max<int64_t>(0, tile[d]) : 0;
    return STENCIL_OK;
}

int stencil_set_coeff_field(stencil_handle h, const double* field, const int64_t ext[3])
{
    if (!h) return STENCIL_EINVAL;
    if (!field) {
        h->field = nullptr;
        for (int d = 0; d < 3; ++d) h->field_ext[d] = 0;
        return STENCIL_OK;
    }
    if (!ext || ((uintptr_t)field & 7)) return STENCIL_EINVAL;
    int64_t n = 1;
    for (int d = 0; d < h->dim; ++d) {
        if (ext[d] < 1 || n > INT64_MAX / ext[d] / 8 / h->K) return STENCIL_EINVAL;
        n *= ext[d];
    }
    h->field = field;
    for (int d = 0; d < 3; ++d) h->field_ext[d] = d < h->dim ? ext[d] : 0;
    return STENCIL_OK;
}

int stencil_get_plan(stencil_handle h, const stencil_grid* g, int64_t T, void* cuda_stream, int* kernel, int* tb,
                     int64_t tile[3])
{
    int rc = check_grid(h, g);
    if (rc) return rc;
    if (T < 0) return STENCIL_EINVAL;
    Plan p = plan_for(h, make_geo(h->dim, g->ext), T, (cudaStream_t)cuda_stream);
    if (h->method == STENCIL_GAUSS_SEIDEL && p.kernel == STENCIL_KERNEL_WAVEFRONT &&
        !gs_wavefront_supported(h, make_geo(h->dim, g->ext)))
        p.kernel = STENCIL_KERNEL_PLAIN;
    if (kernel) *kernel = p.kernel;
    if (tb) *tb = p.tb;
    if (tile)
        for (int d = 0; d < 3; ++d) tile[d] = p.tile[d];
    return STENCIL_OK;
}

int stencil_workspace_bytes(stencil_handle h, const stencil_grid* g, size_t* bytes)
{
    if (!bytes) return STENCIL_EINVAL;
    int rc = check_grid(h, g);
    if (rc) return rc;
    *bytes = h->method == STENCIL_JACOBI ? (size_t)npoints(h->dim, g->ext) * sizeof(double) : 0;
    return STENCIL_OK;
}

int stencil_run(stencil_handle h, const stencil_grid* g, int64_t T, void* cuda_stream)
{
    int rc = check_grid(h, g);
    if (rc) return rc;
    if (T < 0) return STENCIL_EINVAL;
    if (T == 0) return STENCIL_OK;
    RunCtx ctx;
    ctx.h = h;
    ctx.g = make_geo(h->dim, g->ext);
    ctx.st = (cudaStream_t)cuda_stream;
    ctx.sd = make_sd(h, npoints(h->dim, g->ext));
    const size_t bytes = (size_t)npoints(h->dim, g->ext) * sizeof(double);

    if (h->method == STENCIL_GAUSS_SEIDEL) {
        Plan p = plan_for(h, ctx.g, T, ctx.st);
        if (p.kernel == STENCIL_KERNEL_WAVEFRONT) {
            if (!gs_wavefront_supported(h, ctx.g)) return STENCIL_EUNSUPPORTED;
            for (int d = 0; d < 3; ++d) ctx.wtile[d] = p.tile[d];
            return gs_wavefront_run(ctx, g->data, T, p.tb);
        }
        return gs_plain_run(ctx, g->data, T);
    }

    Plan p = plan_for(h, ctx.g, T, ctx.st);
    if (p.kernel == STENCIL_KERNEL_DIAMOND) {
        // in place: the grid's own array is the only one the split tiles need
        if (!jacobi_diamond_supported(h, ctx.g)) return STENCIL_EUNSUPPORTED;
        return jacobi_diamond_run(ctx, g->data, T, p.tb, p.tile);
    }
    double* scratch = g->scratch;
    bool owned = false;
    if (!scratch) {
        if (cudaMallocAsync(&scratch, bytes, ctx.st) != cudaSuccess) {
            cudaGetLastError();
            return STENCIL_ENOMEM;
        }
        owned = true;
    } else if (scratch == g->data) {
        return STENCIL_EINVAL;
    }
    if (p.kernel == STENCIL_KERNEL_BLOCKED) {
        if (!jacobi_blocked_supported(h, ctx.g))
            rc = STENCIL_EUNSUPPORTED;
        else
            rc = jacobi_blocked_run(ctx, g->data, scratch, T, p.tb, p.tile);
    } else if (p.kernel == STENCIL_KERNEL_STREAM) {
        if (!jacobi_stream_supported(h, ctx.g))
            rc = STENCIL_EUNSUPPORTED;
        else
            rc = jacobi_stream_run(ctx, g->data, scratch, T, p.tb, p.tile);
    } else {
        if (p.kernel == STENCIL_KERNEL_PLAIN) ctx.prb = (int)p.tile[2];
        double* a = g->data;
        double* b = scratch;
        for (int64_t t = 0; t < T && rc == STENCIL_OK; ++t) {
            rc = jacobi_plain_step(ctx, a, b);
            std::swap(a, b);
        }
        if (rc == STENCIL_OK && a != g->data)
            rc = cuda_rc(cudaMemcpyAsync(g->data, a, bytes, cudaMemcpyDeviceToDevice, ctx.st));
    }
    if (owned) cudaFreeAsync(scratch, ctx.st);
    return rc;
}

int stencil_run_batch(const stencil_handle* h, const stencil_grid* g, const int64_t* T, int n, void* cuda_stream)
{
    if (n < 0 || (n > 0 && (!h || !g || !T))) return STENCIL_EINVAL;
    return batch_run(h, g, T, n, (cudaStream_t)cuda_stream);
}

int stencil_status(stencil_handle h, void* cuda_stream)
{
    if (!h) return STENCIL_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) return STENCIL_ECUDA;
    int s = 0;
    if (cudaMemcpy(&s, h->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return STENCIL_ECUDA;
    if (s != DEV_OK && cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess) return STENCIL_ECUDA;
#ifdef STENCIL_CHECKED
    if (chk_take_all()) return STENCIL_EBOUNDS;
#endif
    if (s == DEV_TIMEOUT) return STENCIL_ETIMEOUT;
    if (s == DEV_BOUNDS) return STENCIL_EBOUNDS;
    return STENCIL_OK;
}

int stencil_destroy(stencil_handle h)
{
    if (!h) return STENCIL_EINVAL;
    cudaFree(h->d_w);
    cudaFree(h->d_off);
    cudaFree(h->d_status);
    cudaFree(h->wave_ws);
    cudaFree(h->dia_ws);
    delete h;
    return STENCIL_OK;
}

const char* stencil_strerror(int code)
{
    switch (code) {
        case STENCIL_OK: return "success";
        case STENCIL_EINVAL: return "invalid argument";
        case STENCIL_EUNSUPPORTED: return "unsupported configuration";
        case STENCIL_ENOMEM: return "device memory allocation failed";
        case STENCIL_ECUDA: return "CUDA call or kernel launch failed";
        case STENCIL_ETIMEOUT: return "a device-side bounded wait timed out";
        case STENCIL_EBOUNDS: return "a device-side index check failed";
        default: return "unknown error code";
    }
}

int stencil_run_host(stencil_handle h, double* host_data, const int64_t ext[3], double* dev_data, double* dev_scratch,
                     int64_t T, void* cuda_stream)
{
    if (!h || !host_data || !ext || !dev_data) return STENCIL_EINVAL;
    stencil_grid g;
    g.data = dev_data;
    g.scratch = dev_scratch;
    for (int d = 0; d < 3; ++d) g.ext[d] = ext[d];
    int rc = check_grid(h, &g);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t bytes = (size_t)npoints(h->dim, ext) * sizeof(double);
    if (cudaMemcpyAsync(dev_data, host_data, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return STENCIL_ECUDA;
    rc = stencil_run(h, &g, T, cuda_stream);
    if (rc) return rc;
    if (cudaMemcpyAsync(host_data, dev_data, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess) return STENCIL_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? STENCIL_OK : STENCIL_ECUDA;
}

uint64_t stencil_launch_count(void) { return g_launches.load(); }

int stencil_debug_inject_stall(stencil_handle h, int64_t unit, int spin)
{
    if (!h || unit < -1 || spin < 0) return STENCIL_EINVAL;
    h->debug_stall_tile = unit;
    h->debug_spin = spin;
    return STENCIL_OK;
}

int stencil_checked_build(void)
{
#ifdef STENCIL_CHECKED
    return 1;
#else
    return 0;
#endif
}

int stencil_debug_check_index(int64_t i, int64_t n, void* cuda_stream)
{
    k_check_index<<<1, 1, 0, (cudaStream_t)cuda_stream>>>(i, n);
    g_launches++;
    return cuda_rc(cudaGetLastError());
}

}  // extern "C"
