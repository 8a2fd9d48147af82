// Host-side internals shared by the C ABI and the kernel launchers.
#pragma once
#include <atomic>
#include <cstdint>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "stencil.h"  // include/ (the build passes -I include)
#include "common.cuh"

struct stencil_handle_s {
    int dim, shape, r, K, method, bc, arith;
    double c;
    std::vector<double> w_desc;  // weights, descending canonical order
    std::vector<int> off_desc;   // 3 components per offset (padded, slowest first), same order
    double* d_w = nullptr;       // device copies of the two tables
    int* d_off = nullptr;
    int* d_status = nullptr;     // device status word
    // workspace of the wavefront Gauss-Seidel kernel (tile flags, schedule table,
    // ticket counter), owned by the handle and grown on demand
    void* wave_ws = nullptr;
    size_t wave_ws_bytes = 0;
    int wave_epoch = 0;
    // workspace of the split-tiled (diamond) Jacobi kernel: the per-level edge
    // bands of every tile, owned by the handle and grown on demand
    void* dia_ws = nullptr;
    size_t dia_ws_bytes = 0;
    // failure-detection test hook: the next wavefront run never publishes the
    // completion of this tile (2D/3D) or sweep block (1D); its waiters give up
    // after debug_spin polls instead of the default limit
    int64_t debug_stall_tile = -1;
    int debug_spin = 0;
    // per-point weights bound by stencil_set_coeff_field (caller-owned device
    // memory, canonical term-major) and the extents of the grids they belong to
    const double* field = nullptr;
    int64_t field_ext[3] = {0, 0, 0};
    int plan_kernel = STENCIL_KERNEL_AUTO;
    int plan_tb = 0;
    int64_t plan_tile[3] = {0, 0, 0};
    int device = 0;
};

namespace gbst {

extern std::atomic<uint64_t> g_launches;

struct RunCtx {
    stencil_handle_s* h;
    Geo g;
    cudaStream_t st;
    StencilDev sd;
    // wavefront Gauss-Seidel parameters of the run's plan (tile[] of a WAVEFRONT plan, 0 = default)
    int64_t wtile[3] = {0, 0, 0};
    // points per thread of the plain Jacobi step (tile[2] of a PLAIN plan: 2 or 4; 0 = default)
    int prb = 0;
};

inline int cuda_rc(cudaError_t e) { return e == cudaSuccess ? STENCIL_OK : STENCIL_ECUDA; }

// Launch with programmatic stream serialization (see griddep_wait): the kernel
// must call griddep_wait() before its first access to memory that the kernel
// before it in the stream may write.
template <class... P, class... A>
inline cudaError_t launch_pdl(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// Device-side description of h for a grid of npts points (the bound field, if any).
inline StencilDev make_sd(const stencil_handle_s* h, int64_t npts)
{
    return StencilDev{h->K, h->r, h->bc, h->arith, h->c, h->d_w, h->d_off, h->d_status, h->field, npts};
}

// True if the plain kernels have a compile-time specialisation for (dim, shape, r).
bool plain_specialised(int dim, int shape, int r);

// One Jacobi step in -> out (plain, one launch).
int jacobi_plain_step(const RunCtx& ctx, const double* in, double* out);
// T Gauss-Seidel sweeps in place (plain: one sweep at a time).
int gs_plain_run(const RunCtx& ctx, double* u, int64_t T);

// Temporally blocked Jacobi: T steps from a (=g.data) using b (=scratch); the
// result ends in a. Returns EUNSUPPORTED if the configuration is not covered.
int jacobi_blocked_run(const RunCtx& ctx, double* a, double* b, int64_t T, int tb, const int64_t tile[3]);
bool jacobi_blocked_supported(const stencil_handle_s* h, const Geo& g);

// Streaming temporally blocked Jacobi (2D/3D): T steps from a (=g.data) using b
// (=scratch), passes of tb steps; the result ends in a. EUNSUPPORTED if the
// configuration is not covered.
int jacobi_stream_run(const RunCtx& ctx, double* a, double* b, int64_t T, int tb, const int64_t tile[3]);
bool jacobi_stream_supported(const stencil_handle_s* h, const Geo& g);

// Split-tiled (diamond) Jacobi: T steps in place on u, bands of H steps,
// periods of tile[d] points per axis (0 = defaults). Returns EUNSUPPORTED if
// the configuration or the grid is not covered.
int jacobi_diamond_run(const RunCtx& ctx, double* u, int64_t T, int H, const int64_t tile[3]);
bool jacobi_diamond_supported(const stencil_handle_s* h, const Geo& g);

// Time-skewed wavefront Gauss-Seidel: T sweeps in place.
int gs_wavefront_run(const RunCtx& ctx, double* u, int64_t T, int lanes);
// Size the handle's wavefront workspace for (g, T) and the plan's parameters ahead of a captured run.
int gs_wavefront_prepare(stencil_handle_s* h, const Geo& g, int64_t T, const int64_t wtile[3]);
bool gs_wavefront_supported(const stencil_handle_s* h, const Geo& g);

// Geometry from a stencil_grid (padded to three dimensions).
Geo make_geo(int dim, const int64_t ext[3]);

// Validation of a grid against a handle (STENCIL_OK or STENCIL_EINVAL); after
// it succeeds, the product of the extents times 8 fits in int64.
int check_grid(const stencil_handle_s* h, const stencil_grid* g);

}  // namespace gbst
