/*
 * stencil.h - C ABI of the GB300-native FP64 stencil library.
 *
 * The library advances regular FP64 grids by T steps of a Jacobi or
 * Gauss-Seidel stencil, the computation classified in Section 1 of
 * "Temporal Vectorization for Stencils" (dimension, order, star or box
 * shape, Jacobi or Gauss-Seidel dependence, constant or periodic boundary)
 * and written as the naive (d+1)-loop code of Algorithm 1.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid layout: interior points only, C order, ext[0] the slowest dimension
 *   and ext[dim-1] the contiguous one; unused trailing ext[] entries are
 *   ignored. Data pointers are DEVICE pointers unless a name says "host".
 * Offsets: a stencil of radius r holds the offsets o in [-r, r]^dim; a star
 *   keeps those with at most one non-zero component, a box keeps all.
 *   "Canonical order" sorts them lexicographically, slowest dimension first.
 *   Coefficients are passed in canonical order.
 * Update: u'[p] = sum_o w_o * u[B(p + o)], the terms summed in DESCENDING
 *   canonical order. B is the boundary rule: a constant boundary reads the
 *   value c at every index outside the grid (corners included); a periodic
 *   boundary wraps every index modulo its extent.
 * Jacobi (Algorithm 1): every point of step t+1 reads step-t values only.
 * Gauss-Seidel (Section 3.4): one array updated in place, points visited in
 *   increasing lexicographic order, so already-visited neighbours contribute
 *   their newest value (Section 3.2: the space loop runs in increasing order).
 * Arithmetic: STENCIL_ARITH_FMA rounds the first product, then adds each
 *   further term with one fused multiply-add. STENCIL_ARITH_UNFUSED rounds
 *   every product and every sum. Both are bit-for-bit reproducible.
 * Streams: every run is asynchronous and stream-ordered on the given
 *   cudaStream_t (NULL = legacy default stream). Inputs must stay valid until
 *   the stream reaches the run.
 * Errors: synchronous argument and launch errors are returned as negative
 *   codes. Errors that happen on the device while a kernel runs (a bounded
 *   wait that gave up) are recorded in the handle's status word and returned
 *   by stencil_status(). No entry point aborts the process or traps the GPU.
 * Threads: a handle is not thread-safe; distinct handles may be used from
 *   different threads and streams at once.
 */
#ifndef GB300_STENCIL_H
#define GB300_STENCIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define STENCIL_OK 0
#define STENCIL_EINVAL (-1)       /* invalid argument */
#define STENCIL_EUNSUPPORTED (-2) /* valid but not supported (dim > 3, r > 4, ...) */
#define STENCIL_ENOMEM (-3)       /* device allocation failed */
#define STENCIL_ECUDA (-4)        /* a CUDA call or kernel launch failed */
#define STENCIL_ETIMEOUT (-5)     /* a device-side bounded wait gave up */
#define STENCIL_EBOUNDS (-6)      /* a device-side index check failed (checked build only: see
                                     stencil_checked_build) */

/* Stencil shape (Section 1 taxonomy). */
#define STENCIL_STAR 0
#define STENCIL_BOX 1
/* Dependence type (Section 1 taxonomy; Section 3.4). */
#define STENCIL_JACOBI 0
#define STENCIL_GAUSS_SEIDEL 1
/* Boundary condition (Section 1 taxonomy). */
#define STENCIL_BC_CONSTANT 0
#define STENCIL_BC_PERIODIC 1
/* Rounding of the weighted sum. */
#define STENCIL_ARITH_FMA 0
#define STENCIL_ARITH_UNFUSED 1

/* Kernel families a run may use (stencil_set_plan). */
#define STENCIL_KERNEL_AUTO 0      /* autotuned choice (default) */
#define STENCIL_KERNEL_PLAIN 1     /* one launch per Jacobi step / Gauss-Seidel sweep */
#define STENCIL_KERNEL_BLOCKED 2   /* Jacobi: tile + halo staged in shared memory, T_b steps per pass */
#define STENCIL_KERNEL_WAVEFRONT 3 /* Gauss-Seidel: time-skewed wavefront, warp lanes hold sweeps */
#define STENCIL_KERNEL_DIAMOND 4   /* Jacobi: split (diamond) temporal tiles, no redundant work, in place */
#define STENCIL_KERNEL_STREAM 5    /* Jacobi 2D/3D: slowest axis streamed, one ring of planes per time
                                      level in shared memory, T_b steps per pass */

typedef struct stencil_handle_s* stencil_handle; /* opaque, owned by the library */

typedef struct {
    double* data;     /* device pointer, the grid; holds the result after the run */
    int64_t ext[3];   /* extents, ext[0] slowest; entries beyond dim are ignored */
    double* scratch;  /* device pointer to workspace of stencil_workspace_bytes() bytes, or NULL */
} stencil_grid;

/*
 * Create a stencil.
 *   dim            1, 2 or 3.
 *   shape          STENCIL_STAR or STENCIL_BOX.
 *   radius         1..4 (the paper's kernels use 1).
 *   coeffs/ncoeffs host array of the K weights in canonical order; K must be
 *                  2*dim*radius+1 (star) or (2*radius+1)^dim (box). Copied.
 *   method         STENCIL_JACOBI or STENCIL_GAUSS_SEIDEL.
 *   boundary       STENCIL_BC_CONSTANT (value boundary_value) or STENCIL_BC_PERIODIC.
 *   arith          STENCIL_ARITH_FMA or STENCIL_ARITH_UNFUSED.
 *   out            receives the handle.
 * Allocates a small device block (weights, offsets, status word) on the
 * current device. Returns STENCIL_OK, EINVAL, EUNSUPPORTED, ENOMEM or ECUDA.
 */
int stencil_create(int dim, int shape, int radius, const double* coeffs, int ncoeffs, int method,
                   int boundary, double boundary_value, int arith, stencil_handle* out);

/*
 * Fix the kernel family and its parameters instead of the autotuned choice.
 *   kernel   STENCIL_KERNEL_* (AUTO restores the default).
 *   tb       temporal block depth T_b (BLOCKED, DIAMOND) or sweeps per warp
 *            (WAVEFRONT, 1..32); 0 = default.
 *   tile     tile extents (slowest first) for BLOCKED; period lengths per axis
 *            (slowest first) for DIAMOND; for WAVEFRONT in 2D/3D with a
 *            constant boundary, tile[0] = CTAs per SM of the persistent
 *            kernel, in 2D tile[1] = skewed rows per tile (2..64) and, in 2D,
 *            tile[2] = 0 (default) or 2 for rows as lanes
 *            where they apply (one weight per term or, for the 5-point
 *            star, a weight field; also the radius-2 star with one weight
 *            per term; rows of a multiple of 4 columns; a
 *            32-byte-aligned grid and field: a warp's lanes hold 32 rows of
 *            one sweep, the sweeps pipelined across warps; tile[0] = CTAs of
 *            four warps per SM, tile[1] = steps between progress
 *            publications, 8 (default), 16, 64 or 128), 8 or 16 for the
 *            points per lane and step of the one-warp tile (the default
 *            elsewhere, with 16), 1 for the decoupled tile of the 5-point
 *            star with one weight per term (a chain warp, producer warps and
 *            a scheduler warp per tile); for WAVEFRONT with a
 *            periodic boundary (the in-sweep tile DAG), tile[0] and tile[1] =
 *            lines per tile along axes 0 (3D) and 1, one thread each, at most
 *            256 in all, and tile[2] = hyperplane steps per tile; for STREAM,
 *            tile[0] = planes of the slowest axis per CTA (0: shared out
 *            evenly over one wave of resident CTAs), tile[1] = staged rows
 *            (3D), tile[2] = staged columns; for PLAIN Jacobi in 2D/3D with
 *            radius 1 and one weight per term, tile[2] = points per thread
 *            along the slow axis (2 or 4 in 2D, 1 or 2 in 3D); 0 = default.
 * A family that cannot run a given (method, boundary, grid) makes stencil_run
 * return EUNSUPPORTED.
 *
 * STREAM (Jacobi, 2D with radius 1 or 2, 3D with radius 1, constant weights)
 * is temporal blocking without a tile along the slowest axis (Section 1's
 * blocking methods; Section 3.4's tiles of T_b steps): a CTA owns a
 * cross-section tile (tile[2] = W2 staged columns, a multiple of 32 up to
 * 256; in 3D tile[1] = W1 staged rows) including a halo of T_b r per side,
 * and a chunk of tile[0] rows (2D) or planes (3D) of the slowest axis, which
 * it streams through shared memory: one ring of planes per time level, the
 * input planes arriving by TMA (constant boundary) or cp.async (periodic)
 * ahead of use, all T_b levels advancing behind one CTA barrier per group of
 * planes, the last level written straight to the output. HBM is read and
 * written once per T_b steps; only the cross-section halo is computed
 * twice. tb = T_b (1..4 in 2D with radius 1, else 1..2; larger values are
 * lowered); T mod T_b steps run as plain steps. 0 = default.
 *
 * DIAMOND (Jacobi) is the diamond temporal tiling of Section 3.4 in split
 * form on every axis: each axis is cut into periods of an A segment (a
 * trapezoid in space-time, shrinking by r per step) and a B segment (an
 * inverted trapezoid, growing by r per step); the 2^dim tile types of a band
 * of T_b steps run as 2^dim launches, A before B, and no point is computed
 * twice. It works in place on g->data (g->scratch is not used) and keeps the
 * per-level edge values of the tiles in a workspace owned by the handle
 * (about 4 * T_b * r / period of the grid per axis), allocated on first use
 * and grown when a run needs more; that first use must not be inside a
 * stream capture (EUNSUPPORTED there). T_b is lowered to fit the shortest
 * period (period >= 2 * T_b * r); an axis shorter than 2 * r points cannot be
 * tiled and returns EUNSUPPORTED. In 1D, when every period fits on the GPU at
 * once, the whole run is one cooperative launch in which each period advances
 * its two segments together and exchanges edge values with its neighbours
 * through flags (bounded waits: STENCIL_ETIMEOUT, never a hang).
 */
int stencil_set_plan(stencil_handle h, int kernel, int tb, const int64_t tile[3]);

/*
 * Advance g by T >= 0 steps (Jacobi) or sweeps (Gauss-Seidel) on stream
 * (a cudaStream_t). T = 0 returns at once. Jacobi needs workspace of one grid:
 * g->scratch if not NULL (stencil_workspace_bytes bytes, not aliasing data),
 * else the library allocates it stream-ordered and frees it after the run.
 * Periodic boundaries need every used extent >= 2*radius+1.
 * Returns STENCIL_OK or a negative code; device-side failures are reported
 * later by stencil_status().
 */
int stencil_run(stencil_handle h, const stencil_grid* g, int64_t T, void* cuda_stream);

/*
 * Run n independent problems (h[i], g[i], T[i]) with as few launches as
 * possible. One persistent kernel walks a shared work list: the time steps
 * (or T_b-step blocked passes, as each problem's tuned plan says) of every
 * Jacobi problem and the tile diagonals of every Gauss-Seidel sweep, a unit
 * starting once its problem's previous phase is done. Gauss-Seidel problems
 * whose plan is the wavefront kernel run as their own launches on the same
 * stream. The work of a batch shape (handles, pointers, extents, T, plans) is
 * prepared and captured into a CUDA graph on first use and replayed on later
 * calls with the same shape. Every Jacobi g[i] needs its scratch set. The
 * results equal n separate stencil_run calls bit for bit. Inside a stream
 * capture that the caller runs, only a batch shape already run once outside
 * capture is accepted (its prepared work is enqueued without allocating);
 * a new shape there returns STENCIL_EUNSUPPORTED.
 */
int stencil_run_batch(const stencil_handle* h, const stencil_grid* g, const int64_t* T, int n,
                      void* cuda_stream);

/*
 * Bind per-point coefficients: a variable-coefficient stencil, the form in
 * which Section 3.4 treats LCS's second sequence (its value at a point acts
 * as that point's coefficient). Runs of h then compute
 *     u'[p] = sum_o f_o[p] * u[B(p + o)]
 * with the same terms, order and rounding as with constant coefficients.
 *   field  DEVICE pointer to K * N doubles (8-byte aligned), N = ext[0] * ...
 *          * ext[dim-1]: the weight of canonical term q (0 <= q < K) at grid
 *          point p (C order) is field[q * N + p]. NULL unbinds it and
 *          restores the constant coefficients of stencil_create.
 *   ext    extents of the grids the field belongs to; a run of h on a grid of
 *          other extents returns STENCIL_EINVAL while the field is bound.
 * Not copied: the caller keeps the field allocated and unchanged until every
 * run that reads it has finished; the pointer is read at each run, so a
 * field rebound between runs of a captured batch makes a new graph.
 * Kernel families: Jacobi runs use the plain kernel (a BLOCKED plan returns
 * STENCIL_EUNSUPPORTED); Gauss-Seidel runs use the wavefront or plain sweeps
 * as with constant coefficients; in stencil_run_batch a problem with a field
 * runs as its own launches. Returns STENCIL_OK or STENCIL_EINVAL.
 */
int stencil_set_coeff_field(stencil_handle h, const double* field, const int64_t ext[3]);

/*
 * The kernel family and parameters stencil_run(h, g, T, stream) would use:
 * the fixed plan of stencil_set_plan, or the autotuned one (tuning first, on
 * private buffers, if this (stencil, extents, T) class has no cached plan;
 * inside a stream capture the cached or static default). kernel receives a
 * STENCIL_KERNEL_* value other than AUTO, tb the temporal block depth (or
 * sweeps per warp), tile the tile extents or periods (slowest first; 0 =
 * the kernel's default). Any output pointer may be NULL. Returns STENCIL_OK,
 * EINVAL or a CUDA error code.
 */
int stencil_get_plan(stencil_handle h, const stencil_grid* g, int64_t T, void* cuda_stream, int* kernel, int* tb,
                     int64_t tile[3]);

/* Bytes of workspace stencil_run needs for g (0 for Gauss-Seidel). */
int stencil_workspace_bytes(stencil_handle h, const stencil_grid* g, size_t* bytes);

/*
 * Synchronise stream, then return and clear the handle's device status:
 * STENCIL_OK, STENCIL_ETIMEOUT or STENCIL_EBOUNDS (or ECUDA if the
 * synchronisation itself failed). In the checked build it also reads and
 * clears the library's index-check fault records (process-wide, so a fault
 * of any handle's kernel is reported by the next call, whichever handle it
 * names) and answers STENCIL_EBOUNDS if one is set; bounds take precedence
 * over a time-out.
 */
int stencil_status(stencil_handle h, void* cuda_stream);

/* Release the handle and its device block (after its runs have finished). */
int stencil_destroy(stencil_handle h);

/* Static English text for a return code. */
const char* stencil_strerror(int code);

/*
 * End-to-end convenience over host memory: copy host_data (ext[0]*..*ext[dim-1]
 * doubles, pinned or pageable) to dev_data, run T steps, copy the result back
 * to host_data. dev_data and dev_scratch are caller-owned device buffers of one
 * grid each (dev_scratch may be NULL as in stencil_run). Synchronises stream
 * before returning, so host_data holds the result on return.
 */
int stencil_run_host(stencil_handle h, double* host_data, const int64_t ext[3], double* dev_data,
                     double* dev_scratch, int64_t T, void* cuda_stream);

/* Number of kernels this library has launched since load (all handles). */
uint64_t stencil_launch_count(void);

/*
 * Failure-detection test hook (no counterpart in the paper). The next run of h
 * that waits on other CTAs never publishes the completion of one unit of
 * work: in the wavefront Gauss-Seidel kernels tile number `unit` in the 2D/3D
 * schedule order, or sweep block `unit` in 1D; in the concurrent 1D diamond
 * Jacobi kernel period `unit` (-1 disables). Every wait on it gives up after
 * `spin` polls (0 = the default limit, about two seconds; in the diamond kernel
 * the first wait that gives up ends the others at once), the kernel finishes, and
 * stencil_status() then returns STENCIL_ETIMEOUT. The grid's contents after
 * such a run are unspecified. Nothing faults, traps or hangs.
 */
int stencil_debug_inject_stall(stencil_handle h, int64_t unit, int spin);

/*
 * 1 if this library is the checked build, else 0. The checked build (the same
 * sources compiled with -DSTENCIL_CHECKED into libgb300stencil_checked.so) tests
 * every index the stencil kernels form into a grid, a coefficient field, a
 * tile-flag table or a staged shared-memory tile (and that the staged tiles fit
 * the launch's shared memory) before the access; a failing test skips the
 * access and records the index, and stencil_status then returns
 * STENCIL_EBOUNDS. It stands in for a memory checker on small cases: the
 * results are otherwise bit-identical to the normal build's.
 */
int stencil_checked_build(void);

/*
 * Index-check test hook (no counterpart in the paper): one device thread on
 * stream tests index i against extent n with the checked build's index check
 * and touches no memory. In the checked build an i outside [0, n) makes the
 * next stencil_status() return STENCIL_EBOUNDS; the normal build tests
 * nothing. Returns STENCIL_ECUDA if the launch fails.
 */
int stencil_debug_check_index(int64_t i, int64_t n, void* cuda_stream);

/*
 * Jacobi run that allocates nothing (the paper has no counterpart; this is a
 * library service). For callers that may not allocate device memory: code
 * under a device-memory budget fixed in advance, real-time loops that must
 * not enter the CUDA allocator, host code running where allocation is
 * forbidden. Same result as stencil_run with the plain kernel; g->scratch is
 * ignored and the second Jacobi buffer is a fixed 16 MiB array inside the
 * library, held by every GPU that loads the library until the process exits.
 *   h        a Jacobi handle created on the current device (else EINVAL).
 *   g        grid of at most 2^21 points (2,097,152). Extents are checked as
 *            by stencil_run first (EINVAL, including extents whose product
 *            overflows); a valid grid with more points returns
 *            STENCIL_EUNSUPPORTED. Neither touches the GPU.
 *   T        steps, >= 0.
 * All calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller. The first call on each device looks up the
 * array's device address and should come before any stream capture begins;
 * that address is kept until the process exits and does not survive
 * cudaDeviceReset (do not call this entry point on a device after a reset).
 * No cudaMalloc, cudaFree or allocating library routine is called.
 */
int stencil_run_noalloc(stencil_handle h, const stencil_grid* g, int64_t T, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_STENCIL_H */
