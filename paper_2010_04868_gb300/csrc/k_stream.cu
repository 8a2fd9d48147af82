// Streaming temporally blocked Jacobi (2D and 3D): one HBM pass per T_b steps,
// halo redundancy on the cross-section only.
//
// Temporal tiling (Section 1, the blocking methods; Section 3.4: tiles of
// height T_b in time) advances a tile several steps while it stays on chip.
// Here the slowest axis (rows in 2D, planes in 3D) is streamed instead of
// tiled: a cross-section tile (a strip of W2 columns in 2D, W1 x W2 cells in
// 3D, each including a halo of h = T_b r on every side) is streamed over the
// rows/planes of the slowest axis. The tiles' planes, laid end to end, are
// shared out evenly over one wave of resident CTAs: each CTA takes the same
// number of planes, in one or two segments (a segment ends at a tile's last
// plane), so that all CTAs of a pass finish together. For each segment a CTA
// keeps, for every time level
// s = 0 .. T_b - 1, a ring of planes in shared memory and advances all levels
// in one pass along the streamed axis:
//   iteration it: level 0 (the input) receives M planes by TMA (issued two
//   iterations ahead), and each level s >= 1 computes M planes from the
//   planes level s - 1 finished in earlier iterations; level T_b writes its
//   planes straight to the output grid. One CTA barrier per iteration.
// Level s trails level s - 1 by M + r planes, so every value a level reads was
// produced before the last barrier. The streamed axis needs no halo beyond the
// segment's T_b r planes per side, so the only redundant work is the
// cross-section halo: about W2 / (W2 - 2h) in 2D (a warp of 32 columns is the
// unit of cost). Compared with staging a whole 2D or 3D tile per pass, each
// input value is loaded once per pass and nothing is decoded per point: every
// thread keeps its own cross-section cells for the whole kernel.
//
// Boundaries: with a constant boundary, TMA zero-fills the planes and cells
// outside the grid; they are set to c (when c != 0) before use, the rings of
// levels >= 1 hold c in their outside cells from the start, and an outside
// plane of a level is written as c. With a periodic boundary the planes are
// staged with cp.async from wrapped coordinates and every staged cell is a
// real (wrapped) grid value. Each point is computed with the same
// descending-order sum and rounding as the plain kernel, so the result is
// bit-identical to T_b plain steps.
#include <cuda.h>

#include <cstring>

#include "internal.h"

namespace gbst {

// Geometry of one launch (one pass of T_b steps).
struct StrGeo {
    int W1, W2;      // staged cross-section: W1 rows (1 in 2D) x W2 columns (a multiple of 32, <= 256)
    int B1, B2;      // output tile of the cross-section (W - 2h)
    int h;           // halo T_b * r per side on the cross-section axes
    int J;           // cross-section rows per thread (W1 / blockDim.y)
    int64_t per;     // planes of the streamed axis per CTA, the tiles' planes laid end to end
    int ns1, ns2;    // tiles along cross-section axes 1 (3D only) and 2
    int nblk;        // CTAs: ceil(ns1 ns2 nz / per), one balanced wave by default
    int C0, C;       // ring capacities (planes) of level 0 and of levels 1 .. T_b - 1
    int use_tma;     // level-0 planes by TMA (constant boundary) or by cp.async (periodic)
};

__device__ __forceinline__ uint32_t s_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bounded wait on an mbarrier phase; false on time-out.
__device__ __forceinline__ bool mbar_wait_parity(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 24); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// After a time-out: the same wait with a back-off, bounded at about a second,
// so that the CTA does not move on while the copy may still be landing.
__device__ __forceinline__ void mbar_wait_parity_backoff(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 20); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return;
        __nanosleep(1000);
    }
}

__device__ __forceinline__ int64_t wrap_mod(int64_t i, int64_t n)
{
    const int64_t m = i % n;
    return m < 0 ? m + n : m;
}

// Non-negative remainder of a (which may be negative, but > -4 c) modulo c.
__device__ __forceinline__ int ring_mod(int a, int c)
{
    a += 4 * c;
    return a % c;
}


// Input planes are requested this many iterations before the iteration that waits for them.
constexpr int STREAM_PF = 2;

// Level-0 load of planes [c0 + j M, + M) into ring slots (j M) mod C0 ...: by TMA (thread 0,
// mbarrier k mod (STREAM_PF + 1), k the CTA's running count of loads) or by cp.async from
// wrapped / checked coordinates (every thread, its own cells).
template <int DIM, int M>
__device__ __forceinline__ void stream_load(const CUtensorMap* tmap, const double* __restrict__ in, const Geo& g,
                                            int bc, double c, const StrGeo& sg, double* ring0, uint32_t bar_base,
                                            int64_t c0, int j, int k, int64_t gj0, int64_t gx0, int jb)
{
    const int P = sg.W1 * sg.W2;
    const int slot = (j * M) % sg.C0;
    const int64_t z = c0 + (int64_t)j * M;
    if (sg.use_tma) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const uint32_t bar = bar_base + 8u * (uint32_t)(k % (STREAM_PF + 1));
            const uint32_t bytes = (uint32_t)(M * P * 8);
            if (!GBST_IN((int64_t)(slot + M) * P - 1, (int64_t)sg.C0 * P)) {
                // checked build: the box would overrun ring 0; complete the phase without a copy
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
                return;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
            const uint32_t dst = s_u32(ring0 + (int64_t)slot * P);
            if (DIM == 2)
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                    "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst), "l"(tmap), "r"((int)gx0), "r"((int)z), "r"(bar)
                    : "memory");
            else
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                    "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst), "l"(tmap), "r"((int)gx0), "r"((int)gj0), "r"((int)z),
                    "r"(bar)
                    : "memory");
        }
        return;
    }
    const int64_t nz = DIM == 2 ? g.n1 : g.n0;
    const int64_t n1 = DIM == 3 ? g.n1 : 1;
    const int x = threadIdx.x;
    const int64_t gx = gx0 + x;
    for (int m = 0; m < M; ++m) {
        int64_t zz = z + m;
        bool zin = zz >= 0 && zz < nz;
        if (bc == BC_PERIODIC) zz = wrap_mod(zz, nz);
        for (int jj = jb; jj < jb + sg.J; ++jj) {
            int64_t gj = gj0 + jj;
            int64_t gxx = gx;
            bool in_grid = zin && gx >= 0 && gx < g.n2 && (DIM == 2 || (gj >= 0 && gj < n1));
            if (bc == BC_PERIODIC) {
                gxx = wrap_mod(gx, g.n2);
                if (DIM == 3) gj = wrap_mod(gj, n1);
                in_grid = true;
            }
            const int64_t di = (int64_t)(slot + m) * P + jj * sg.W2 + x;
            if (!GBST_IN(di, (int64_t)sg.C0 * P)) continue;
            double* d = ring0 + di;
            if (in_grid) {
                const int64_t si = (DIM == 3 ? zz * n1 + gj : zz) * g.n2 + gxx;
                if (!GBST_IN(si, g.n0 * g.n1 * g.n2)) continue;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s_u32(d)), "l"(in + si) : "memory");
            } else {
                *d = c;
            }
        }
    }
}

template <int DIM, int SHAPE, int R, int ARITH, int M, int TB>
__global__ void __launch_bounds__(256, 2) k_jacobi_stream(const __grid_constant__ CUtensorMap tmap,
                                                          const double* __restrict__ in, double* __restrict__ out,
                                                          Geo g, int bc, double c, StrGeo sg,
                                                          WArr<Stn<DIM, SHAPE, R>::K> w, int* status)
{
    using S = Stn<DIM, SHAPE, R>;
    constexpr int K = S::K;
    constexpr int ZA = DIM == 2 ? 1 : 0;  // the streamed axis among Stn's three offset components
    extern __shared__ __align__(128) double sm[];
    __shared__ __align__(8) uint64_t bars[STREAM_PF + 1];
    const int P = sg.W1 * sg.W2;
    // checked build: all rings inside the launch's dynamic shared memory (uniform per CTA)
    if (!GBST_IN((int64_t)(sg.C0 + (TB - 1) * sg.C) * P - 1, (int64_t)(dyn_smem_bytes() / 8))) return;
    double* ring[TB];
    ring[0] = sm;
#pragma unroll
    for (int s = 1; s < TB; ++s) ring[s] = sm + (int64_t)(sg.C0 + (s - 1) * sg.C) * P;

    const int64_t nz = DIM == 2 ? g.n1 : g.n0;
    const int64_t n1 = DIM == 3 ? g.n1 : 1;
    const int pad = sg.h & 1;  // staged columns start one early when h is odd (TMA 16-byte rule)
    const int x = threadIdx.x;
    const int jb = threadIdx.y * sg.J;
    const bool constant = bc == BC_CONSTANT;
    const uint32_t bar_base = s_u32(&bars[0]);
    if (sg.use_tma && threadIdx.x == 0 && threadIdx.y == 0) {
        for (int i = 0; i <= STREAM_PF; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_base + 8u * i) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    griddep_wait();  // launched programmatically: the previous pass has finished writing its output

    // This CTA's planes: [a, e) of the tiles' planes laid end to end (tile-major), split into
    // segments at tile boundaries; every CTA gets the same number of planes.
    const int64_t total = (int64_t)sg.ns1 * sg.ns2 * nz;
    int64_t a = (int64_t)blockIdx.x * sg.per;
    const int64_t e = a + sg.per < total ? a + sg.per : total;
    int kbase = 0;  // level-0 loads issued by earlier segments (mbarrier phases)
    while (a < e) {
        const int64_t tile = a / nz;
        const int64_t z0 = a - tile * nz;
        const int64_t z1 = z0 + (e - a) < nz ? z0 + (e - a) : nz;
        const int t2 = (int)(tile % sg.ns2);
        const int t1 = (int)(tile / sg.ns2);
        const int64_t gj0 = DIM == 3 ? (int64_t)t1 * sg.B1 - sg.h : 0;
        const int64_t gx0 = (int64_t)t2 * sg.B2 - sg.h - pad;
        const int64_t gx = gx0 + x;
        const bool xout = gx < 0 || gx >= g.n2;
        const int64_t c0 = z0 - TB * R;
        const int niter = (int)((z1 - z0 - 1 + 2 * TB * R + TB * M) / M) + 1;
        const int64_t hi0 = z1 + TB * R;
        // cells outside the grid hold c in every plane of the rings of levels 1 .. TB - 1
        if (constant && TB > 1) {
            for (int jj = jb; jj < jb + sg.J; ++jj) {
                const int64_t gj = gj0 + jj;
                if (xout || (DIM == 3 && (gj < 0 || gj >= n1)))
                    for (int s = 1; s < TB; ++s)
                        for (int sl = 0; sl < sg.C; ++sl)
                            st_in(ring[s], (int64_t)sl * P + jj * sg.W2 + x, (int64_t)sg.C * P, c);
            }
        }
        __syncthreads();  // the rings are free (the previous segment is done) and the barriers initialised

        // the first STREAM_PF loads (one cp.async group each, possibly empty)
        for (int j = 0; j < STREAM_PF; ++j) {
            if (j < niter && c0 + (int64_t)j * M < hi0)
                stream_load<DIM, M>(&tmap, in, g, bc, c, sg, ring[0], bar_base, c0, j, kbase + j, gj0, gx0, jb);
            if (!sg.use_tma) asm volatile("cp.async.commit_group;" ::: "memory");
        }

        for (int it = 0; it < niter; ++it) {
            // (a) the load of level-0 planes for iteration it + STREAM_PF; its slots were last read
            //     before the previous barrier
            if (it + STREAM_PF < niter && c0 + (int64_t)(it + STREAM_PF) * M < hi0)
                stream_load<DIM, M>(&tmap, in, g, bc, c, sg, ring[0], bar_base, c0, it + STREAM_PF,
                                    kbase + it + STREAM_PF, gj0, gx0, jb);
            // (b) the planes loaded for iteration it are complete (and set to c where outside the grid);
            //     they are first read in iteration it + 1, after the barrier below
            if (!sg.use_tma) {
                asm volatile("cp.async.commit_group;" ::: "memory");
                asm volatile("cp.async.wait_group %0;" ::"n"(STREAM_PF) : "memory");
            } else if (c0 + (int64_t)it * M < hi0) {
                const int k = kbase + it;
                const uint32_t bar = bar_base + 8u * (uint32_t)(k % (STREAM_PF + 1));
                const uint32_t par = (uint32_t)((k / (STREAM_PF + 1)) & 1);
                if (!mbar_wait_parity(bar, par)) {
                    if (x == 0 && threadIdx.y == 0) atomicExch(status, DEV_TIMEOUT);
                    mbar_wait_parity_backoff(bar, par);
                }
                if (constant && c != 0.0) {
                    const int slot = (it * M) % sg.C0;
                    for (int m = 0; m < M; ++m) {
                        const int64_t zz = c0 + (int64_t)it * M + m;
                        const bool zout = zz < 0 || zz >= nz;
                        for (int jj = jb; jj < jb + sg.J; ++jj) {
                            const int64_t gj = gj0 + jj;
                            if (zout || xout || (DIM == 3 && (gj < 0 || gj >= n1)))
                                st_in(ring[0], (int64_t)(slot + m) * P + jj * sg.W2 + x, (int64_t)sg.C0 * P, c);
                        }
                    }
                }
            }
            // (c) every level advances M planes, from planes finished before the last barrier
    #pragma unroll
            for (int s = 1; s <= TB; ++s) {
                const int64_t cs = c0 - (int64_t)s * (M + R);
                const int64_t y0 = cs + (int64_t)it * M;
                const int64_t lo = z0 - (int64_t)(TB - s) * R, hi = z1 + (int64_t)(TB - s) * R;
                if (y0 + M <= lo || y0 >= hi) continue;
                const int lo_col = pad + s * R, hi_col = pad + 2 * sg.h + sg.B2 - s * R;
                if (x < lo_col || x >= hi_col) continue;
                const double* src = ring[s - 1];
                const int Cin = s == 1 ? sg.C0 : sg.C;
                const int64_t cin = c0 - (int64_t)(s - 1) * (M + R);
                int so[M + 2 * R];  // plane offsets of the input rows y0 - R .. y0 + M - 1 + R
                {
                    const int s0 = ring_mod((int)(y0 - R - cin), Cin);
    #pragma unroll
                    for (int i = 0; i < M + 2 * R; ++i) {
                        int t = s0 + i;
                        if (t >= Cin) t -= Cin;
                        so[i] = t * P;
                    }
                }
                int oo[M];  // plane offsets of the output rows in this level's ring
                {
                    const int d0 = (it * M) % sg.C;
    #pragma unroll
                    for (int m = 0; m < M; ++m) {
                        int t = d0 + m;
                        if (t >= sg.C) t -= sg.C;
                        oo[m] = t * P;
                    }
                }
                for (int jj = jb; jj < jb + sg.J; ++jj) {
                    if (DIM == 3 && (jj < s * R || jj >= sg.W1 - s * R)) continue;
                    const int64_t gj = gj0 + jj;
                    if (constant && (xout || (DIM == 3 && (gj < 0 || gj >= n1)))) continue;  // keeps c
                    const int cell = jj * sg.W2 + x;
                    double acc[M];
    #pragma unroll
                    for (int q = 0; q < K; ++q) {
                        const int dz = S::o(q, ZA), dj = DIM == 3 ? S::o(q, 1) : 0, dx = S::o(q, 2);
                        const int co = cell + dj * sg.W2 + dx;
    #pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const double v = ld_in(src, (int64_t)so[m + R + dz] + co, (int64_t)Cin * P);
                            acc[m] = q == 0 ? __dmul_rn(w.w[0], v) : acc_step<ARITH>(acc[m], w.w[q], v);
                        }
                    }
                    if (s < TB) {
                        double* dst = ring[s < TB ? s : 0];
    #pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const int64_t y = y0 + m;
                            if (y < lo || y >= hi) continue;
                            st_in(dst, (int64_t)oo[m] + cell, (int64_t)sg.C * P,
                                  (constant && (y < 0 || y >= nz)) ? c : acc[m]);
                        }
                    } else {
                        // the last level: the output tile, inside the grid
                        const int lx = x - pad - sg.h;
                        const int lj = DIM == 3 ? jj - sg.h : 0;
                        if (lx < 0 || lx >= sg.B2 || gx >= g.n2) continue;
                        if (DIM == 3 && (lj < 0 || lj >= sg.B1 || gj >= n1)) continue;
    #pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const int64_t y = y0 + m;
                            if (y < lo || y >= hi) continue;
                            st_in(out, (DIM == 3 ? y * n1 + gj : y) * g.n2 + gx, g.n0 * g.n1 * g.n2, acc[m]);
                        }
                    }
                }
            }
            __syncthreads();
        }
        // loads issued in this segment: j = 0 .. while c0 + j M < hi0, below niter
        {
            const int64_t need = (hi0 - c0 + M - 1) / M;
            kbase += (int)(need < niter ? need : niter);
        }
        if (!sg.use_tma) asm volatile("cp.async.wait_all;" ::: "memory");
        a += z1 - z0;
    }
}

// ------------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFnS)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFnS stream_encode_fn()
{
    static EncodeTiledFnS fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFnS)p;
        cudaGetLastError();
    }
    return fn;
}

// Planes per iteration (register blocking along the streamed axis).
template <int DIM>
constexpr int stream_m() { return DIM == 2 ? 4 : 2; }

bool jacobi_stream_supported(const stencil_handle_s* h, const Geo& g)
{
    (void)g;
    if (h->method != JACOBI || h->field) return false;
    if (h->dim == 2) return h->r <= 2;
    if (h->dim == 3) return h->r == 1;
    return false;
}

// Temporal depths with a compiled kernel, largest first.
static int stream_tb(const stencil_handle_s* h, int tb)
{
    const int maxtb = (h->dim == 2 && h->r == 1) ? 4 : 2;
    if (tb <= 0) tb = 2;
    if (tb > maxtb) tb = maxtb;
    if (h->dim == 2 && h->r == 1 && tb == 3) return 3;
    return tb;
}

// Geometry for depth tb from the plan's tile (Z, W1, W2); 0 = defaults. Returns the dynamic
// shared memory in bytes, or 0 if no valid geometry fits.
static size_t make_str(const stencil_handle_s* h, const Geo& g, int tb, const int64_t tile[3], StrGeo& sg, dim3& block)
{
    const int dim = h->dim, r = h->r;
    const int M = dim == 2 ? stream_m<2>() : stream_m<3>();
    const int64_t nz = dim == 2 ? g.n1 : g.n0;
    const int64_t n1 = dim == 3 ? g.n1 : 1;
    sg.h = tb * r;
    const int pad = sg.h & 1;
    int64_t W2 = tile && tile[2] > 0 ? tile[2] : (dim == 2 ? 256 : 64);
    W2 = (W2 + 31) / 32 * 32;
    if (W2 > 256) W2 = 256;
    while (W2 - 2 * sg.h - 2 * pad < 2 && W2 < 256) W2 += 32;
    // no wider than the grid needs (one tile)
    while (W2 > 32 && W2 - 32 - 2 * sg.h - 2 * pad >= g.n2) W2 -= 32;
    sg.W2 = (int)W2;
    sg.B2 = sg.W2 - 2 * sg.h - 2 * pad;
    if (sg.B2 < 2) return 0;
    if (dim == 3) {
        int64_t W1 = tile && tile[1] > 0 ? tile[1] : 16;
        if (W1 < 2 * sg.h + 1) W1 = 2 * sg.h + 1;
        if (W1 > 256) return 0;
        const int jg = (int)(256 / sg.W2);
        W1 = (W1 + jg - 1) / jg * jg;  // whole rows per thread
        sg.W1 = (int)W1;
        sg.B1 = sg.W1 - 2 * sg.h;
        sg.J = sg.W1 / jg;
        block = dim3(sg.W2, jg, 1);
    } else {
        sg.W1 = 1;
        sg.B1 = 1;
        sg.J = 1;
        block = dim3(sg.W2, 1, 1);
    }
    sg.C0 = ((STREAM_PF + 2) * M + 2 * r + M - 1) / M * M;
    sg.C = 2 * M + 2 * r;
    sg.ns2 = (int)((g.n2 + sg.B2 - 1) / sg.B2);
    sg.ns1 = dim == 3 ? (int)((n1 + sg.B1 - 1) / sg.B1) : 1;
    sg.per = tile && tile[0] > 0 ? tile[0] : 0;  // 0: set from the occupancy (stream_balance)
    sg.nblk = 0;
    const int64_t planes = sg.C0 + (int64_t)(tb - 1) * sg.C;
    const size_t smem = (size_t)planes * sg.W1 * sg.W2 * sizeof(double);
    if (smem > 227 * 1024) return 0;
    return smem;
}

// Planes per CTA: by default the tiles' planes shared out evenly over one wave of resident CTAs
// (occ per SM), so that every CTA of a pass finishes at about the same time; at least 2 M.
static bool stream_balance(StrGeo& sg, const Geo& g, int dim, int occ, int M)
{
    int nsm = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nz = dim == 2 ? g.n1 : g.n0;
    const int64_t total = (int64_t)sg.ns1 * sg.ns2 * nz;
    if (sg.per <= 0) {
        const int64_t slots = (int64_t)nsm * (occ > 0 ? occ : 1);
        sg.per = (total + slots - 1) / slots;
    }
    if (sg.per < 2 * M) sg.per = 2 * M;
    const int64_t nblk = (total + sg.per - 1) / sg.per;
    if (nblk > 0x7fffffffLL) return false;
    sg.nblk = (int)nblk;
    return true;
}

static bool stream_map(CUtensorMap& m, const double* base, const Geo& g, int dim, const StrGeo& sg, int M)
{
    if (((uintptr_t)base & 15) != 0 || (g.n2 * 8) % 16 != 0 || !stream_encode_fn()) return false;
    if (g.n2 >= (1LL << 31) || g.n1 >= (1LL << 31) || g.n0 >= (1LL << 31)) return false;
    cuuint64_t gdim[3], gstr[2];
    cuuint32_t box[3], es[3] = {1, 1, 1};
    if (dim == 2) {
        gdim[0] = (cuuint64_t)g.n2;
        gdim[1] = (cuuint64_t)g.n1;
        gstr[0] = (cuuint64_t)g.n2 * 8;
        box[0] = (cuuint32_t)sg.W2;
        box[1] = (cuuint32_t)M;
    } else {
        gdim[0] = (cuuint64_t)g.n2;
        gdim[1] = (cuuint64_t)g.n1;
        gdim[2] = (cuuint64_t)g.n0;
        gstr[0] = (cuuint64_t)g.n2 * 8;
        gstr[1] = (cuuint64_t)g.n2 * g.n1 * 8;
        box[0] = (cuuint32_t)sg.W2;
        box[1] = (cuuint32_t)sg.W1;
        box[2] = (cuuint32_t)M;
    }
    CUresult rr = stream_encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)dim, (void*)base, gdim, gstr,
                                     box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return rr == CUDA_SUCCESS;
}

template <int DIM, int SHAPE, int R, int TB>
static int stream_passes(const RunCtx& ctx, double*& src, double*& dst, int64_t npass, const int64_t tile[3])
{
    constexpr int K = Stn<DIM, SHAPE, R>::K;
    constexpr int M = stream_m<DIM>();
    WArr<K> w;
    for (int q = 0; q < K; ++q) w.w[q] = ctx.h->w_desc[q];
    StrGeo sg;
    dim3 block;
    const size_t smem = make_str(ctx.h, ctx.g, TB, tile, sg, block);
    if (!smem) return STENCIL_EUNSUPPORTED;
    auto kern = ctx.h->arith == ARITH_FMA ? k_jacobi_stream<DIM, SHAPE, R, ARITH_FMA, M, TB>
                                          : k_jacobi_stream<DIM, SHAPE, R, ARITH_UNFUSED, M, TB>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return STENCIL_ECUDA;
    // TMA for the constant boundary (zero fill outside, then c); periodic wraps with cp.async
    CUtensorMap mapA, mapB;
    memset(&mapA, 0, sizeof(mapA));
    memset(&mapB, 0, sizeof(mapB));
    bool tma = ctx.h->bc == BC_CONSTANT && stream_map(mapA, src, ctx.g, DIM, sg, M) &&
               stream_map(mapB, dst, ctx.g, DIM, sg, M);
    sg.use_tma = tma ? 1 : 0;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (int)(block.x * block.y), smem) != cudaSuccess) {
        cudaGetLastError();
        occ = 1;
    }
    if (!stream_balance(sg, ctx.g, DIM, occ, M)) return STENCIL_EUNSUPPORTED;
    const unsigned nblk = (unsigned)sg.nblk;
    const double* a0 = src;
    for (int64_t p = 0; p < npass; ++p) {
        const CUtensorMap& map = src == a0 ? mapA : mapB;
        if (launch_pdl(kern, dim3(nblk), block, smem, ctx.st, map, (const double*)src, dst, ctx.g, ctx.h->bc,
                       ctx.h->c, sg, w, ctx.h->d_status) != cudaSuccess) {
            cudaGetLastError();
            kern<<<nblk, block, smem, ctx.st>>>(map, src, dst, ctx.g, ctx.h->bc, ctx.h->c, sg, w, ctx.h->d_status);
        }
        g_launches++;
        if (cudaGetLastError() != cudaSuccess) return STENCIL_ECUDA;
        double* t = src;
        src = dst;
        dst = t;
    }
    return STENCIL_OK;
}

template <int DIM, int SHAPE, int R>
static int stream_dispatch(const RunCtx& ctx, double*& src, double*& dst, int64_t npass, int tb, const int64_t tile[3])
{
    if (tb == 1) return stream_passes<DIM, SHAPE, R, 1>(ctx, src, dst, npass, tile);
    if (tb == 2) return stream_passes<DIM, SHAPE, R, 2>(ctx, src, dst, npass, tile);
    if (DIM == 2 && R == 1 && tb == 3) return stream_passes<DIM, SHAPE, R, (DIM == 2 && R == 1) ? 3 : 2>(ctx, src, dst, npass, tile);
    if (DIM == 2 && R == 1 && tb == 4) return stream_passes<DIM, SHAPE, R, (DIM == 2 && R == 1) ? 4 : 2>(ctx, src, dst, npass, tile);
    return STENCIL_EUNSUPPORTED;
}

int jacobi_stream_run(const RunCtx& ctx, double* a, double* b, int64_t T, int tb_req, const int64_t tile[3])
{
    const stencil_handle_s* h = ctx.h;
    const int tb = stream_tb(h, tb_req);
    double* src = a;
    double* dst = b;
    const int64_t npass = T / tb;
    int rc = STENCIL_EUNSUPPORTED;
#define X(D, S, R) \
    if (h->dim == D && h->shape == S && h->r == R) rc = stream_dispatch<D, S, R>(ctx, src, dst, npass, tb, tile);
    X(2, STAR, 1) X(2, BOX, 1) X(2, STAR, 2) X(2, BOX, 2) X(3, STAR, 1) X(3, BOX, 1)
#undef X
    if (rc) return rc;
    // the remaining T mod T_b steps: plain steps
    for (int64_t t = npass * tb; t < T && rc == STENCIL_OK; ++t) {
        rc = jacobi_plain_step(ctx, src, dst);
        double* x = src;
        src = dst;
        dst = x;
    }
    if (rc == STENCIL_OK && src != a) {
        const size_t bytes = (size_t)(ctx.g.n0 * ctx.g.n1 * ctx.g.n2) * sizeof(double);
        rc = cuda_rc(cudaMemcpyAsync(a, src, bytes, cudaMemcpyDeviceToDevice, ctx.st));
    }
    return rc;
}

}  // namespace gbst
