// Plain kernels: the on-GPU comparison point.
//
// Jacobi: one launch per time step (Algorithm 1: the time loop outside, all
// points of step t+1 from step-t values), ping-pong between two buffers.
//
// Gauss-Seidel: one sweep at a time, in place (Section 3.4). The points of a
// sweep are visited so that every point sees the newest value of each
// neighbour that precedes it lexicographically and the old value of each
// neighbour that follows it:
//   * 1D: one thread walks x = 0 .. N-1 (the recurrence is serial).
//   * 2D/3D: points ordered by a point hyperplane index
//     theta(p) = sum_d c_d p_d, whose weights make every lexicographically
//     smaller neighbour precede and every larger one follow: c = 1 on every
//     axis for a star; for a box c_fast = 1, c_mid = 1 + r,
//     c_slow = 1 + r (c_mid + c_fast). Parallelogram tiles in (i, j, theta)
//     run one tile diagonal per launch, one CTA barrier per theta inside.
//   * Periodic boxes in 2D/3D: the wrap links the end of each row to its
//     start through a corner neighbour, which no hyperplane order respects;
//     one thread walks the grid in lexicographic order.
#include "internal.h"

namespace gbst {

std::atomic<uint64_t> g_launches{0};

#define GBST_SPECIALISED(X)          \
    X(1, STAR, 1) X(1, STAR, 2)      \
    X(1, STAR, 3) X(1, STAR, 4)      \
    X(2, STAR, 1) X(2, BOX, 1)       \
    X(2, STAR, 2) X(2, BOX, 2)       \
    X(3, STAR, 1) X(3, BOX, 1)       \
    X(3, STAR, 2)

#define GBST_TILE_SPECIALISED(X) \
    X(2, STAR, 1) X(2, BOX, 1)       \
    X(2, STAR, 2) X(2, BOX, 2)       \
    X(3, STAR, 1) X(3, BOX, 1)       \
    X(3, STAR, 2)

bool plain_specialised(int dim, int shape, int r)
{
#define X(D, S, R) \
    if (dim == D && shape == S && r == R) return true;
    GBST_SPECIALISED(X)
#undef X
    return false;
}

// ---------------------------------------------------------------- Jacobi ----

// Points per thread along the blocked axis (axis 1 in 2D, axis 0 in 3D): the
// unrolled points give each thread independent FMA chains, let their loads
// issue early and share the neighbour rows they have in common.
// With per-point weights (FIELD) every point also streams K weights from
// HBM: one point per thread and more resident warps hide that latency
// better than several points per thread (measured on 4096^2 5-point and
// 256^3 7-point grids: 63 -> 85 and 48 -> 52 GStencil/s).
constexpr int PLAIN_FIELD_RB2 = 1, PLAIN_FIELD_RB3 = 1;
constexpr int PLAIN_FIELD_MINB2 = 3, PLAIN_FIELD_MINB3 = 4;

template <int DIM, int K, bool FIELD = false>
__host__ __device__ constexpr int plain_rb()
{
    return DIM == 1 ? 1
                    : (DIM == 2 ? (FIELD ? PLAIN_FIELD_RB2 : (K <= 9 ? 4 : 2)) : (FIELD ? PLAIN_FIELD_RB3 : 2));
}

// Resident CTAs of 256 threads per SM the register budget must allow. The
// interior path needs few registers but the boundary path in the same body
// drove the allocation up (2D 72, 3D 7-point 80 with spills: 3 CTAs per SM);
// capped at 64 (4 CTAs) they fit without spills, and the 4096^2 5-point step
// runs ~6 % faster: 3 -> 4 resident CTAs of the same kernel shape measured
// 93-96 -> 98-102 GStencil/s on one GB300. The 2D radius-2 star fits 3 CTAs
// (78 registers, was 94: 2 CTAs); the 2D radius-2 box and the 27-point box
// would spill under a tighter cap and keep the looser one.
template <int DIM, int SHAPE, int R, bool FIELD>
__host__ __device__ constexpr int plain_minb()
{
    if (FIELD) return DIM == 3 ? PLAIN_FIELD_MINB3 : (DIM == 2 ? PLAIN_FIELD_MINB2 : 1);
    if (DIM == 2) return R == 1 ? 4 : (SHAPE == STAR ? 3 : 1);
    if (DIM == 3) return SHAPE == STAR && R == 1 ? 4 : 3;
    return 1;
}

// RBX: points per thread when a plain plan fixes it (0 = plain_rb's default).
template <int DIM, int SHAPE, int R, int ARITH, class WS, int RBX = 0>
__global__ void __launch_bounds__(256, plain_minb<DIM, SHAPE, R, WS::per_point>()) k_jacobi_plain(const double* __restrict__ u,
                                                      double* __restrict__ v, Geo g, int bc, double c, WS w)
{
    constexpr int RB = RBX > 0 ? RBX : plain_rb<DIM, Stn<DIM, SHAPE, R>::K, WS::per_point>();
    griddep_wait();  // launched programmatically: the previous step's writes are visible after this
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n2) return;
    const int64_t s1 = g.n2, s0 = g.n1 * g.n2, np = g.n0 * s0;
    const bool kin = k >= R && k < g.n2 - R;
    if (DIM == 3) {
        for (int64_t i0 = (int64_t)blockIdx.z * RB; i0 < g.n0; i0 += (int64_t)gridDim.z * RB)
            for (int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; j < g.n1;
                 j += (int64_t)gridDim.y * blockDim.y) {
                const bool jin = j >= R && j < g.n1 - R;
#pragma unroll
                for (int rb = 0; rb < RB; ++rb) {
                    const int64_t i = i0 + rb;
                    if (i < g.n0) {
                        const int64_t p = i * s0 + j * s1 + k;
                        const bool in = kin && jin && i >= R && i < g.n0 - R;
                        st_in(v, p, np, in ? update_interior<DIM, SHAPE, R, ARITH, true>(u, p, s0, s1, w, np)
                                           : update_bc<DIM, SHAPE, R, ARITH>(u, i, j, k, g, bc, c, w));
                    }
                }
            }
    } else {
        for (int64_t j0 = ((int64_t)blockIdx.y * blockDim.y + threadIdx.y) * RB; j0 < g.n1;
             j0 += (int64_t)gridDim.y * blockDim.y * RB) {
#pragma unroll
            for (int rb = 0; rb < RB; ++rb) {
                const int64_t j = j0 + rb;
                if (j < g.n1) {
                    const int64_t p = j * s1 + k;
                    const bool in = kin && (DIM < 2 || (j >= R && j < g.n1 - R));
                    st_in(v, p, np, in ? update_interior<DIM, SHAPE, R, ARITH, true>(u, p, s0, s1, w, np)
                                       : update_bc<DIM, SHAPE, R, ARITH>(u, 0, j, k, g, bc, c, w));
                }
            }
        }
    }
}

template <int ARITH>
__global__ void __launch_bounds__(256) k_jacobi_plain_rt(const double* __restrict__ u, double* __restrict__ v, Geo g,
                                                         StencilDev s)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n2) return;
    for (int64_t i = blockIdx.z; i < g.n0; i += gridDim.z)
        for (int64_t j = (int64_t)blockIdx.y * blockDim.y + threadIdx.y; j < g.n1;
             j += (int64_t)gridDim.y * blockDim.y)
            st_in(v, (i * g.n1 + j) * g.n2 + k, g.n0 * g.n1 * g.n2, update_rt<ARITH>(u, i, j, k, g, s));
}

static void plain_launch_shape(const Geo& g, dim3& grid, dim3& block)
{
    // 3D: 64 x 4 threads, so that the j +- 1 neighbours of a point come from rows this block also reads
    int bx = g.n0 > 1 ? 64 : 256;
    while (bx > 32 && bx / 2 >= g.n2) bx /= 2;
    block = dim3(bx, 256 / bx, 1);
    int64_t gx = (g.n2 + bx - 1) / bx;
    int64_t gy = (g.n1 + block.y - 1) / block.y;
    grid = dim3((unsigned)gx, (unsigned)(gy < 65535 ? gy : 65535), (unsigned)(g.n0 < 65535 ? g.n0 : 65535));
}

template <int DIM, int SHAPE, int R, class WS, int RBX = 0>
static void launch_jacobi_plain(const RunCtx& ctx, const double* in, double* out, const WS& w)
{
    constexpr int K = Stn<DIM, SHAPE, R>::K;
    constexpr int RB = RBX > 0 ? RBX : plain_rb<DIM, K, WS::per_point>();
    dim3 grid, block;
    plain_launch_shape(ctx.g, grid, block);
    if (DIM == 3) {
        const int64_t gz = (ctx.g.n0 + RB - 1) / RB;
        grid.z = (unsigned)(gz < 65535 ? gz : 65535);
    } else {
        const int64_t gy = (ctx.g.n1 + (int64_t)block.y * RB - 1) / ((int64_t)block.y * RB);
        grid.y = (unsigned)(gy < 65535 ? gy : 65535);
    }
    // programmatic launch: the next step's CTAs are scheduled while this one drains (+1-2 %)
    auto kern = ctx.h->arith == ARITH_FMA ? k_jacobi_plain<DIM, SHAPE, R, ARITH_FMA, WS, RBX>
                                          : k_jacobi_plain<DIM, SHAPE, R, ARITH_UNFUSED, WS, RBX>;
    if (launch_pdl(kern, grid, block, 0, ctx.st, in, out, ctx.g, ctx.h->bc, ctx.h->c, w) != cudaSuccess) {
        cudaGetLastError();  // a stream that refuses the attribute: an ordinary launch
        kern<<<grid, block, 0, ctx.st>>>(in, out, ctx.g, ctx.h->bc, ctx.h->c, w);
    }
}

template <int DIM, int SHAPE, int R>
static void launch_jacobi_plain(const RunCtx& ctx, const double* in, double* out)
{
    constexpr int K = Stn<DIM, SHAPE, R>::K;
    if (ctx.sd.field) {
        launch_jacobi_plain<DIM, SHAPE, R>(ctx, in, out, WField<K>{ctx.sd.field, ctx.sd.npts});
    } else {
        WArr<K> w;
        for (int q = 0; q < K; ++q) w.w[q] = ctx.h->w_desc[q];
        // a plain plan may fix the points per thread (radius 1: 2 or 4 in 2D, 1 or 2 in 3D, where 4 spills)
        if constexpr (DIM == 2 && R == 1) {
            if (ctx.prb == 2) return launch_jacobi_plain<DIM, SHAPE, R, WArr<K>, 2>(ctx, in, out, w);
            if (ctx.prb == 4) return launch_jacobi_plain<DIM, SHAPE, R, WArr<K>, 4>(ctx, in, out, w);
        }
        if constexpr (DIM == 3 && R == 1) {
            if (ctx.prb == 1) return launch_jacobi_plain<DIM, SHAPE, R, WArr<K>, 1>(ctx, in, out, w);
            if (ctx.prb == 2) return launch_jacobi_plain<DIM, SHAPE, R, WArr<K>, 2>(ctx, in, out, w);
        }
        launch_jacobi_plain<DIM, SHAPE, R>(ctx, in, out, w);
    }
}

int jacobi_plain_step(const RunCtx& ctx, const double* in, double* out)
{
    const stencil_handle_s* h = ctx.h;
    bool done = false;
#define X(D, S, R)                                                    \
    if (!done && h->dim == D && h->shape == S && h->r == R) {         \
        launch_jacobi_plain<D, S, R>(ctx, in, out);                   \
        done = true;                                                  \
    }
    GBST_SPECIALISED(X)
#undef X
    if (!done) {
        dim3 grid, block;
        plain_launch_shape(ctx.g, grid, block);
        if (h->arith == ARITH_FMA)
            k_jacobi_plain_rt<ARITH_FMA><<<grid, block, 0, ctx.st>>>(in, out, ctx.g, ctx.sd);
        else
            k_jacobi_plain_rt<ARITH_UNFUSED><<<grid, block, 0, ctx.st>>>(in, out, ctx.g, ctx.sd);
    }
    g_launches++;
    return cuda_rc(cudaGetLastError());
}

// ---------------------------------------------------------- Gauss-Seidel ----

// 1D: one thread, x ascending. win[m] holds the value at x - R + m: the R
// newest values to the left, the old centre, the R old values to the right.
// Indices that fall outside the grid read c (constant) or wrap (periodic);
// a right neighbour that wraps lands on an index this sweep has already
// updated, so it is read back from memory.
template <int R, int ARITH, class WS>
__global__ void k_gs1d_serial(double* u, int64_t n, int bc, double c, WS w)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    auto fetch = [&](int64_t x) -> double {
        if (x >= 0 && x < n) return ld_in(u, x, n);
        if (bc == BC_PERIODIC) return ld_in(u, x < 0 ? x + n : x - n, n);
        return c;
    };
    double win[2 * R + 1];
#pragma unroll
    for (int m = 0; m <= 2 * R; ++m) win[m] = fetch(m - R);
    for (int64_t x = 0; x < n; ++x) {
        // descending canonical order: offsets +R .. -R, i.e. win[2R] .. win[0]
        double acc = __dmul_rn(w.at(0, x), win[2 * R]);
#pragma unroll
        for (int q = 1; q <= 2 * R; ++q) acc = acc_step<ARITH>(acc, w.at(q, x), win[2 * R - q]);
        st_in(u, x, n, acc);
#pragma unroll
        for (int m = 0; m < 2 * R; ++m) win[m] = win[m + 1];
        win[R - 1] = acc;
        win[2 * R] = fetch(x + 1 + R);
    }
}

// Any dimension and shape: one thread visits every point in lexicographic order.
template <int ARITH>
__global__ void k_gs_serial_rt(double* u, Geo g, StencilDev s)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int64_t i = 0; i < g.n0; ++i)
        for (int64_t j = 0; j < g.n1; ++j)
            for (int64_t k = 0; k < g.n2; ++k)
                st_in(u, (i * g.n1 + j) * g.n2 + k, g.n0 * g.n1 * g.n2, update_rt<ARITH>(u, i, j, k, g, s));
}

// Parallelogram tiles for a Gauss-Seidel sweep (the paper uses parallelogram
// tiling for Gauss-Seidel stencils, Section 3.4). Points are placed in the
// skewed coordinates (i, sigma, theta): theta = cp0*i + cp1*j + k is the point
// hyperplane index and sigma = j + skew*i (skew = r for a 3D box, else 0).
// Every neighbour a point reads as "newest" then has all three coordinates
// <= its own and a smaller theta; every neighbour it reads as "old" has all
// three >= and a larger theta. So the points of one theta are independent,
// and boxes of B0 x B1 x BS in (i, sigma, theta) (2D: B1 x BS in (j, theta))
// can be processed whole in the tile order I + SIGMA + S: every tile a tile
// reads newest values from has a smaller index, every tile whose old values
// it reads a larger one.
struct TileGS {
    int b0, b1, bs;          // tile extents in (i, j, theta) (b0 = 1 in 2D)
    int64_t nt0, nt1, nts;   // tiles per axis
    int cp0, cp1;            // point hyperplane weights (fast axis weight 1)
    int skew;                // sigma = j + skew * i (3D)
};

// One tile diagonal D. Threads own the (i, j) lines of a tile (2D: j) and
// walk theta, one CTA barrier per theta.
template <int DIM, int SHAPE, int R, int ARITH, class WS>
__global__ void __launch_bounds__(256) k_gs_tile(double* u, Geo g, int bc, double c, WS w, TileGS t, int64_t D)
{
    int64_t T0, T1;
    if (DIM == 3) {
        T0 = blockIdx.x / t.nt1;
        T1 = blockIdx.x % t.nt1;
    } else {
        T0 = 0;
        T1 = blockIdx.x;
    }
    const int64_t TS = D - T0 - T1;
    if (TS < 0 || TS >= t.nts) return;
    const int64_t s1 = g.n2, s0 = g.n1 * g.n2;
    const int l1 = threadIdx.x % t.b1;
    const int l0 = threadIdx.x / t.b1;
    const int64_t i = T0 * t.b0 + l0;
    const int64_t j = T1 * t.b1 + l1 - (int64_t)t.skew * i;
    const bool owner = l0 < t.b0 && i < g.n0 && j >= 0 && j < g.n1;
    const int64_t kb = TS * t.bs - (int64_t)t.cp0 * i - (int64_t)t.cp1 * j;  // k at the tile's first theta
    const bool in01 = (DIM < 3 || (i >= R && i < g.n0 - R)) && (j >= R && j < g.n1 - R);
    for (int ls = 0; ls < t.bs; ++ls) {
        const int64_t k = kb + ls;
        if (owner && k >= 0 && k < g.n2) {
            const int64_t p = i * s0 + j * s1 + k;
            double r = (in01 && k >= R && k < g.n2 - R)
                           ? update_interior<DIM, SHAPE, R, ARITH, false>(u, p, s0, s1, w, g.n0 * s0)
                           : update_bc<DIM, SHAPE, R, ARITH>(u, i, j, k, g, bc, c, w);
            st_in(u, p, g.n0 * s0, r);
        }
        __syncthreads();
    }
}

template <int DIM, int SHAPE, int R, class WS>
static int gs_tiles(const RunCtx& ctx, double* u, int64_t T, const WS& w)
{
    const Geo& g = ctx.g;
    const bool box = SHAPE == BOX;
    TileGS t;
    t.cp1 = box ? 1 + R : 1;
    t.cp0 = DIM == 3 ? (box ? 1 + R * (t.cp1 + 1) : 1) : 0;
    t.skew = (DIM == 3 && box) ? R : 0;
    if (DIM == 3) {
        t.b0 = 16; t.b1 = 16; t.bs = 32;
    } else {
        t.b0 = 1; t.b1 = 64; t.bs = 64;
    }
    const int64_t thmax = t.cp0 * (g.n0 - 1) + t.cp1 * (g.n1 - 1) + (g.n2 - 1);
    t.nt0 = (g.n0 + t.b0 - 1) / t.b0;
    t.nt1 = (g.n1 + t.skew * (g.n0 - 1) + t.b1 - 1) / t.b1;
    t.nts = thmax / t.bs + 1;
    const int64_t Dmax = (t.nt0 - 1) + (t.nt1 - 1) + (t.nts - 1);
    const unsigned nblk = (unsigned)(DIM == 3 ? t.nt0 * t.nt1 : t.nt1);
    const unsigned nthr = (unsigned)(t.b0 * t.b1);
    for (int64_t s = 0; s < T; ++s)
        for (int64_t D = 0; D <= Dmax; ++D) {
            if (ctx.h->arith == ARITH_FMA)
                k_gs_tile<DIM, SHAPE, R, ARITH_FMA, WS><<<nblk, nthr, 0, ctx.st>>>(u, g, ctx.h->bc, ctx.h->c, w, t, D);
            else
                k_gs_tile<DIM, SHAPE, R, ARITH_UNFUSED, WS><<<nblk, nthr, 0, ctx.st>>>(u, g, ctx.h->bc, ctx.h->c, w, t, D);
            g_launches++;
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return STENCIL_ECUDA;
        }
    return STENCIL_OK;
}

template <int DIM, int SHAPE, int R>
static int gs_tiles(const RunCtx& ctx, double* u, int64_t T)
{
    constexpr int K = Stn<DIM, SHAPE, R>::K;
    if (ctx.sd.field) return gs_tiles<DIM, SHAPE, R>(ctx, u, T, WField<K>{ctx.sd.field, ctx.sd.npts});
    WArr<K> w;
    for (int q = 0; q < K; ++q) w.w[q] = ctx.h->w_desc[q];
    return gs_tiles<DIM, SHAPE, R>(ctx, u, T, w);
}

template <int R, class WS>
static int gs_1d(const RunCtx& ctx, double* u, int64_t T, const WS& w)
{
    for (int64_t s = 0; s < T; ++s) {
        if (ctx.h->arith == ARITH_FMA)
            k_gs1d_serial<R, ARITH_FMA, WS><<<1, 32, 0, ctx.st>>>(u, ctx.g.n2, ctx.h->bc, ctx.h->c, w);
        else
            k_gs1d_serial<R, ARITH_UNFUSED, WS><<<1, 32, 0, ctx.st>>>(u, ctx.g.n2, ctx.h->bc, ctx.h->c, w);
        g_launches++;
        if (cudaGetLastError() != cudaSuccess) return STENCIL_ECUDA;
    }
    return STENCIL_OK;
}

template <int R>
static int gs_1d(const RunCtx& ctx, double* u, int64_t T)
{
    if (ctx.sd.field) return gs_1d<R>(ctx, u, T, WField<2 * R + 1>{ctx.sd.field, ctx.sd.npts});
    WArr<2 * R + 1> w;
    for (int q = 0; q < 2 * R + 1; ++q) w.w[q] = ctx.h->w_desc[q];
    return gs_1d<R>(ctx, u, T, w);
}

int gs_plain_run(const RunCtx& ctx, double* u, int64_t T)
{
    const stencil_handle_s* h = ctx.h;
    if (h->dim == 1) {
        switch (h->r) {
            case 1: return gs_1d<1>(ctx, u, T);
            case 2: return gs_1d<2>(ctx, u, T);
            case 3: return gs_1d<3>(ctx, u, T);
            case 4: return gs_1d<4>(ctx, u, T);
        }
    }
    const bool tiles_ok = !(h->bc == BC_PERIODIC && h->shape == BOX);
    if (tiles_ok) {
#define X(D, S, R) \
    if (h->dim == D && h->shape == S && h->r == R) return gs_tiles<D, S, R>(ctx, u, T);
        GBST_TILE_SPECIALISED(X)
#undef X
    }
    for (int64_t s = 0; s < T; ++s) {
        if (h->arith == ARITH_FMA)
            k_gs_serial_rt<ARITH_FMA><<<1, 32, 0, ctx.st>>>(u, ctx.g, ctx.sd);
        else
            k_gs_serial_rt<ARITH_UNFUSED><<<1, 32, 0, ctx.st>>>(u, ctx.g, ctx.sd);
        g_launches++;
        if (cudaGetLastError() != cudaSuccess) return STENCIL_ECUDA;
    }
    return STENCIL_OK;
}

}  // namespace gbst
