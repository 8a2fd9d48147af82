// Jacobi with split ("diamond") temporal tiles: no redundant work.
//
// Section 3.4 runs 1D Jacobi under diamond tiling, each time tile being a
// trapezoid or an inverted trapezoid, and higher-dimensional Jacobi under a
// diamond/parallelogram hybrid; unlike the overlapped tiles of the blocked
// kernel, no point is computed twice. Here the diamond tiling is realised as
// split tiling in every axis, which suits a GPU better than the hybrid: every
// tile of a phase is independent, so a phase is one launch and no tile waits
// for another.
//
// Along each used axis the grid is cut into n periods; period c spans
// [s_c, s_{c+1}) with s_c = floor(c N / n) and holds an A segment
// [s_c, s_c + W) followed by a B segment [s_c + W, s_{c+1}), where
// W = ceil((P + 2 H r) / 2) for the period length P and the band height H.
// Over a band of h <= H steps an A segment shrinks by r per step on each side
// that has a neighbour (a trapezoid) and a B segment grows by r per step on
// each side (an inverted trapezoid), so at every level the segments still
// partition the axis. A tile is one segment per axis; its type says A or B
// for each axis. The 2^d types run as 2^d phases in lexicographic order
// (A before B, slowest axis first), one launch each:
//   * a tile needs, outside its own level-(k-1) region, only values of tiles
//     that are A in the axes where it is B: an earlier phase;
//   * those tiles publish, for every level k < h and every axis where they
//     are A, the 2r points next to each of their edges (the band) in a
//     workspace array indexed by level, edge, offset and the full-grid
//     coordinates of the other two axes, so a consumer finds any point of
//     its ring, corners included, in one place;
//   * a tile reads its level-0 region from the grid and writes its level-h
//     region back to the grid, in place: a later phase's base never meets an
//     earlier phase's output (they differ in an axis where the earlier one is
//     A and the later B), so no second grid is needed.
// Inside a tile, levels run between two shared-memory buffers with one CTA
// barrier per level; the ring of level k is fetched with cp.async three levels
// ahead, into frame positions that no level in between reads or writes. Every
// point is computed once, with the same descending-order sum and rounding as
// the plain kernel, so the result equals T plain steps bit for bit. In 1D,
// when every period fits on the GPU at once, k_jacobi_hex1d below runs the
// whole run in one launch instead.
#include <algorithm>

#include "internal.h"

namespace gbst {

struct DiaGeo {
    int N[3];           // extents, slowest first (1 on unused axes)
    int n[3];           // periods per axis (1 on unused axes)
    int act[3];         // 1 on used axes
    int H;              // band height the segment widths are sized for
    int h;              // steps of this band (1..H)
    int fw[3];          // shared-memory frame extents (1 on unused axes)
    int bc;
    double c;
    double* band[3];    // per-axis band arrays (nullptr on unused axes)
    int64_t other[3];   // points of the two other axes
};

// Ring fetches in flight: the ring of level k is requested while level
// k - (DIA_AHEAD - 1) is computed, hiding the L2 latency behind that many levels.
constexpr int DIA_AHEAD = 4;

__device__ __forceinline__ int wrapn(int q, int n)
{
    while (q < 0) q += n;
    while (q >= n) q -= n;
    return q;
}

__device__ __forceinline__ void cp_async8(double* dst, const double* src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Walks the points of an e0 x e1 x e2 box (e2 fastest) from index i0 in steps
// of `stride` without a division per step.
struct BoxWalk {
    int x0, x1, x2, d0, d1, d2, e1, e2;
    __device__ __forceinline__ BoxWalk(int i0, int stride, int e1_, int e2_) : e1(e1_), e2(e2_)
    {
        x2 = i0 % e2;
        x1 = (i0 / e2) % e1;
        x0 = i0 / (e2 * e1);
        d2 = stride % e2;
        d1 = (stride / e2) % e1;
        d0 = stride / (e2 * e1);
    }
    __device__ __forceinline__ void next()
    {
        x2 += d2;
        x1 += d1;
        x0 += d0;
        if (x2 >= e2) {
            x2 -= e2;
            ++x1;
        }
        if (x1 >= e1) {
            x1 -= e1;
            ++x0;
        }
    }
};

// Geometry of one tile, per axis (global coordinates, unwrapped).
struct DiaTile {
    int lo[3], hi[3];  // level-0 segment
    int f0[3];         // frame origin
    int c[3];          // period index
    int isB[3];        // 1 if the tile is a B segment on this axis
    int shL[3];        // A only: the left side shrinks (has a neighbour)
};

__device__ __forceinline__ void dia_tile(const DiaGeo& G, int phase, int R, DiaTile& t)
{
    int b = (int)blockIdx.x;
    int cc[3];
    cc[2] = b % G.n[2];
    b /= G.n[2];
    cc[1] = b % G.n[1];
    cc[0] = b / G.n[1];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        t.c[d] = cc[d];
        if (!G.act[d]) {
            t.lo[d] = 0;
            t.hi[d] = 1;
            t.f0[d] = 0;
            t.isB[d] = 0;
            t.shL[d] = 0;
            continue;
        }
        const int64_t N = G.N[d], n = G.n[d];
        const int s0 = (int)(cc[d] * N / n), s1 = (int)((cc[d] + 1) * N / n), P = s1 - s0;
        const int W = min(P, (P + 2 * G.H * R + 1) / 2);
        t.isB[d] = (phase >> (2 - d)) & 1;
        if (!t.isB[d]) {
            t.lo[d] = s0;
            t.hi[d] = s0 + W;
            t.f0[d] = s0 - R;
            t.shL[d] = (G.bc == BC_PERIODIC || s0 > 0) ? 1 : 0;
        } else {
            t.lo[d] = s0 + W;
            t.hi[d] = s1;
            t.f0[d] = s0 + W - (G.H + 1) * R;
            t.shL[d] = 1;
        }
    }
}

// Region of the tile at level k on axis d: [L, U).
__device__ __forceinline__ void dia_range(const DiaGeo& G, const DiaTile& t, int d, int k, int R, int& L, int& U)
{
    if (!G.act[d]) {
        L = 0;
        U = 1;
    } else if (!t.isB[d]) {
        L = t.lo[d] + (t.shL[d] ? k * R : 0);
        U = t.hi[d] - k * R;
    } else {
        L = t.lo[d] - k * R;
        U = t.hi[d] + k * R;
        if (G.bc == BC_CONSTANT && U > G.N[d]) U = G.N[d];
    }
}

// Start of level k, edge e in the band array of axis d.
__device__ __forceinline__ double* dia_band(const DiaGeo& G, int d, int k, int e, int R)
{
    return G.band[d] + (((int64_t)k * 2 * G.n[d] + e) * 2 * R) * G.other[d];
}

// Publish the bands of level k (buffer b) on every axis where the tile is A:
// the 2r points next to each edge that has a neighbour, over the tile's
// level-k region on the other two axes.
template <int DIM, int R>
__device__ __forceinline__ void dia_export(const DiaGeo& G, const DiaTile& t, int k, const double* b)
{
    const int fs1 = G.fw[2], fs0 = G.fw[1] * G.fw[2];
    int L[3], U[3];
    if constexpr (DIM == 1) {
        // 1D: 2r values per side; the band of an edge is 2r consecutive doubles
        if (t.isB[2] || threadIdx.x >= 4 * R) return;
        dia_range(G, t, 2, k, R, L[2], U[2]);
        const int side = threadIdx.x < 2 * R ? 0 : 1, j = threadIdx.x - 2 * R * side;
        if (side == 0 && !t.shL[2]) return;
        const int start = side == 0 ? L[2] : U[2] - 2 * R;
        dia_band(G, 2, k, 2 * t.c[2] + side, R)[j] = b[start + j - t.f0[2]];
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) dia_range(G, t, d, k, R, L[d], U[d]);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (!G.act[d] || t.isB[d]) continue;
            // band of axis d: 2r x e0 x e1 points (e1 fastest); one warp per (j, row), lanes along e1
            const int a0 = d == 0 ? 1 : 0, a1 = d == 2 ? 1 : 2;
            const int e0 = U[a0] - L[a0], e1 = U[a1] - L[a1];
            const int fsd = d == 0 ? fs0 : (d == 1 ? fs1 : 1);
            const int fa0 = a0 == 0 ? fs0 : fs1, fa1 = a1 == 1 ? fs1 : 1;
            const int64_t na1 = G.N[a1];
            const int rows = 2 * R * e0;
            for (int side = t.shL[d] ? 0 : 1; side < 2; ++side) {
                const int start = side == 0 ? L[d] : U[d] - 2 * R;
                double* dst = dia_band(G, d, k, 2 * t.c[d] + side, R);
                const double* srcb = b + (start - t.f0[d]) * fsd + (L[a0] - t.f0[a0]) * fa0 + (L[a1] - t.f0[a1]) * fa1;
                for (int row = warp; row < rows; row += nwarp) {
                    const int j = row / e0, x0 = row - j * e0;
                    const int q0 = wrapn(L[a0] + x0, G.N[a0]);
                    double* drow = dst + (int64_t)j * G.other[d] + q0 * na1;
                    const double* srow = srcb + j * fsd + x0 * fa0;
                    for (int x1 = lane; x1 < e1; x1 += 32) drow[wrapn(L[a1] + x1, G.N[a1])] = srow[x1 * fa1];
                }
            }
        }
    }
}

// Request the ring of level k (the 2r points beyond the region on every axis
// where the tile is B, corners included) into buffer b with cp.async.
template <int DIM, int R>
__device__ __forceinline__ void dia_import(const DiaGeo& G, const DiaTile& t, int k, double* b)
{
    const int fs1 = G.fw[2], fs0 = G.fw[1] * G.fw[2];
    int L[3], U[3];
    if constexpr (DIM == 1) {
        // 1D: 2r values from the A segment on each side
        if (!t.isB[2] || threadIdx.x >= 4 * R) return;
        dia_range(G, t, 2, k, R, L[2], U[2]);
        const int jj = threadIdx.x;
        const int qd = jj < 2 * R ? L[2] - 2 * R + jj : t.hi[2] + k * R + jj - 2 * R;
        if (G.bc == BC_CONSTANT && (qd < 0 || qd >= G.N[2])) return;
        const double* src = jj < 2 * R ? dia_band(G, 2, k, 2 * t.c[2] + 1, R) + jj
                                       : dia_band(G, 2, k, 2 * ((t.c[2] + 1) % G.n[2]), R) + jj - 2 * R;
        cp_async8(b + qd - t.f0[2], src);
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) dia_range(G, t, d, k, R, L[d], U[d]);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (!G.act[d] || !t.isB[d]) continue;
            // slab of axis d: 4r positions on axis d; on other B axes, the region
            // (axes before d) or the region widened by 2r (axes after d)
            int lo[3], ex[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lo[a] = L[a];
                ex[a] = U[a] - L[a];
                if (a > d && G.act[a] && t.isB[a]) {
                    lo[a] -= 2 * R;
                    ex[a] += 4 * R;
                }
            }
            const int a0 = d == 0 ? 1 : 0, a1 = d == 2 ? 1 : 2;
            const int e0 = ex[a0], e1 = ex[a1];
            const int fsd = d == 0 ? fs0 : (d == 1 ? fs1 : 1);
            const int fa0 = a0 == 0 ? fs0 : fs1, fa1 = a1 == 1 ? fs1 : 1;
            const int64_t na1 = G.N[a1];
            const int Uu = t.hi[d] + k * R;  // right end before clipping to the grid
            const double* left = dia_band(G, d, k, 2 * t.c[d] + 1, R);                // right band of A on the left
            const double* right = dia_band(G, d, k, 2 * ((t.c[d] + 1) % G.n[d]), R);  // left band of the next A
            const int rows = 4 * R * e0;
            for (int row = warp; row < rows; row += nwarp) {
                const int jj = row / e0, x0 = row - jj * e0;  // jj 0..4r-1: left part, then right part
                const int qd = jj < 2 * R ? L[d] - 2 * R + jj : Uu + jj - 2 * R;
                const int qa0 = lo[a0] + x0;
                if (G.bc == BC_CONSTANT && (qd < 0 || qd >= G.N[d] || qa0 < 0 || qa0 >= G.N[a0]))
                    continue;  // outside the grid: holds c already
                const double* srow = (jj < 2 * R ? left + (int64_t)jj * G.other[d]
                                                 : right + (int64_t)(jj - 2 * R) * G.other[d]) +
                                     wrapn(qa0, G.N[a0]) * na1;
                double* drow = b + (qd - t.f0[d]) * fsd + (qa0 - t.f0[a0]) * fa0 + (lo[a1] - t.f0[a1]) * fa1;
                for (int x1 = lane; x1 < e1; x1 += 32) {
                    const int qa1 = lo[a1] + x1;
                    if (G.bc == BC_CONSTANT && (qa1 < 0 || qa1 >= G.N[a1])) continue;
                    cp_async8(drow + x1 * fa1, srow + wrapn(qa1, G.N[a1]));
                }
            }
        }
    }
}

// Two vertically adjacent points (rows y and y + 1 of the frame, frame offset
// p of the first) from one window of shared-memory loads: the terms of the
// second point are those of the first one row down, so the (2r + 2) rows of
// the window are loaded once (12 loads instead of 18 for a 9-point box). Each
// sum keeps the descending canonical order and rounding of update_interior.
template <int DIM, int SHAPE, int R, int ARITH, class WS>
__device__ __forceinline__ void update_pair(const double* src, int p, int fs0, int fs1, const WS& w, double& va,
                                            double& vb, int n)
{
    using S = Stn<DIM, SHAPE, R>;
    double a[S::K], b[S::K];
#pragma unroll
    for (int q = 0; q < S::K; ++q) {
        a[q] = ld_in(src, p + S::o(q, 0) * fs0 + S::o(q, 1) * fs1 + S::o(q, 2), n);
        b[q] = ld_in(src, p + S::o(q, 0) * fs0 + (S::o(q, 1) + 1) * fs1 + S::o(q, 2), n);
    }
    double acc = __dmul_rn(w.at(0, 0), a[0]), acb = __dmul_rn(w.at(0, 0), b[0]);
#pragma unroll
    for (int q = 1; q < S::K; ++q) {
        acc = acc_step<ARITH>(acc, w.at(q, 0), a[q]);
        acb = acc_step<ARITH>(acb, w.at(q, 0), b[q]);
    }
    va = acc;
    vb = acb;
}

template <int DIM, int SHAPE, int R, int ARITH>
__global__ void __launch_bounds__(256, (DIM == 2 && SHAPE == STAR && R == 1) ? 4 : 2) k_jacobi_diamond(double* __restrict__ u, DiaGeo G, int phase,
                                                           WArr<Stn<DIM, SHAPE, R>::K> w)
{
    extern __shared__ __align__(16) double sm[];
    const int F = G.fw[0] * G.fw[1] * G.fw[2];
    double* const bufA = sm;
    double* const bufB = sm + ((F + 1) & ~1);
    // checked build: both level buffers inside the launch's dynamic shared memory (uniform per CTA)
    if (!GBST_IN(((F + 1) & ~1) + F - 1, (int64_t)(dyn_smem_bytes() / 8))) return;
    auto buf = [&](int k) { return (k & 1) ? bufB : bufA; };  // level k's buffer, no local-memory array
    const int64_t NP = (int64_t)G.N[0] * G.N[1] * G.N[2];
    const int fs1 = G.fw[2], fs0 = G.fw[1] * G.fw[2];
    DiaTile t;
    dia_tile(G, phase, R, t);
    const int nthr = blockDim.x;

    // ---- level 0: constant boundary cells, the base from the grid, the rings of the first levels
    if (G.bc == BC_CONSTANT) {
        BoxWalk it(threadIdx.x, nthr, G.fw[1], G.fw[2]);
        for (int i = threadIdx.x; i < F; i += nthr, it.next()) {
            const int q0 = t.f0[0] + it.x0, q1 = t.f0[1] + it.x1, q2 = t.f0[2] + it.x2;
            if (q0 < 0 || q0 >= G.N[0] || q1 < 0 || q1 >= G.N[1] || q2 < 0 || q2 >= G.N[2]) {
                bufA[i] = G.c;
                bufB[i] = G.c;
            }
        }
    }
    {
        int L[3], U[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) dia_range(G, t, d, 0, R, L[d], U[d]);
        const int e2 = U[2] - L[2], e1 = U[1] - L[1];
        const int cnt = (U[0] - L[0]) * e1 * e2;
        BoxWalk it(threadIdx.x, nthr, e1, e2);
        for (int i = threadIdx.x; i < cnt; i += nthr, it.next()) {
            const int q0 = L[0] + it.x0, q1 = L[1] + it.x1, q2 = L[2] + it.x2;
            const int64_t gi = ((int64_t)wrapn(q0, G.N[0]) * G.N[1] + wrapn(q1, G.N[1])) * G.N[2] + wrapn(q2, G.N[2]);
            const int l = (q0 - t.f0[0]) * fs0 + (q1 - t.f0[1]) * fs1 + (q2 - t.f0[2]);
            if (GBST_IN(l, F) && GBST_IN(gi, NP)) cp_async8(bufA + l, u + gi);
        }
    }
    // groups: {base, ring 0}, ring 1, ..., ring DIA_AHEAD-1 (empty groups past the band)
    dia_import<DIM, R>(G, t, 0, bufA);
    cp_async_commit();
#pragma unroll
    for (int k = 1; k < DIA_AHEAD; ++k) {
        if (k < G.h) dia_import<DIM, R>(G, t, k, buf(k));
        cp_async_commit();
    }
    cp_async_wait<DIA_AHEAD - 1>();
    __syncthreads();

    if constexpr (DIM == 1) {
        // 1D: every per-level quantity is a tile constant plus a multiple of k
        const int f0 = t.f0[2], lo = t.lo[2], hi = t.hi[2], N = G.N[2], shL = t.shL[2];
        const bool isB = t.isB[2], clip = G.bc == BC_CONSTANT;
        const int64_t lvl = (int64_t)4 * G.n[2] * R;  // band doubles per level
        const int tid = threadIdx.x, side = tid < 2 * R ? 0 : 1, j = tid - 2 * R * side;
        const bool io = tid < 4 * R;
        // export (A): edge 2c + side; import (B): right band of A_c, left band of A_{c+1}
        double* const ex = G.band[2] + (2 * t.c[2] + side) * 2 * R + j;
        const double* const im =
            G.band[2] + (side == 0 ? (2 * t.c[2] + 1) * 2 * R : 2 * ((t.c[2] + 1) % G.n[2]) * 2 * R) + j;
        for (int k = 1; k <= G.h; ++k) {
            const double* src = buf(k - 1);
            double* dst = buf(k);
            if (io && !isB && (side == 1 || shL)) {
                const int km = k - 1;
                const int q = side == 0 ? lo + km * R + j : hi - km * R - 2 * R + j;
                ex[km * lvl] = src[q - f0];
            }
            const int kr = k + DIA_AHEAD - 1;
            if (io && isB && kr < G.h) {
                const int q = side == 0 ? lo - kr * R - 2 * R + j : hi + kr * R + j;
                if (!clip || (q >= 0 && q < N)) cp_async8(buf(kr) + (q - f0), im + kr * lvl);
            }
            cp_async_commit();
            const int L = isB ? lo - k * R : lo + (shL ? k * R : 0);
            const int U = isB ? (clip ? min(hi + k * R, N) : hi + k * R) : hi - k * R;
            for (int i = L - f0 + tid; i < U - f0; i += nthr)
                st_in(dst, i, F, update_interior<DIM, SHAPE, R, ARITH, false>(src, i, fs0, fs1, w, F));
            cp_async_wait<DIA_AHEAD - 1>();  // ring k has landed
            __syncthreads();
        }
    } else {
    // ---- levels 1..h: publish level k-1, compute level k, request ring k + DIA_AHEAD - 1
    for (int k = 1; k <= G.h; ++k) {
        const double* src = buf(k - 1);
        double* dst = buf(k);
        dia_export<DIM, R>(G, t, k - 1, src);
        {
            // the ring goes to positions no level before it reads or writes
            const int kr = k + DIA_AHEAD - 1;
            if (kr < G.h) dia_import<DIM, R>(G, t, kr, buf(kr));
            cp_async_commit();
        }
        int L[3], U[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) dia_range(G, t, d, k, R, L[d], U[d]);
        const int e2 = U[2] - L[2], e1 = U[1] - L[1];
        const int base = (L[0] - t.f0[0]) * fs0 + (L[1] - t.f0[1]) * fs1 + (L[2] - t.f0[2]);
        if constexpr (DIM == 3) {
            // two points per thread and pass, so that two independent sums are in flight
            const int cnt = (U[0] - L[0]) * e1 * e2;
            BoxWalk it(threadIdx.x, nthr, e1, e2);
            int i = threadIdx.x;
            for (; i + nthr < cnt; i += 2 * nthr) {
                const int pa = base + it.x0 * fs0 + it.x1 * fs1 + it.x2;
                it.next();
                const int pb = base + it.x0 * fs0 + it.x1 * fs1 + it.x2;
                it.next();
                const double va = update_interior<DIM, SHAPE, R, ARITH, false>(src, pa, fs0, fs1, w, F);
                const double vb = update_interior<DIM, SHAPE, R, ARITH, false>(src, pb, fs0, fs1, w, F);
                st_in(dst, pa, F, va);
                st_in(dst, pb, F, vb);
            }
            if (i < cnt) {
                const int pa = base + it.x0 * fs0 + it.x1 * fs1 + it.x2;
                st_in(dst, pa, F, update_interior<DIM, SHAPE, R, ARITH, false>(src, pa, fs0, fs1, w, F));
            }
            cp_async_wait<DIA_AHEAD - 1>();  // ring k has landed
            __syncthreads();
            continue;
        }
        // 2D: units of two vertically adjacent points (rows 2m and 2m + 1 of
        // the region, the second absent when the row count is odd), sharing loads
        const int e1h = (e1 + 1) >> 1, cntu = (U[0] - L[0]) * e1h * e2;
        BoxWalk it(threadIdx.x, nthr, e1h, e2);
        for (int i = threadIdx.x; i < cntu; i += nthr, it.next()) {
            const int y = 2 * it.x1;
            const int pa = base + it.x0 * fs0 + y * fs1 + it.x2;
            if (y + 1 < e1) {
                double va, vb;
                update_pair<DIM, SHAPE, R, ARITH>(src, pa, fs0, fs1, w, va, vb, F);
                st_in(dst, pa, F, va);
                st_in(dst, pa + fs1, F, vb);
            } else {
                st_in(dst, pa, F, update_interior<DIM, SHAPE, R, ARITH, false>(src, pa, fs0, fs1, w, F));
            }
        }
        cp_async_wait<DIA_AHEAD - 1>();  // ring k has landed
        __syncthreads();
    }
    }

    // ---- write level h back to the grid
    {
        const double* b = buf(G.h);
        int L[3], U[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) dia_range(G, t, d, G.h, R, L[d], U[d]);
        const int e2 = U[2] - L[2], e1 = U[1] - L[1];
        const int cnt = (U[0] - L[0]) * e1 * e2;
        BoxWalk it(threadIdx.x, nthr, e1, e2);
        for (int i = threadIdx.x; i < cnt; i += nthr, it.next()) {
            const int q0 = L[0] + it.x0, q1 = L[1] + it.x1, q2 = L[2] + it.x2;
            const int64_t gi = ((int64_t)wrapn(q0, G.N[0]) * G.N[1] + wrapn(q1, G.N[1])) * G.N[2] + wrapn(q2, G.N[2]);
            st_in(u, gi, NP, ld_in(b, (q0 - t.f0[0]) * fs0 + (q1 - t.f0[1]) * fs1 + (q2 - t.f0[2]), F));
        }
    }
}

// ---------------------------------------------------------- 1D, concurrent ---
//
// The same split tiles in 1D, but with the A and B segments of one period
// advancing together in one persistent launch, so that every step has all of
// a level's points in flight (the phase launches above hold half of them, and
// a 1D level has few points per SM). CTA c owns period c: its A segment (the
// trapezoid) computes level s at step s, its B segment (the inverted
// trapezoid, right of A) computes level s - HEX_LAG at the same step, one CTA
// barrier per step. B's ring comes from A's right band (shared memory) and
// from the left band of the next period's A (published by CTA c + 1). At the
// end of a band, A's next base takes its two edges from B tops: its own and
// the previous period's (published by CTA c - 1). The grid is read once at
// the start and written once at the end; every level stays on chip.
//
// Warp 0 does each step's edge I/O (bands, ring) and no stencil work, so that
// its latencies hide behind the other warps' FP64 chains; those synchronise on
// a named barrier once per step and count the steps in shared memory. The last
// warp does all inter-CTA traffic and no stencil work either, decoupled from
// the steps: it releases this CTA's A levels as the step count passes them,
// acquires the next period's progress, and copies the next period's A left
// band into a shared ring of 8 levels as soon as it is published and a slot is
// free, marking each level ready with a CTA-scope release; B's ring is written
// from it HEX_LAG steps after the level, so the L2 round trips never sit on a
// step. Every CTA must be resident at once: the launch is cooperative (after an
// occupancy check); every wait is bounded and records STENCIL_ETIMEOUT instead of
// hanging.
constexpr int HEX_LAG = 16;
constexpr int SPIN_LIMIT_DIAMOND = 1 << 23;  // x ~0.25-0.5 us per poll: a wait gives up after two to four seconds

struct HexGeo {
    int N, n, H, bc;
    double c;
    int64_t T;
    int fwA, fwB;        // frame widths of the A and B segments
    int* flagA;          // n: sequence number of the last A level whose left band is published
    int* flagB;          // n: last band whose B top is published
    double* aband;       // n x H x 2r: left band of A per level of the current band
    double* btop;        // n x H r: the part of B's top right of the period
    int* status;
    int* abort;          // grid-wide: set by the first wait that times out, so the others stop polling
    int spin;
    int stall;           // failure-detection test hook: this period never publishes (-1: none)
};

__device__ __forceinline__ int hex_ld_acquire(const int* f)
{
    int x;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(x) : "l"(f) : "memory");
    return x;
}

// A wait gave up: the CTA's other waits (*fail) and every other CTA's (*abort) stop polling.
__device__ __forceinline__ void hex_give_up(volatile int* fail, int* abort)
{
    *fail = 1;
    *(volatile int*)abort = 1;
}

// True once another wait of this CTA or of the grid has given up.
__device__ __forceinline__ bool hex_aborted(const volatile int* fail, const int* abort)
{
    return *fail || *(const volatile int*)abort;
}

// Bounded wait for *f >= v; gives up at once when another wait has timed out.
__device__ __forceinline__ bool hex_wait_ge(const int* f, int v, int spin, volatile int* fail, int* abort)
{
    for (int it = 0; it < spin && !hex_aborted(fail, abort); ++it) {
        if (hex_ld_acquire(f) >= v) return true;
        __nanosleep(it < 64 ? 32 : 256);
    }
    hex_give_up(fail, abort);
    return false;
}

__device__ __forceinline__ void hex_release(int* f, int v)
{
    __threadfence();
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(f), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire_cta(const int* p)
{
    int x;
    asm volatile("ld.acquire.cta.shared.b32 %0, [%1];" : "=r"(x) : "r"((uint32_t)__cvta_generic_to_shared(p)) : "memory");
    return x;
}

__device__ __forceinline__ void st_release_cta(int* p, int v)
{
    asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v) : "memory");
}

template <int R, int ARITH>
__global__ void __launch_bounds__(512) k_jacobi_hex1d(double* __restrict__ u, HexGeo G, WArr<2 * R + 1> w)
{
    extern __shared__ __align__(16) double sm[];
    __shared__ int step_done;   // compute warps: steps of the band completed
    __shared__ int ring_ready;  // comm warp: levels of the band in the ring
    __shared__ int fail;        // a wait of this CTA timed out: every other wait gives up at once
    const int c = blockIdx.x, n = G.n, N = G.N;
    const int s0 = (int)((int64_t)c * N / n), s1 = (int)((int64_t)(c + 1) * N / n), P = s1 - s0;
    const int W = min(P, (P + 2 * G.H * R + 1) / 2);
    const int loA = s0, hiA = s0 + W, loB = s0 + W, hiB = s1;
    const bool clip = G.bc == BC_CONSTANT;
    const bool hasL = !clip || c > 0;      // A shrinks on its left; its left band has a consumer
    const bool hasR = !clip || c < n - 1;  // B has an A segment on its right
    const int fA = loA - R, fB = loB - (G.H + 1) * R;  // frame origins (global coordinates, unwrapped)
    double* const A0 = sm;
    double* const A1 = A0 + G.fwA;
    double* const B0 = A1 + G.fwA;
    double* const B1 = B0 + G.fwB;
    double* const arb = B1 + G.fwB;         // H x 2r: A's right band per level
    double* const rvb = arb + G.H * 2 * R;  // 8 x 2r: the next period's A left band, ring of levels
    double* const alb = rvb + 8 * 2 * R;    // H x 2r: A's left band per level, staged for the comm warp
    const int nAB = 2 * G.fwA + 2 * G.fwB;  // the four level buffers
    // checked build: every staged array inside the launch's dynamic shared memory (uniform per CTA)
    if (!GBST_IN((int64_t)nAB + (2 * G.H + 8) * 2 * R - 1, (int64_t)(dyn_smem_bytes() / 8))) return;
    auto Ab = [&](int g) { return (g & 1) ? A1 : A0; };
    auto Bb = [&](int g) { return (g & 1) ? B1 : B0; };
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ncomp = nthr - 32;  // compute threads; the last warp communicates
    const bool comm = tid >= ncomp;
    const int lane = tid - ncomp;
    const int cl = (c + n - 1) % n, cr = (c + 1) % n;
    const int seqH = G.H + 1;
    const bool pub = c != G.stall;  // the failure-detection hook silences this period
    volatile int* vfail = &fail;
    if (tid == 0) fail = 0;

    // ---- the grid's values into buffer 0; cells outside the grid hold c in both buffers
    for (int i = tid; i < G.fwA; i += nthr) {
        const int q = fA + i;
        if (q < 0 || q >= N) {
            A0[i] = G.c;
            A1[i] = G.c;
        } else if (q >= loA && q < hiA) {
            A0[i] = u[q];
        }
    }
    for (int i = tid; i < G.fwB; i += nthr) {
        const int q = fB + i;
        if (clip && (q < 0 || q >= N)) {
            B0[i] = G.c;
            B1[i] = G.c;
        } else if (q >= loB && q < hiB) {
            B0[i] = u[q < N ? q : q - N];
        }
    }

    int g0 = 0;  // global level at the start of the band (buffer parity)
    for (int64_t done = 0, b = 0; done < G.T; ++b) {
        const int h = (int)min((int64_t)G.H, G.T - done);
        if (tid == 0) {
            step_done = 0;
            ring_ready = 0;
        }
        __syncthreads();
        if (!comm) {
            // ---- compute warps: step s = A at level s and B at level s - HEX_LAG, one named barrier per step
            int ring_known = 0;  // I/O warp: ring levels known to be ready
            for (int s = 1; s <= h + HEX_LAG; ++s) {
                const int kB = s - HEX_LAG, kx = s - 1, kr = s - HEX_LAG;
                const int aL = loA + (hasL ? s * R : 0) - fA, nA = s <= h ? hiA - s * R - fA - aL : 0;
                const int bL = loB - kB * R - fB;
                const int nB = (kB >= 1 && kB <= h) ? (clip ? min(hiB + kB * R, N) : hiB + kB * R) - fB - bL : 0;
                // offsets into the shared array itself, so that every access is a shared-memory one
                const int oAs = ((g0 + s - 1) & 1) * G.fwA, oAd = ((g0 + s) & 1) * G.fwA;
                const int oBs = 2 * G.fwA + ((g0 + kB - 1) & 1) * G.fwB, oBd = 2 * G.fwA + ((g0 + kB) & 1) * G.fwB;
                // warp 0 does this step's shared-memory and band I/O below; warps 1.. the points
                for (int i = tid - 32; i < nA + nB; i += ncomp - 32) {
                    if (i < 0) break;
                    const bool inA = i < nA;
                    const int ps = inA ? oAs + aL + i : oBs + bL + i - nA;
                    const int pd = inA ? oAd + aL + i : oBd + bL + i - nA;
                    st_in(sm, pd, nAB, update_interior<1, STAR, R, ARITH, false>(sm, ps, 0, 0, w, nAB));
                }
                // A's bands of level s - 1: the left one staged for the previous period, the right one for B
                if (kx < h && tid < 4 * R) {
                    const double* a = Ab(g0 + kx);
                    if (tid < 2 * R) {
                        if (hasL) alb[kx * 2 * R + tid] = a[loA + kx * R + tid - fA];
                    } else {
                        const int j = tid - 2 * R;
                        arb[kx * 2 * R + j] = a[hiA - (kx + 2) * R + j - fA];
                    }
                }
                // B's ring of level s - HEX_LAG (read by level s - HEX_LAG + 1 next step)
                if (kr >= 0 && kr < h && tid < 4 * R) {
                    double* bb = Bb(g0 + kr);
                    if (tid < 2 * R) {
                        bb[loB - (kr + 2) * R + tid - fB] = arb[kr * 2 * R + tid];
                    } else if (hasR) {
                        const int j = tid - 2 * R;
                        // the comm warp runs several levels ahead: acquire only when the known count runs out
                        for (int it = 0; ring_known <= kr; ++it) {
                            ring_known = ld_acquire_cta(&ring_ready);
                            if (ring_known > kr) break;
                            if (it >= G.spin || *vfail) {
                                hex_give_up(vfail, G.abort);
                                break;
                            }
                            __nanosleep(32);
                        }
                        bb[hiB + kr * R + j - fB] = rvb[(kr & 7) * 2 * R + j];
                    }
                }
                asm volatile("bar.sync 1, %0;" ::"r"(ncomp) : "memory");
                if (tid == 0) st_release_cta(&step_done, s);
            }
        } else {
            // ---- comm warp: release this CTA's A levels as the compute warps finish them, fetch
            // the next period's A levels into the ring as it publishes them and slots free up
            int rel = 0;    // levels of this CTA released
            int lv = 0;     // next level to fetch
            int known = 0;  // next period's last acquired sequence number
            int it = 0;
            while ((hasL && rel < h) || (hasR && lv < h)) {
                int sd = 0;  // read by one lane and broadcast: the warp's control flow stays uniform
                if (lane == 0) sd = ld_acquire_cta(&step_done);
                sd = __shfl_sync(0xffffffffu, sd, 0);
                bool progressed = false;
                // level k's band is staged at step k + 1: copy to global, then release
                if (hasL && rel < h && sd >= rel + 1) {
                    const int upto = min(sd, h);
                    for (int i = lane; i < (upto - rel) * 2 * R; i += 32)
                        G.aband[((int64_t)c * G.H + rel) * 2 * R + i] = alb[rel * 2 * R + i];
                    __syncwarp();
                    if (lane == 0 && pub) hex_release(G.flagA + c, (int)b * seqH + upto);
                    rel = upto;
                    progressed = true;
                }
                // slot lv & 7 held level lv - 8, consumed at step lv - 8 + HEX_LAG
                if (hasR && lv < h && sd >= lv - 8 + HEX_LAG) {
                    if (known < (int)b * seqH + lv + 1) {
                        int v = 0;
                        if (lane == 0) v = hex_ld_acquire(G.flagA + cr);
                        known = __shfl_sync(0xffffffffu, v, 0);
                        __syncwarp();  // the other lanes' loads come after lane 0's acquire
                    }
                    if (known >= (int)b * seqH + lv + 1) {
                        // every level the next period has published whose slot is free, in one batch
                        const int last = min(min(known - (int)b * seqH - 1, h - 1), sd + 8 - HEX_LAG);
                        for (int l = lv; l <= last; ++l)
                            if (lane < 2 * R)
                                rvb[(l & 7) * 2 * R + lane] = __ldcg(G.aband + ((int64_t)cr * G.H + l) * 2 * R + lane);
                        __syncwarp();
                        if (lane == 0) st_release_cta(&ring_ready, last + 1);
                        lv = last + 1;
                        progressed = true;
                    }
                }
                if (progressed) {
                    it = 0;  // the limit is on consecutive polls without progress
                } else {
                    __nanosleep(64);
                    if (++it >= G.spin || ((it & 31) == 0 && hex_aborted(vfail, G.abort))) {
                        hex_give_up(vfail, G.abort);
                        break;
                    }
                }
            }
        }
        __syncthreads();
        // ---- band end: B's top right part to the next period, A's next base from the B tops
        const double* btop = Bb(g0 + h);
        double* abase = Ab(g0 + h);
        if (hasR)
            for (int i = tid; i < h * R; i += nthr) G.btop[(int64_t)c * G.H * R + i] = btop[hiB + i - fB];
        for (int i = tid; i < h * R; i += nthr) abase[loB - h * R + i - fA] = btop[loB - h * R + i - fB];
        __syncthreads();
        if (tid == 0) {
            if (hasR && pub) hex_release(G.flagB + c, (int)b + 1);
            if (hasL) hex_wait_ge(G.flagB + cl, (int)b + 1, G.spin, vfail, G.abort);
        }
        __syncthreads();
        if (hasL)
            for (int i = tid; i < h * R; i += nthr) abase[loA + i - fA] = __ldcg(G.btop + (int64_t)cl * G.H * R + i);
        done += h;
        g0 += h;
    }
    __syncthreads();
    // ---- the period's final values back to the grid
    for (int i = loA + tid; i < hiA; i += nthr) u[i] = Ab(g0)[i - fA];
    for (int i = loB + tid; i < hiB; i += nthr) u[i] = Bb(g0)[i - fB];
    if (tid == 0 && *vfail) atomicExch(G.status, DEV_TIMEOUT);
}

// ------------------------------------------------------------------ host side

bool jacobi_diamond_supported(const stencil_handle_s* h, const Geo& g)
{
    (void)g;
    return h->method == JACOBI && !h->field && plain_specialised(h->dim, h->shape, h->r);
}

// Tiling of one run: periods per axis, band height, frame extents. Returns
// EUNSUPPORTED when an extent is too short for even one step per band.
int diamond_geometry(const stencil_handle_s* h, const Geo& g, int H, const int64_t tile_in[3], DiaGeo& G,
                     size_t& smem, size_t& ws_doubles)
{
    const int dim = h->dim, r = h->r;
    const int64_t N[3] = {g.n0, g.n1, g.n2};
    int nsm = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t P[3] = {tile_in ? tile_in[0] : 0, tile_in ? tile_in[1] : 0, tile_in ? tile_in[2] : 0};
    if (H <= 0) H = dim == 1 ? 32 : (dim == 2 ? 16 : 4);
    for (int d = 0; d < 3; ++d) {
        if (N[d] >= (int64_t(1) << 30)) return STENCIL_EUNSUPPORTED;
        G.act[d] = d >= 3 - dim;
        G.N[d] = (int)N[d];
        if (!G.act[d]) {
            P[d] = 1;
            continue;
        }
        if (P[d] <= 0) P[d] = dim == 1 ? std::max<int64_t>((N[d] + 4 * nsm - 1) / (4 * nsm), 64 * r) : (dim == 2 ? 88 : 24);
        if (P[d] < 2 * r) P[d] = 2 * r;
    }
    // periods: as many as fit the target length, at least one
    int64_t pmin = INT64_MAX;
    for (int d = 0; d < 3; ++d) {
        if (!G.act[d]) {
            G.n[d] = 1;
            continue;
        }
        int64_t n = N[d] / P[d];
        if (n < 1) n = 1;
        if (n > (1 << 30)) return STENCIL_EUNSUPPORTED;
        G.n[d] = (int)n;
        pmin = std::min(pmin, N[d] / n);
    }
    // every A segment must keep 2r points per side through the band: P >= 2 H r
    H = (int)std::min<int64_t>(H, pmin / (2 * r));
    if (H < 1) return STENCIL_EUNSUPPORTED;
    G.H = H;
    G.h = H;
    int64_t tiles = 1;
    for (int d = 0; d < 3; ++d) {
        G.fw[d] = 1;
        G.band[d] = nullptr;
        G.other[d] = 1;
        if (!G.act[d]) continue;
        int64_t fw = 0;
        for (int64_t c = 0; c < G.n[d]; ++c) {
            const int64_t s0 = c * N[d] / G.n[d], s1 = (c + 1) * N[d] / G.n[d], Pc = s1 - s0;
            const int64_t W = std::min<int64_t>(Pc, (Pc + 2 * (int64_t)H * r + 1) / 2);
            fw = std::max(fw, std::max(W + 2 * r, Pc - W + 2 * (int64_t)(H + 1) * r));
        }
        if (fw > (1 << 20)) return STENCIL_EUNSUPPORTED;
        G.fw[d] = (int)fw;
        tiles *= G.n[d];
    }
    const int64_t F = (int64_t)G.fw[0] * G.fw[1] * G.fw[2];
    smem = (size_t)(((F + 1) & ~int64_t(1)) + F) * sizeof(double);
    if (smem > 227 * 1024 || tiles > 0x7fffffffLL) return STENCIL_EUNSUPPORTED;
    ws_doubles = 0;
    for (int d = 0; d < 3; ++d) {
        if (!G.act[d]) continue;
        G.other[d] = (N[0] * N[1] * N[2]) / N[d];
        ws_doubles += (size_t)H * 2 * G.n[d] * 2 * r * G.other[d];
    }
    G.bc = h->bc;
    G.c = h->c;
    return STENCIL_OK;
}

// Grow the handle's band workspace to at least `bytes` (never inside a capture).
static int diamond_workspace(stencil_handle_s* h, size_t bytes, cudaStream_t st)
{
    if (h->dia_ws_bytes >= bytes) return STENCIL_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return STENCIL_EUNSUPPORTED;
    }
    if (h->dia_ws) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return STENCIL_ECUDA;
        cudaFree(h->dia_ws);
        h->dia_ws = nullptr;
        h->dia_ws_bytes = 0;
    }
    if (cudaMalloc(&h->dia_ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return STENCIL_ENOMEM;
    }
    h->dia_ws_bytes = bytes;
    return STENCIL_OK;
}

// 1D with every period resident at once: the concurrent kernel, one launch.
// Returns EUNSUPPORTED (nothing enqueued) when the periods do not all fit.
template <int R>
static int diamond_hex1d(const RunCtx& ctx, double* u, int64_t T, int H, const int64_t tile[3])
{
    const stencil_handle_s* h = ctx.h;
    const int64_t N = ctx.g.n2;
    int nsm = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (N >= (int64_t(1) << 30)) return STENCIL_EUNSUPPORTED;
    const int64_t P = tile && tile[2] > 0 ? tile[2] : (N + nsm - 1) / nsm;
    int64_t n = N / (P > 0 ? P : 1);
    if (n < 1) n = 1;
    if (n > 4 * nsm) return STENCIL_EUNSUPPORTED;
    const int64_t pmin = N / n;
    if (H <= 0) H = 100;
    H = (int)std::min<int64_t>(H, pmin / (2 * R));
    if (H < 1) return STENCIL_EUNSUPPORTED;
    int64_t fwA = 0, fwB = 0, pmax = 0;
    for (int64_t c = 0; c < n; ++c) {
        const int64_t s0 = c * N / n, s1 = (c + 1) * N / n, Pc = s1 - s0;
        const int64_t W = std::min<int64_t>(Pc, (Pc + 2 * (int64_t)H * R + 1) / 2);
        fwA = std::max(fwA, W + 2 * R);
        fwB = std::max(fwB, Pc - W + 2 * (int64_t)(H + 1) * R);
        pmax = std::max(pmax, Pc);
    }
    fwA = (fwA + 1) & ~int64_t(1);
    fwB = (fwB + 1) & ~int64_t(1);
    const size_t smem = (size_t)(2 * fwA + 2 * fwB + (int64_t)H * 4 * R + 8 * 2 * R) * sizeof(double);
    if (smem > 200 * 1024) return STENCIL_EUNSUPPORTED;
    // one communication warp plus compute warps for about one point per thread and step
    const int nthr = pmax > 384 ? 512 : (pmax > 192 ? 288 : 160);
    auto kern = h->arith == ARITH_FMA ? k_jacobi_hex1d<R, ARITH_FMA> : k_jacobi_hex1d<R, ARITH_UNFUSED>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return STENCIL_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nthr, smem) != cudaSuccess) {
        cudaGetLastError();
        return STENCIL_ECUDA;
    }
    if ((int64_t)per_sm * nsm < n) return STENCIL_EUNSUPPORTED;  // every CTA waits on its neighbours
    // workspace: flags (two per period and the abort word), A left bands, B top parts
    const size_t flag_bytes = (size_t)(((2 * n + 1) * sizeof(int) + 255) & ~size_t(255));
    const size_t bytes = flag_bytes + (size_t)n * H * 3 * R * sizeof(double);
    int rc = diamond_workspace(const_cast<stencil_handle_s*>(h), bytes, ctx.st);
    if (rc) return rc;
    HexGeo G;
    G.N = (int)N;
    G.n = (int)n;
    G.H = H;
    G.bc = h->bc;
    G.c = h->c;
    G.T = T;
    G.fwA = (int)fwA;
    G.fwB = (int)fwB;
    G.flagA = (int*)h->dia_ws;
    G.flagB = G.flagA + n;
    G.abort = G.flagA + 2 * n;
    G.aband = (double*)((char*)h->dia_ws + flag_bytes);
    G.btop = G.aband + (size_t)n * H * 2 * R;
    G.status = h->d_status;
    // failure-detection test hook (stencil_debug_inject_stall): consumed by this run
    stencil_handle_s* hm = const_cast<stencil_handle_s*>(h);
    G.spin = hm->debug_spin > 0 ? hm->debug_spin : SPIN_LIMIT_DIAMOND;
    G.stall = hm->debug_stall_tile >= 0 && hm->debug_stall_tile < n ? (int)hm->debug_stall_tile : -1;
    hm->debug_stall_tile = -1;
    hm->debug_spin = 0;
    WArr<2 * R + 1> w;
    for (int q = 0; q < 2 * R + 1; ++q) w.w[q] = h->w_desc[q];
    if (cudaMemsetAsync(h->dia_ws, 0, (2 * n + 1) * sizeof(int), ctx.st) != cudaSuccess) return STENCIL_ECUDA;
    // a cooperative launch: every CTA waits on its neighbours, so all of them must be resident
    // at once even when other streams' kernels share the GPU
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n);
    cfg.blockDim = dim3(nthr);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx.st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, u, G, w) != cudaSuccess) {
        cudaGetLastError();
        return STENCIL_EUNSUPPORTED;  // nothing but the flag reset enqueued: the phase launches run instead
    }
    g_launches++;
    return STENCIL_OK;
}

template <int DIM, int SHAPE, int R>
static int diamond_bands(const RunCtx& ctx, double* u, int64_t T, int H, const int64_t tile[3])
{
    if constexpr (DIM == 1) {
        const int rc = diamond_hex1d<R>(ctx, u, T, H, tile);
        if (rc != STENCIL_EUNSUPPORTED) return rc;
    }
    constexpr int K = Stn<DIM, SHAPE, R>::K;
    WArr<K> w;
    for (int q = 0; q < K; ++q) w.w[q] = ctx.h->w_desc[q];
    DiaGeo G;
    size_t smem = 0, wsd = 0;
    int rc = diamond_geometry(ctx.h, ctx.g, H, tile, G, smem, wsd);
    if (rc) return rc;
    rc = diamond_workspace(ctx.h, wsd * sizeof(double), ctx.st);
    if (rc) return rc;
    double* p = (double*)ctx.h->dia_ws;
    for (int d = 0; d < 3; ++d) {
        if (!G.act[d]) continue;
        G.band[d] = p;
        p += (size_t)G.H * 2 * G.n[d] * 2 * R * G.other[d];
    }
    auto kern = ctx.h->arith == ARITH_FMA ? k_jacobi_diamond<DIM, SHAPE, R, ARITH_FMA>
                                          : k_jacobi_diamond<DIM, SHAPE, R, ARITH_UNFUSED>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return STENCIL_ECUDA;
    const unsigned nblk = (unsigned)((int64_t)G.n[0] * G.n[1] * G.n[2]);
    // threads per tile: one level of a 1D tile is at most fw points, so small
    // CTAs there (more tiles resident per SM, a cheaper barrier per level)
    const int nthr = DIM == 1 ? (G.fw[2] <= 128 ? 128 : 256) : 256;
    // phases: types over the used axes in lexicographic order, A (0) before B (1), slowest axis first
    int phases[8], np = 0;
    for (int m = 0; m < 8; ++m) {
        bool ok = true;
        for (int d = 0; d < 3; ++d)
            if (((m >> (2 - d)) & 1) && !G.act[d]) ok = false;
        if (ok) phases[np++] = m;
    }
    for (int64_t done = 0; done < T;) {
        G.h = (int)std::min<int64_t>(G.H, T - done);
        for (int q = 0; q < np; ++q) {
            kern<<<nblk, nthr, smem, ctx.st>>>(u, G, phases[q], w);
            g_launches++;
            if (cudaGetLastError() != cudaSuccess) return STENCIL_ECUDA;
        }
        done += G.h;
    }
    return STENCIL_OK;
}

int jacobi_diamond_run(const RunCtx& ctx, double* u, int64_t T, int H, const int64_t tile[3])
{
    const stencil_handle_s* h = ctx.h;
#define X(D, S, R) \
    if (h->dim == D && h->shape == S && h->r == R) return diamond_bands<D, S, R>(ctx, u, T, H, tile);
    X(1, STAR, 1) X(1, STAR, 2) X(1, STAR, 3) X(1, STAR, 4)
    X(2, STAR, 1) X(2, BOX, 1) X(2, STAR, 2) X(2, BOX, 2)
    X(3, STAR, 1) X(3, BOX, 1) X(3, STAR, 2)
#undef X
    return STENCIL_EUNSUPPORTED;
}

}  // namespace gbst
