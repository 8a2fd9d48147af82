// Batched execution: many independent stencil problems in one persistent launch.
//
// Each problem is cut into phases of independent units:
//   Jacobi, plain plan    one phase per time step; a unit is a slab of rows
//                         (the plain kernel's thread mapping: several points per
//                         thread along the slow axis)
//   Jacobi, blocked plan  one phase per pass of T_b steps; a unit is one
//                         staged tile (tile + T_b*r halo in shared memory,
//                         T_b steps on chip, interior written once)
//   Gauss-Seidel          one phase per (sweep, tile diagonal) of the
//                         parallelogram tiling of the plain sweep kernel; a
//                         unit is one tile (1D: the whole serial sweep)
// A unit of a phase may run once every unit of the problem's previous phase
// has finished (per-problem completion counter). CTAs claim units
// dynamically: each problem hands out its units in order through its own
// ticket counter, and a CTA takes the first unit of the first problem (in
// order of decreasing phase count, so long dependence chains go first) whose
// next phase is open. A unit claimed ahead of its phase waits (bounded) for
// it; the units it waits for were all claimed earlier by running CTAs, so the
// wait always ends. Jacobi and Gauss-Seidel-tile units of the common radius-1
// stencils run the same compile-time specialised code as the single-problem
// kernels; other stencils use run-time offset tables. The tiles and depths
// T_b come from each problem's tuned plan. Gauss-Seidel problems whose plan
// is the wavefront kernel, Jacobi problems whose plan is the streaming blocked
// kernel, and stencils with more than 125 points, run as their own launches
// on the same stream. The whole enqueue is captured once
// into a CUDA graph, cached on the batch's shape (handles, pointers, extents,
// step counts, plans) and replayed afterwards. Every point is computed with
// the same descending-order sum and rounding as the single-problem kernels,
// so the results equal separate runs bit for bit.
#include <algorithm>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "tune.h"

namespace gbst {

namespace {

constexpr int BT = 256;          // threads per batch CTA
constexpr int BMAXK = 125;       // largest stencil the batch kernel takes
constexpr int J1CHUNK = 8192;    // points per 1D Jacobi unit
constexpr int J2ROWS = 4;        // rows per 2D Jacobi unit (one row per unrolled point)
constexpr int J3PLANES = 2;      // planes per 3D Jacobi unit ...
constexpr int J3ROWS = 8;        // ... times rows
constexpr int BSPIN = 1 << 23;   // bounded waits (x ~0.1-0.25 us)

enum { BK_JPLAIN = 0, BK_JBLOCK = 1, BK_GSTILE = 2, BK_GS1D = 3 };
// compile-time specialisations: (dim, shape, r = 1)
enum { SP_NONE = 0, SP_1S = 1, SP_2S = 2, SP_2B = 3, SP_3S = 4, SP_3B = 5 };

struct BProb {
    int kind, spec, dim, K, r, bc, arith;
    double c;
    const double* w;  // descending canonical order
    const int* off;   // 3 per term, same order
    double* a;        // the grid (result)
    double* b;        // scratch (Jacobi)
    Geo g;
    int64_t T, nph, units, total;
    int64_t nj8;      // 3D Jacobi units per plane pair
    // blocked Jacobi
    int B0, B1, B2, h0, h1, h2, E0, E1, E2, tb;
    int64_t nt0, nt1, nt2;
    // Gauss-Seidel tiles
    int gb0, gb1, gbs, cp0, cp1, skew;
    int64_t gnt0, gnt1, gnts, Dn, sweep_units;
    const int64_t* dpre;           // units on diagonals before D (Dn + 1 entries)
    unsigned long long* next;      // units handed out
    unsigned long long* done;      // units completed
    int* status;
};

__device__ __forceinline__ unsigned long long ld_acq64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// phase of unit ticket t, and its index within the phase
__device__ __forceinline__ int64_t phase_of(const BProb& P, int64_t t, int64_t& unit)
{
    if (P.kind == BK_GSTILE) {
        const int64_t sw = t / P.sweep_units, rem = t % P.sweep_units;
        int64_t lo = 0, hi = P.Dn - 1;  // last D with dpre[D] <= rem
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) / 2;
            if (P.dpre[mid] <= rem) lo = mid; else hi = mid - 1;
        }
        unit = rem - P.dpre[lo];
        return sw * P.Dn + lo;
    }
    unit = t % P.units;
    return t / P.units;
}

__device__ __forceinline__ int64_t units_before(const BProb& P, int64_t ph)
{
    if (P.kind == BK_GSTILE) return (ph / P.Dn) * P.sweep_units + P.dpre[ph % P.Dn];
    return ph * P.units;
}

// ---- run-time-offset paths (any stencil up to BMAXK points)

template <int ARITH>
__device__ double point_bc(const double* u, int64_t i, int64_t j, int64_t k, const BProb& P, const double* sw,
                           const int* so)
{
    double acc = 0.0;
    for (int q0 = 0; q0 < P.K; q0 += 8) {
        double v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int q = q0 + t;
            if (q < P.K) v[t] = fetch_bc(u, i + so[3 * q], j + so[3 * q + 1], k + so[3 * q + 2], P.g, P.bc, P.c);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int q = q0 + t;
            if (q < P.K) acc = q == 0 ? __dmul_rn(sw[0], v[0]) : acc_step<ARITH>(acc, sw[q], v[t]);
        }
    }
    return acc;
}

template <int ARITH>
__device__ double point_lin(const double* u, int64_t p, const long long* lo, const double* sw, int K, int64_t n)
{
    double acc = 0.0;
    for (int q0 = 0; q0 < K; q0 += 8) {
        double v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (q0 + t < K) v[t] = ld_in(u, p + lo[q0 + t], n);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int q = q0 + t;
            if (q < K) acc = q == 0 ? __dmul_rn(sw[0], v[0]) : acc_step<ARITH>(acc, sw[q], v[t]);
        }
    }
    return acc;
}

__device__ __forceinline__ bool interior(const BProb& P, int64_t i, int64_t j, int64_t k)
{
    const int r = P.r;
    return (P.dim < 3 || (i >= r && i < P.g.n0 - r)) && (P.dim < 2 || (j >= r && j < P.g.n1 - r)) &&
           (k >= r && k < P.g.n2 - r);
}

// Points of plain Jacobi unit u, visited as (i, j, k) with the same mapping for
// the specialised and the run-time paths: f(i, j, k, linear index).
template <bool UNROLL3 = true, typename F>
__device__ __forceinline__ void for_jacobi_unit(const BProb& P, int64_t u, F f)
{
    const Geo& g = P.g;
    const int tid = threadIdx.x;
    if (P.dim == 1) {
        const int64_t beg = u * J1CHUNK;
#pragma unroll 4
        for (int m = 0; m < J1CHUNK / BT; ++m) {
            const int64_t k = beg + m * BT + tid;
            if (k < g.n2) f(0, 0, k, k);
        }
    } else if (P.dim == 2) {
        const int64_t j0 = u * J2ROWS;
        for (int64_t k = tid; k < g.n2; k += BT)
#pragma unroll
            for (int rb = 0; rb < J2ROWS; ++rb) {
                const int64_t j = j0 + rb;
                if (j < g.n1) f(0, j, k, j * g.n2 + k);
            }
    } else {
        const int64_t i0 = (u / P.nj8) * J3PLANES, j0 = (u % P.nj8) * J3ROWS;
        const int tx = tid % 64, ty = tid / 64;
        for (int jj = ty; jj < J3ROWS; jj += BT / 64) {
            const int64_t j = j0 + jj;
            if (j >= g.n1) break;
            for (int64_t k = tx; k < g.n2; k += 64) {
                if (UNROLL3) {
#pragma unroll
                    for (int rb = 0; rb < J3PLANES; ++rb) {
                        const int64_t i = i0 + rb;
                        if (i < g.n0) f(i, j, k, (i * g.n1 + j) * g.n2 + k);
                    }
                } else {
#pragma unroll 1
                    for (int rb = 0; rb < J3PLANES; ++rb) {
                        const int64_t i = i0 + rb;
                        if (i < g.n0) f(i, j, k, (i * g.n1 + j) * g.n2 + k);
                    }
                }
            }
        }
    }
}

template <int DIM, int SHAPE, int ARITH>
__device__ __noinline__ void unit_jplain_sp(const BProb& P, int64_t ph, int64_t u, const double* sw)
{
    const double* src = (ph & 1) ? P.b : P.a;
    double* dst = (ph & 1) ? P.a : P.b;
    const int64_t s1 = P.g.n2, s0 = P.g.n1 * P.g.n2;
    // a 3D box keeps one point in flight per thread: two would not fit the register budget
    for_jacobi_unit<!(DIM == 3 && SHAPE == BOX)>(P, u, [&](int64_t i, int64_t j, int64_t k, int64_t p) {
        const bool in = (DIM < 3 || (i >= 1 && i < P.g.n0 - 1)) && (DIM < 2 || (j >= 1 && j < P.g.n1 - 1)) &&
                        k >= 1 && k < P.g.n2 - 1;
        st_in(dst, p, P.g.n0 * s0,
              in ? update_interior<DIM, SHAPE, 1, ARITH, false>(src, p, s0, s1, WPtr{sw}, P.g.n0 * s0)
                 : update_bc<DIM, SHAPE, 1, ARITH>(src, i, j, k, P.g, P.bc, P.c, WPtr{sw}));
    });
}

template <int ARITH>
__device__ __noinline__ void unit_jplain_rt(const BProb& P, int64_t ph, int64_t u, const double* sw, const int* so, long long* lo)
{
    const double* src = (ph & 1) ? P.b : P.a;
    double* dst = (ph & 1) ? P.a : P.b;
    const int64_t n12 = P.g.n1 * P.g.n2;
    for (int q = threadIdx.x; q < P.K; q += BT) lo[q] = (long long)so[3 * q] * n12 + so[3 * q + 1] * P.g.n2 + so[3 * q + 2];
    __syncthreads();
    for_jacobi_unit(P, u, [&](int64_t i, int64_t j, int64_t k, int64_t p) {
        const int64_t np = P.g.n0 * n12;
        st_in(dst, p, np,
              interior(P, i, j, k) ? point_lin<ARITH>(src, p, lo, sw, P.K, np) : point_bc<ARITH>(src, i, j, k, P, sw, so));
    });
}

template <int ARITH>
__device__ __noinline__ void unit_jblock(const BProb& P, int64_t ph, int64_t unit, const double* sw, const int* so, long long* lo,
                            double* sm)
{
    const double* src = (ph & 1) ? P.b : P.a;
    double* dst = (ph & 1) ? P.a : P.b;
    const int tb = (int)((P.T - ph * P.tb) < P.tb ? (P.T - ph * P.tb) : P.tb);
    const int64_t T2 = unit % P.nt2, T1 = (unit / P.nt2) % P.nt1, T0 = unit / (P.nt2 * P.nt1);
    const int64_t g0 = T0 * P.B0 - P.h0, g1 = T1 * P.B1 - P.h1, g2 = T2 * P.B2 - P.h2;
    const int64_t region = (int64_t)P.E0 * P.E1 * P.E2;
    double* A = sm;
    double* B = sm + ((region + 31) & ~int64_t(31));
    // checked build: both staged buffers inside the launch's dynamic shared memory (uniform per CTA)
    if (!GBST_IN(((region + 31) & ~int64_t(31)) + region - 1, (int64_t)(dyn_smem_bytes() / 8))) return;
    const int64_t st1 = P.E2, st0 = (int64_t)P.E1 * P.E2;
    for (int q = threadIdx.x; q < P.K; q += BT) lo[q] = (long long)so[3 * q] * st0 + so[3 * q + 1] * st1 + so[3 * q + 2];
    // the staged region fits in shared memory: 32-bit cell indices
    for (int idx = threadIdx.x; idx < (int)region; idx += BT) {
        const int64_t i = g0 + idx / (P.E1 * P.E2), j = g1 + (idx / P.E2) % P.E1, k = g2 + idx % P.E2;
        A[idx] = fetch_bc(src, i, j, k, P.g, P.bc, P.c);
        if (P.bc == BC_CONSTANT && (i < 0 || i >= P.g.n0 || j < 0 || j >= P.g.n1 || k < 0 || k >= P.g.n2)) B[idx] = P.c;
    }
    __syncthreads();
    double* s = A;
    double* d = B;
    for (int st = 1; st <= tb; ++st) {
        const int lo0 = P.dim >= 3 ? st * P.r : 0, hi0 = P.dim >= 3 ? P.E0 - st * P.r : 1;
        const int lo1 = P.dim >= 2 ? st * P.r : 0, hi1 = P.dim >= 2 ? P.E1 - st * P.r : 1;
        const int lo2 = st * P.r, hi2 = P.E2 - st * P.r;
        const int w1 = hi1 - lo1, w2 = hi2 - lo2;  // >= 1: the halo is tb * r wide on every used axis
        auto cell = [&](int s0, int s1, int s2) {
            if (P.bc == BC_CONSTANT) {
                const int64_t i = g0 + s0, j = g1 + s1, k = g2 + s2;
                if (i < 0 || i >= P.g.n0 || j < 0 || j >= P.g.n1 || k < 0 || k >= P.g.n2) return;
            }
            const int64_t p = s0 * st0 + s1 * st1 + s2;
            st_in(d, p, region, point_lin<ARITH>(s, p, lo, sw, P.K, region));
        };
        if (P.dim == 1) {
            for (int s2 = lo2 + (int)threadIdx.x; s2 < hi2; s2 += BT) cell(0, 0, s2);
        } else {
            // each thread advances its (s0, s1, s2) by the digits of BT with carries: no division per cell
            const int cnt = (hi0 - lo0) * w1 * w2;
            const int dr = BT % w2, dq = BT / w2, dq1 = dq % w1, dq0 = dq / w1;
            int s2 = lo2 + (int)threadIdx.x % w2;
            int s1 = lo1 + ((int)threadIdx.x / w2) % w1;
            int s0 = lo0 + (int)threadIdx.x / (w2 * w1);
            for (int idx = threadIdx.x; idx < cnt; idx += BT) {
                cell(s0, s1, s2);
                s2 += dr;
                s1 += dq1;
                s0 += dq0;
                if (s2 >= hi2) {
                    s2 -= w2;
                    ++s1;
                }
                if (s1 >= hi1) {
                    s1 -= w1;
                    ++s0;
                }
            }
        }
        __syncthreads();
        double* t = s;
        s = d;
        d = t;
    }
    const int cnt = P.B0 * P.B1 * P.B2;
    for (int idx = threadIdx.x; idx < cnt; idx += BT) {
        const int l2 = idx % P.B2, l1 = (idx / P.B2) % P.B1, l0 = idx / (P.B2 * P.B1);
        const int64_t i = T0 * P.B0 + l0, j = T1 * P.B1 + l1, k = T2 * P.B2 + l2;
        if (i < P.g.n0 && j < P.g.n1 && k < P.g.n2)
            st_in(dst, (i * P.g.n1 + j) * P.g.n2 + k, P.g.n0 * P.g.n1 * P.g.n2,
                  ld_in(s, (l0 + P.h0) * st0 + (l1 + P.h1) * st1 + (l2 + P.h2), region));
    }
}

// tile (T0, T1, TS) of the problem's parallelogram tiling for diagonal D
__device__ __forceinline__ void gs_tile_of(const BProb& P, int64_t D, int64_t unit, int64_t& T0, int64_t& T1,
                                           int64_t& TS)
{
    T0 = 0;
    T1 = 0;
    int64_t rem = unit;
    for (int64_t t0 = 0; t0 < P.gnt0; ++t0) {
        int64_t lo = D - t0 - P.gnts + 1, hi = D - t0;
        if (lo < 0) lo = 0;
        if (hi > P.gnt1 - 1) hi = P.gnt1 - 1;
        const int64_t cnt = hi >= lo ? hi - lo + 1 : 0;
        if (rem < cnt) {
            T0 = t0;
            T1 = lo + rem;
            break;
        }
        rem -= cnt;
    }
    TS = D - T0 - T1;
}

template <int DIM, int SHAPE, int ARITH, bool SPEC>
__device__ __noinline__ void unit_gstile(const BProb& P, int64_t ph, int64_t unit, const double* sw, const int* so)
{
    int64_t T0, T1, TS;
    gs_tile_of(P, ph % P.Dn, unit, T0, T1, TS);
    double* u = P.a;
    const int l1 = threadIdx.x % P.gb1, l0 = threadIdx.x / P.gb1;
    const int64_t i = T0 * P.gb0 + l0;
    const int64_t j = T1 * P.gb1 + l1 - (int64_t)P.skew * i;
    const bool owner = l0 < P.gb0 && i < P.g.n0 && j >= 0 && j < P.g.n1;
    const int64_t kb = TS * P.gbs - (int64_t)P.cp0 * i - (int64_t)P.cp1 * j;
    const int64_t s1 = P.g.n2, s0 = P.g.n1 * P.g.n2;
    const bool in01 = (DIM < 3 || (i >= 1 && i < P.g.n0 - 1)) && (j >= 1 && j < P.g.n1 - 1);
    for (int ls = 0; ls < P.gbs; ++ls) {
        const int64_t k = kb + ls;
        if (owner && k >= 0 && k < P.g.n2) {
            const int64_t p = i * s0 + j * s1 + k;
            double r;
            if (SPEC)
                r = (in01 && k >= 1 && k < P.g.n2 - 1)
                        ? update_interior<DIM, SHAPE, 1, ARITH, false>(u, p, s0, s1, WPtr{sw}, P.g.n0 * s0)
                        : update_bc<DIM, SHAPE, 1, ARITH>(u, i, j, k, P.g, P.bc, P.c, WPtr{sw});
            else
                r = point_bc<ARITH>(u, i, j, k, P, sw, so);
            st_in(u, p, P.g.n0 * s0, r);
        }
        __syncthreads();
    }
}

template <int ARITH>
__device__ __noinline__ void unit_gs1d(const BProb& P, const double* sw, const int* so)
{
    if (threadIdx.x != 0) return;
    for (int64_t k = 0; k < P.g.n2; ++k) P.a[k] = point_bc<ARITH>(P.a, 0, 0, k, P, sw, so);
}

template <int ARITH>
__device__ void run_unit(const BProb& P, int64_t ph, int64_t u, const double* sw, const int* so, long long* lo,
                         double* dyn)
{
    switch (P.kind) {
        case BK_JPLAIN:
            switch (P.spec) {
                case SP_1S: unit_jplain_sp<1, STAR, ARITH>(P, ph, u, sw); break;
                case SP_2S: unit_jplain_sp<2, STAR, ARITH>(P, ph, u, sw); break;
                case SP_2B: unit_jplain_sp<2, BOX, ARITH>(P, ph, u, sw); break;
                case SP_3S: unit_jplain_sp<3, STAR, ARITH>(P, ph, u, sw); break;
                case SP_3B: unit_jplain_sp<3, BOX, ARITH>(P, ph, u, sw); break;
                default: unit_jplain_rt<ARITH>(P, ph, u, sw, so, lo);
            }
            break;
        case BK_JBLOCK: unit_jblock<ARITH>(P, ph, u, sw, so, lo, dyn); break;
        case BK_GSTILE:
            switch (P.spec) {
                case SP_2S: unit_gstile<2, STAR, ARITH, true>(P, ph, u, sw, so); break;
                case SP_2B: unit_gstile<2, BOX, ARITH, true>(P, ph, u, sw, so); break;
                case SP_3S: unit_gstile<3, STAR, ARITH, true>(P, ph, u, sw, so); break;
                case SP_3B: unit_gstile<3, BOX, ARITH, true>(P, ph, u, sw, so); break;
                default: unit_gstile<3, STAR, ARITH, false>(P, ph, u, sw, so);
            }
            break;
        default: unit_gs1d<ARITH>(P, sw, so);
    }
}

__global__ void __launch_bounds__(BT, 2) k_batch(const BProb* __restrict__ probs, int np, const int* __restrict__ order)
{
    extern __shared__ __align__(16) double bsm[];
    __shared__ __align__(16) BProb sP;
    __shared__ int s_p;
    __shared__ long long s_ph, s_unit;
    __shared__ double s_w[BMAXK];
    __shared__ int s_off[3 * BMAXK];
    __shared__ long long s_lo[BMAXK];
    for (;;) {
        if (threadIdx.x == 0) {
            // claim: the first problem (longest dependence chain first) whose next unit's phase is open
            int p = -1;
            long long tk = 0;
            for (int spin = 0; spin < BSPIN && p < 0; ++spin) {
                bool all_out = true;
                for (int oi = 0; oi < np && p < 0; ++oi) {
                    const BProb& Q = probs[order[oi]];
                    const unsigned long long nx = ld_relaxed64(Q.next);
                    if (nx >= (unsigned long long)Q.total) continue;
                    all_out = false;
                    int64_t uu;
                    const int64_t ph = phase_of(Q, (int64_t)nx, uu);
                    if (ld_relaxed64(Q.done) < (unsigned long long)units_before(Q, ph)) continue;
                    const unsigned long long t = atomicAdd(Q.next, 1ull);
                    if (t >= (unsigned long long)Q.total) continue;
                    p = order[oi];
                    tk = (long long)t;
                }
                if (all_out) break;
                if (p < 0) __nanosleep(spin < 64 ? 32 : 128);
            }
            s_p = p;
            if (p >= 0) {
                const BProb& Q = probs[p];
                int64_t uu;
                const int64_t ph = phase_of(Q, tk, uu);
                s_ph = ph;
                s_unit = uu;
                // a unit claimed ahead of its phase waits for the units claimed before it
                const unsigned long long need = (unsigned long long)units_before(Q, ph);
                int it = 0;
                while (ld_acq64(Q.done) < need && it < BSPIN) {
                    __nanosleep(it < 64 ? 32 : 128);
                    ++it;
                }
                if (it >= BSPIN) atomicExch(Q.status, DEV_TIMEOUT);
                __threadfence();
            }
        }
        __syncthreads();
        if (s_p < 0) return;
        {
            const int* src = (const int*)&probs[s_p];
            int* dst = (int*)&sP;
            for (int q = threadIdx.x; q < (int)(sizeof(BProb) / sizeof(int)); q += BT) dst[q] = src[q];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < sP.K; q += BT) {
            s_w[q] = sP.w[q];
            s_off[3 * q] = sP.off[3 * q];
            s_off[3 * q + 1] = sP.off[3 * q + 1];
            s_off[3 * q + 2] = sP.off[3 * q + 2];
        }
        __syncthreads();
        if (sP.arith == ARITH_FMA)
            run_unit<ARITH_FMA>(sP, s_ph, s_unit, s_w, s_off, s_lo, bsm);
        else
            run_unit<ARITH_UNFUSED>(sP, s_ph, s_unit, s_w, s_off, s_lo, bsm);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(sP.done, 1ull);
        }
    }
}

// ------------------------------------------------------------------ host side

// Everything a batch of a given shape needs on the device, prepared once.
struct BatchEntry {
    cudaGraphExec_t exec = nullptr;  // the captured enqueue (absent until first launched outside a capture)
    char* dev = nullptr;             // descriptors, claim order, GS tables, counters
    size_t off_probs = 0, off_order = 0, off_cnt = 0, total_bytes = 0;
    int np = 0;
    int64_t nblk = 1;
    size_t smem = 0;
    std::vector<double*> copy_dst, copy_src;  // Jacobi results that end in scratch
    std::vector<size_t> copy_bytes;
    std::vector<int> outside;                 // problems run as their own launches
    uint64_t launches = 0;                    // kernels one execution launches
    bool pinned = false;                      // enqueued into a caller's graph: never freed
};

std::mutex g_bmu;
std::map<std::string, BatchEntry> g_batches;
std::list<std::string> g_lru;
constexpr size_t MAX_BATCHES = 32;

int64_t count_gs_units(const BProb& P, int64_t D)
{
    int64_t n = 0;
    for (int64_t t0 = 0; t0 < P.gnt0; ++t0) {
        int64_t lo = D - t0 - P.gnts + 1, hi = D - t0;
        if (lo < 0) lo = 0;
        if (hi > P.gnt1 - 1) hi = P.gnt1 - 1;
        if (hi >= lo) n += hi - lo + 1;
    }
    return n;
}

// Fill the descriptor of problem i (device pointers patched in later).
bool describe(stencil_handle_s* h, const stencil_grid* g, int64_t T, const Plan& pl, BProb& P)
{
    memset(&P, 0, sizeof P);
    P.dim = h->dim;
    P.K = h->K;
    P.r = h->r;
    P.bc = h->bc;
    P.arith = h->arith;
    P.c = h->c;
    P.w = h->d_w;
    P.off = h->d_off;
    P.a = g->data;
    P.b = g->scratch;
    P.g = make_geo(h->dim, g->ext);
    P.T = T;
    P.status = h->d_status;
    const int64_t npts = P.g.n0 * P.g.n1 * P.g.n2;
    if (h->method == JACOBI) {
        if (pl.kernel == STENCIL_KERNEL_BLOCKED) {
            int tb = pl.tb > 0 ? pl.tb : 2;
            int64_t t[3] = {pl.tile[0], pl.tile[1], pl.tile[2]};
            if (h->dim == 1) { t[0] = t[1] = 1; if (t[2] <= 0) t[2] = 256; }
            if (h->dim == 2) { t[0] = 1; if (t[1] <= 0) t[1] = 32; if (t[2] <= 0) t[2] = 64; }
            if (h->dim == 3) { if (t[0] <= 0) t[0] = 8; if (t[1] <= 0) t[1] = 16; if (t[2] <= 0) t[2] = 32; }
            P.kind = BK_JBLOCK;
            P.tb = tb;
            P.B0 = (int)t[0]; P.B1 = (int)t[1]; P.B2 = (int)t[2];
            P.h0 = h->dim >= 3 ? tb * h->r : 0;
            P.h1 = h->dim >= 2 ? tb * h->r : 0;
            P.h2 = tb * h->r;
            P.E0 = P.B0 + 2 * P.h0; P.E1 = P.B1 + 2 * P.h1; P.E2 = P.B2 + 2 * P.h2;
            P.nt0 = (P.g.n0 + P.B0 - 1) / P.B0;
            P.nt1 = (P.g.n1 + P.B1 - 1) / P.B1;
            P.nt2 = (P.g.n2 + P.B2 - 1) / P.B2;
            P.units = P.nt0 * P.nt1 * P.nt2;
            P.nph = (T + tb - 1) / tb;
            const int64_t region = (int64_t)P.E0 * P.E1 * P.E2;
            if ((size_t)(((region + 31) & ~int64_t(31)) + region) * 8 > 200 * 1024) P.kind = BK_JPLAIN;
        }
        if (P.kind != BK_JBLOCK) {
            P.kind = BK_JPLAIN;
            if (h->dim == 1) P.units = (npts + J1CHUNK - 1) / J1CHUNK;
            if (h->dim == 2) P.units = (P.g.n1 + J2ROWS - 1) / J2ROWS;
            if (h->dim == 3) {
                P.nj8 = (P.g.n1 + J3ROWS - 1) / J3ROWS;
                P.units = (P.g.n0 + J3PLANES - 1) / J3PLANES * P.nj8;
            }
            P.nph = T;
        }
        P.total = P.units * P.nph;
        return true;
    }
    if (h->dim == 1) {
        P.kind = BK_GS1D;
        P.units = 1;
        P.nph = T;
        P.total = T;
        return true;
    }
    if (h->bc == BC_PERIODIC && h->shape == BOX) return false;
    const bool box = h->shape == BOX;
    const int R = h->r;
    P.kind = BK_GSTILE;
    P.cp1 = box ? 1 + R : 1;
    P.cp0 = h->dim == 3 ? (box ? 1 + R * (P.cp1 + 1) : 1) : 0;
    P.skew = (h->dim == 3 && box) ? R : 0;
    if (h->dim == 3) { P.gb0 = 16; P.gb1 = 16; P.gbs = 32; }
    else { P.gb0 = 1; P.gb1 = 256; P.gbs = 64; }
    const int64_t thmax = P.cp0 * (P.g.n0 - 1) + P.cp1 * (P.g.n1 - 1) + (P.g.n2 - 1);
    P.gnt0 = (P.g.n0 + P.gb0 - 1) / P.gb0;
    P.gnt1 = (P.g.n1 + P.skew * (P.g.n0 - 1) + P.gb1 - 1) / P.gb1;
    P.gnts = thmax / P.gbs + 1;
    P.Dn = (P.gnt0 - 1) + (P.gnt1 - 1) + (P.gnts - 1) + 1;
    P.nph = T * P.Dn;
    return true;  // total is set once the tile counts per diagonal are known
}

// compile-time specialisation available for (dim, shape, r)
int spec_of(const stencil_handle_s* h)
{
    if (h->r != 1) return SP_NONE;
    if (h->dim == 1) return SP_1S;
    if (h->dim == 2) return h->shape == STAR ? SP_2S : SP_2B;
    return h->shape == STAR ? SP_3S : SP_3B;
}

}  // namespace

int batch_run(const stencil_handle* hs, const stencil_grid* gs, const int64_t* Ts, int n, cudaStream_t st)
{
    // validate, plan (may tune: never inside the capture below)
    std::vector<Plan> plans(n);
    for (int i = 0; i < n; ++i) {
        stencil_handle_s* h = hs[i];
        const stencil_grid* g = &gs[i];
        if (!h || !g->data || Ts[i] < 0) return STENCIL_EINVAL;
        for (int d = 0; d < h->dim; ++d)
            if (g->ext[d] < 1 || (h->bc == BC_PERIODIC && g->ext[d] < 2 * h->r + 1)) return STENCIL_EINVAL;
        if (h->method == JACOBI && (!g->scratch || g->scratch == g->data)) return STENCIL_EINVAL;
        plans[i] = plan_for(h, make_geo(h->dim, g->ext), Ts[i] > 0 ? Ts[i] : 1, st);
    }
    // which problems the persistent kernel takes; the others run as their own launches
    std::vector<int> inside, outside;
    std::vector<BProb> probs;
    for (int i = 0; i < n; ++i) {
        if (Ts[i] == 0) continue;
        stencil_handle_s* h = hs[i];
        BProb P;
        // the time-skewed wavefront (constant boundary) runs as its own launch; periodic Gauss-Seidel
        // cannot overlap its sweeps anyway and stays in the shared kernel as tile units
        const bool wave = h->method == GAUSS_SEIDEL && h->bc == BC_CONSTANT &&
                          plans[i].kernel == STENCIL_KERNEL_WAVEFRONT &&
                          gs_wavefront_supported(h, make_geo(h->dim, gs[i].ext));
        // the streaming blocked Jacobi plan keeps its own kernel (its passes need no workspace, so they
        // are captured with the rest); per-point weights: the problem runs as its own launches (the shared
        // kernel reads constant weights)
        const bool stream = h->method == JACOBI && plans[i].kernel == STENCIL_KERNEL_STREAM &&
                            jacobi_stream_supported(h, make_geo(h->dim, gs[i].ext));
        if (!wave && !stream && !h->field && h->K <= BMAXK && describe(h, &gs[i], Ts[i], plans[i], P)) {
            P.spec = spec_of(h);
            if (P.kind == BK_GSTILE && h->dim == 1) P.spec = SP_NONE;
            inside.push_back(i);
            probs.push_back(P);
        } else {
            outside.push_back(i);
        }
    }
    // graph key: everything the enqueued work depends on
    std::string key;
    {
        char buf[256];
        for (int i = 0; i < n; ++i) {
            snprintf(buf, sizeof buf, "%p,%p,%p,%p,%lld,%lld,%lld,%lld,%d,%d,%lld,%lld,%lld;", (void*)hs[i],
                     (const void*)hs[i]->field, (void*)gs[i].data, (void*)gs[i].scratch, (long long)gs[i].ext[0], (long long)gs[i].ext[1],
                     (long long)gs[i].ext[2], (long long)Ts[i], plans[i].kernel, plans[i].tb,
                     (long long)plans[i].tile[0], (long long)plans[i].tile[1], (long long)plans[i].tile[2]);
            key += buf;
        }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return STENCIL_ECUDA;
    const bool capturing = cs != cudaStreamCaptureStatusNone;

    auto enqueue = [&](const BatchEntry& e, cudaStream_t s) -> int {
        if (e.np > 0) {
            if (cudaMemsetAsync(e.dev + e.off_cnt, 0, e.total_bytes - e.off_cnt, s) != cudaSuccess) return STENCIL_ECUDA;
            k_batch<<<(unsigned)e.nblk, BT, e.smem, s>>>((const BProb*)(e.dev + e.off_probs), e.np,
                                                          (const int*)(e.dev + e.off_order));
            if (cudaGetLastError() != cudaSuccess) return STENCIL_ECUDA;
            for (size_t q = 0; q < e.copy_dst.size(); ++q)
                if (cudaMemcpyAsync(e.copy_dst[q], e.copy_src[q], e.copy_bytes[q], cudaMemcpyDeviceToDevice, s) !=
                    cudaSuccess)
                    return STENCIL_ECUDA;
        }
        for (int i : e.outside) {
            int rc = stencil_run(hs[i], &gs[i], Ts[i], s);
            if (rc) return rc;
        }
        return STENCIL_OK;
    };

    {
        std::lock_guard<std::mutex> lk(g_bmu);
        auto it = g_batches.find(key);
        if (it != g_batches.end()) {
            g_lru.remove(key);
            g_lru.push_front(key);
            BatchEntry& e = it->second;
            if (!capturing && e.exec) {
                g_launches += e.launches;
                return cuda_rc(cudaGraphLaunch(e.exec, st));
            }
            if (capturing) {
                // inside the caller's capture: enqueue the prepared work, allocate nothing
                const uint64_t before = g_launches.load();
                int rc = enqueue(e, st);
                g_launches.store(before + e.launches);
                e.pinned = true;  // the caller's graph refers to this block from now on
                return rc;
            }
        }
    }
    // a batch seen for the first time needs allocations, which a capture forbids
    if (capturing) return STENCIL_EUNSUPPORTED;

    // wavefront workspaces must exist before capture (growing them allocates)
    for (int i : outside) {
        stencil_handle_s* h = hs[i];
        if (h->method == GAUSS_SEIDEL && plans[i].kernel == STENCIL_KERNEL_WAVEFRONT) {
            int rc = gs_wavefront_prepare(h, make_geo(h->dim, gs[i].ext), Ts[i], plans[i].tile);
            if (rc) return rc;
        }
    }
    BatchEntry e;
    e.outside = outside;
    // device block: descriptors, GS schedule tables, round prefix, counters, ticket
    const int np = (int)probs.size();
    e.np = np;
    std::vector<std::vector<int64_t>> dpre(np);
    size_t smem = 0;
    int64_t total_units = 0;
    for (int p = 0; p < np; ++p) {
        BProb& P = probs[p];
        if (P.kind == BK_GSTILE) {
            dpre[p].assign((size_t)P.Dn + 1, 0);
            for (int64_t D = 0; D < P.Dn; ++D) dpre[p][(size_t)D + 1] = dpre[p][(size_t)D] + count_gs_units(P, D);
            P.sweep_units = dpre[p][(size_t)P.Dn];
            P.total = P.sweep_units * P.T;
        }
        if (P.kind == BK_JBLOCK) {
            const int64_t region = (int64_t)P.E0 * P.E1 * P.E2;
            const size_t b = (size_t)(((region + 31) & ~int64_t(31)) + region) * 8;
            if (b > smem) smem = b;
        }
        total_units += P.total;
        if ((P.kind == BK_JPLAIN || P.kind == BK_JBLOCK) && (P.nph & 1)) {
            e.copy_dst.push_back(P.a);
            e.copy_src.push_back(P.b);
            e.copy_bytes.push_back((size_t)(P.g.n0 * P.g.n1 * P.g.n2) * sizeof(double));
        }
    }
    // claim order: longest dependence chain (most phases) first
    std::vector<int> order(np);
    for (int p = 0; p < np; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return probs[x].nph > probs[y].nph; });
    e.off_probs = 0;
    e.off_order = ((size_t)np * sizeof(BProb) + 255) & ~size_t(255);
    const size_t off_dpre = e.off_order + (((size_t)np * sizeof(int) + 255) & ~size_t(255));
    std::vector<size_t> dpre_off(np, 0);
    size_t cur = off_dpre;
    for (int p = 0; p < np; ++p) {
        dpre_off[p] = cur;
        cur += (dpre[p].size() * 8 + 255) & ~size_t(255);
    }
    e.off_cnt = cur;  // per problem: units handed out, units completed
    e.total_bytes = e.off_cnt + (((size_t)np * 16 + 255) & ~size_t(255));
    e.smem = smem;
    if (np > 0) {
        if (cudaMalloc(&e.dev, e.total_bytes) != cudaSuccess) {
            cudaGetLastError();
            return STENCIL_ENOMEM;
        }
        for (int p = 0; p < np; ++p) {
            probs[p].dpre = probs[p].kind == BK_GSTILE ? (const int64_t*)(e.dev + dpre_off[p]) : nullptr;
            probs[p].next = (unsigned long long*)(e.dev + e.off_cnt) + 2 * p;
            probs[p].done = (unsigned long long*)(e.dev + e.off_cnt) + 2 * p + 1;
        }
        bool ok = cudaMemcpy(e.dev + e.off_probs, probs.data(), (size_t)np * sizeof(BProb), cudaMemcpyHostToDevice) ==
                      cudaSuccess &&
                  cudaMemcpy(e.dev + e.off_order, order.data(), (size_t)np * sizeof(int), cudaMemcpyHostToDevice) ==
                      cudaSuccess;
        for (int p = 0; p < np && ok; ++p)
            if (!dpre[p].empty())
                ok = cudaMemcpy(e.dev + dpre_off[p], dpre[p].data(), dpre[p].size() * 8, cudaMemcpyHostToDevice) ==
                     cudaSuccess;
        if (!ok || cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(e.dev);
            return STENCIL_ECUDA;
        }
        int nsm = 0, per_sm = 0, devid = 0;
        cudaGetDevice(&devid);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, devid);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, BT, smem);
        if (per_sm < 1) per_sm = 1;
        e.nblk = (int64_t)nsm * per_sm;
        if (e.nblk > total_units) e.nblk = total_units > 0 ? total_units : 1;
    }

    // capture on a private stream (the caller's may be the legacy default stream,
    // which cannot be captured); the graph is then launched on the caller's stream
    static thread_local cudaStream_t cap = nullptr;
    if (!cap && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(e.dev);
        return STENCIL_ECUDA;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(e.dev);
        return STENCIL_ECUDA;
    }
    const uint64_t before = g_launches.load();
    int rc = enqueue(e, cap);
    cudaError_t ec = cudaStreamEndCapture(cap, &graph);
    if (rc == STENCIL_OK && ec == cudaSuccess) ec = cudaGraphInstantiate(&e.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    // launches recorded into the graph count when the graph runs, not when captured
    e.launches = g_launches.load() - before + (np > 0 ? 1 : 0);
    g_launches.store(before);
    if (rc != STENCIL_OK || ec != cudaSuccess) {
        cudaGetLastError();
        if (e.exec) cudaGraphExecDestroy(e.exec);
        cudaFree(e.dev);
        return rc != STENCIL_OK ? rc : STENCIL_ECUDA;
    }
    cudaGraphExec_t exec = e.exec;
    const uint64_t nl = e.launches;
    {
        std::lock_guard<std::mutex> lk(g_bmu);
        if (g_batches.size() >= MAX_BATCHES) {
            for (auto it = g_lru.rbegin(); it != g_lru.rend(); ++it) {
                BatchEntry& o = g_batches[*it];
                if (o.pinned) continue;
                if (o.exec) cudaGraphExecDestroy(o.exec);
                cudaFree(o.dev);  // waits for the device, so a run still in flight is not cut short
                g_batches.erase(*it);
                g_lru.erase(std::next(it).base());
                break;
            }
        }
        g_batches[key] = std::move(e);
        g_lru.push_front(key);
    }
    g_launches += nl;
    return cuda_rc(cudaGraphLaunch(exec, st));
}

}  // namespace gbst
