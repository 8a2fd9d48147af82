// Batched execution: many independent stencil problems in one persistent launch.
//
// Each problem is cut into phases of independent units:
//   Jacobi, plain plan    one phase per time step; a unit is a chunk of points
//   Jacobi, blocked plan  one phase per pass of T_b steps; a unit is one
//                         staged tile (tile + T_b*r halo in shared memory,
//                         T_b steps on chip, interior written once)
//   Gauss-Seidel          one phase per (sweep, tile diagonal) of the
//                         parallelogram tiling of the plain sweep kernel; a
//                         unit is one tile (1D: the whole serial sweep)
// A phase may start when every unit of the problem's previous phase has
// finished (a per-problem completion counter). The work list interleaves the
// problems round by round (phase 0 of every problem, then phase 1, ...), so a
// unit only ever waits for units with smaller tickets; one persistent kernel
// walks the list through a ticket counter and every wait is bounded. The
// tiles and depths T_b come from each problem's tuned plan. Gauss-Seidel
// problems whose plan is the wavefront kernel, and stencils with more than
// 125 points, run as their own launches on the same stream. The whole
// enqueue is captured once into a CUDA graph, cached on the batch's shape
// (handles, pointers, extents, step counts, plans) and replayed afterwards.
// Every point is computed with the same descending-order sum and rounding as
// the single-problem kernels, so the results equal separate runs bit for bit.
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
constexpr int JCHUNK = 2048;     // points per plain Jacobi unit
constexpr int BSPIN = 1 << 23;   // bounded waits (x ~0.25 us)

enum { BK_JPLAIN = 0, BK_JBLOCK = 1, BK_GSTILE = 2, BK_GS1D = 3 };

struct BProb {
    int kind, dim, K, r, bc, arith;
    double c;
    const double* w;  // descending canonical order
    const int* off;   // 3 per term, same order
    double* a;        // the grid (result)
    double* b;        // scratch (Jacobi)
    Geo g;
    int64_t T, nph, units;
    // blocked Jacobi
    int B0, B1, B2, h0, h1, h2, E0, E1, E2, tb;
    int64_t nt0, nt1, nt2;
    // Gauss-Seidel tiles
    int gb0, gb1, gbs, cp0, cp1, skew;
    int64_t gnt0, gnt1, gnts, Dn, sweep_units;
    const int64_t* dpre;           // units on diagonals before D (Dn + 1 entries)
    unsigned long long* done;      // completed units
    int* status;
};

__device__ __forceinline__ unsigned long long ld_acq64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int64_t units_of(const BProb& P, int64_t ph)
{
    if (P.kind == BK_GSTILE) {
        const int64_t D = ph % P.Dn;
        return P.dpre[D + 1] - P.dpre[D];
    }
    return P.units;
}

__device__ __forceinline__ int64_t units_before(const BProb& P, int64_t ph)
{
    if (P.kind == BK_GSTILE) return (ph / P.Dn) * P.sweep_units + P.dpre[ph % P.Dn];
    return ph * P.units;
}

// weighted sum with run-time offsets: values v[] already fetched
template <int ARITH>
__device__ __forceinline__ double chain(const double* w, const double* v, int K)
{
    double acc = __dmul_rn(w[0], v[0]);
    for (int q = 1; q < K; ++q) acc = acc_step<ARITH>(acc, w[q], v[q]);
    return acc;
}

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
__device__ double point_lin(const double* u, int64_t p, const long long* lo, const double* sw, int K)
{
    double acc = 0.0;
    for (int q0 = 0; q0 < K; q0 += 8) {
        double v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (q0 + t < K) v[t] = u[p + lo[q0 + t]];
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

template <int ARITH>
__device__ void unit_jplain(const BProb& P, int64_t ph, int64_t unit, const double* sw, const int* so, long long* lo)
{
    const double* src = (ph & 1) ? P.b : P.a;
    double* dst = (ph & 1) ? P.a : P.b;
    const int64_t n12 = P.g.n1 * P.g.n2, npts = P.g.n0 * n12;
    for (int q = threadIdx.x; q < P.K; q += BT) lo[q] = (long long)so[3 * q] * n12 + so[3 * q + 1] * P.g.n2 + so[3 * q + 2];
    __syncthreads();
    const int64_t beg = unit * JCHUNK, end = beg + JCHUNK < npts ? beg + JCHUNK : npts;
    for (int64_t p = beg + threadIdx.x; p < end; p += BT) {
        const int64_t i = p / n12, j = (p / P.g.n2) % P.g.n1, k = p % P.g.n2;
        dst[p] = interior(P, i, j, k) ? point_lin<ARITH>(src, p, lo, sw, P.K) : point_bc<ARITH>(src, i, j, k, P, sw, so);
    }
}

template <int ARITH>
__device__ void unit_jblock(const BProb& P, int64_t ph, int64_t unit, const double* sw, const int* so, long long* lo,
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
    const int64_t st1 = P.E2, st0 = (int64_t)P.E1 * P.E2;
    for (int q = threadIdx.x; q < P.K; q += BT) lo[q] = (long long)so[3 * q] * st0 + so[3 * q + 1] * st1 + so[3 * q + 2];
    for (int64_t idx = threadIdx.x; idx < region; idx += BT) {
        const int64_t i = g0 + idx / st0, j = g1 + (idx / st1) % P.E1, k = g2 + idx % st1;
        const double v = fetch_bc(src, i, j, k, P.g, P.bc, P.c);
        A[idx] = v;
        if (P.bc == BC_CONSTANT && (i < 0 || i >= P.g.n0 || j < 0 || j >= P.g.n1 || k < 0 || k >= P.g.n2)) B[idx] = P.c;
    }
    __syncthreads();
    double* s = A;
    double* d = B;
    for (int st = 1; st <= tb; ++st) {
        const int lo0 = P.dim >= 3 ? st * P.r : 0, hi0 = P.dim >= 3 ? P.E0 - st * P.r : 1;
        const int lo1 = P.dim >= 2 ? st * P.r : 0, hi1 = P.dim >= 2 ? P.E1 - st * P.r : 1;
        const int lo2 = st * P.r, hi2 = P.E2 - st * P.r;
        const int w1 = hi1 - lo1, w2 = hi2 - lo2;
        const int64_t cnt = (int64_t)(hi0 - lo0) * w1 * w2;
        for (int64_t idx = threadIdx.x; idx < cnt; idx += BT) {
            const int s2 = lo2 + (int)(idx % w2), s1 = lo1 + (int)((idx / w2) % w1), s0 = lo0 + (int)(idx / ((int64_t)w2 * w1));
            if (P.bc == BC_CONSTANT) {
                const int64_t i = g0 + s0, j = g1 + s1, k = g2 + s2;
                if (i < 0 || i >= P.g.n0 || j < 0 || j >= P.g.n1 || k < 0 || k >= P.g.n2) continue;
            }
            const int64_t p = s0 * st0 + s1 * st1 + s2;
            d[p] = point_lin<ARITH>(s, p, lo, sw, P.K);
        }
        __syncthreads();
        double* t = s;
        s = d;
        d = t;
    }
    const int64_t cnt = (int64_t)P.B0 * P.B1 * P.B2;
    for (int64_t idx = threadIdx.x; idx < cnt; idx += BT) {
        const int l2 = (int)(idx % P.B2), l1 = (int)((idx / P.B2) % P.B1), l0 = (int)(idx / ((int64_t)P.B2 * P.B1));
        const int64_t i = T0 * P.B0 + l0, j = T1 * P.B1 + l1, k = T2 * P.B2 + l2;
        if (i < P.g.n0 && j < P.g.n1 && k < P.g.n2)
            dst[(i * P.g.n1 + j) * P.g.n2 + k] = s[(l0 + P.h0) * st0 + (l1 + P.h1) * st1 + (l2 + P.h2)];
    }
}

template <int ARITH>
__device__ void unit_gstile(const BProb& P, int64_t ph, int64_t unit, const double* sw, const int* so)
{
    const int64_t D = ph % P.Dn;
    // unit -> (T0, T1) among the tiles with 0 <= D - T0 - T1 < gnts
    int64_t T0 = 0, T1 = 0, rem = unit;
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
    const int64_t TS = D - T0 - T1;
    double* u = P.a;
    const int l1 = threadIdx.x % P.gb1, l0 = threadIdx.x / P.gb1;
    const int64_t i = T0 * P.gb0 + l0;
    const int64_t j = T1 * P.gb1 + l1 - (int64_t)P.skew * i;
    const bool owner = l0 < P.gb0 && i < P.g.n0 && j >= 0 && j < P.g.n1;
    const int64_t kb = TS * P.gbs - (int64_t)P.cp0 * i - (int64_t)P.cp1 * j;
    for (int ls = 0; ls < P.gbs; ++ls) {
        const int64_t k = kb + ls;
        if (owner && k >= 0 && k < P.g.n2) u[(i * P.g.n1 + j) * P.g.n2 + k] = point_bc<ARITH>(u, i, j, k, P, sw, so);
        __syncthreads();
    }
}

template <int ARITH>
__device__ void unit_gs1d(const BProb& P, const double* sw, const int* so)
{
    if (threadIdx.x != 0) return;
    for (int64_t k = 0; k < P.g.n2; ++k) P.a[k] = point_bc<ARITH>(P.a, 0, 0, k, P, sw, so);
}

__global__ void __launch_bounds__(BT) k_batch(const BProb* __restrict__ probs, int np, const int64_t* __restrict__ rpre,
                                             int64_t nrounds, unsigned long long* ticket)
{
    extern __shared__ __align__(16) double bsm[];
    __shared__ long long s_tk;
    __shared__ int s_p;
    __shared__ long long s_ph, s_unit;
    __shared__ double s_w[BMAXK];
    __shared__ int s_off[3 * BMAXK];
    __shared__ long long s_lo[BMAXK];
    const int64_t total = rpre[nrounds];
    for (;;) {
        if (threadIdx.x == 0) {
            s_tk = (long long)atomicAdd(ticket, 1ull);
            if (s_tk < total) {
                int64_t lo = 0, hi = nrounds - 1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) / 2;
                    if (rpre[mid] <= s_tk) lo = mid; else hi = mid - 1;
                }
                int64_t rem = s_tk - rpre[lo];
                int p = 0;
                for (; p < np; ++p) {
                    if (lo >= probs[p].nph) continue;
                    const int64_t u = units_of(probs[p], lo);
                    if (rem < u) break;
                    rem -= u;
                }
                s_p = p;
                s_ph = lo;
                s_unit = rem;
                // wait until the problem's previous phase has finished
                const BProb& P = probs[p];
                const unsigned long long need = (unsigned long long)units_before(P, lo);
                int it = 0;
                while (ld_acq64(P.done) < need && it < BSPIN) {
                    __nanosleep(256);
                    ++it;
                }
                if (it >= BSPIN) atomicExch(P.status, DEV_TIMEOUT);
            }
        }
        __syncthreads();
        if (s_tk >= total) return;
        const BProb& P = probs[s_p];
        for (int q = threadIdx.x; q < P.K; q += BT) {
            s_w[q] = P.w[q];
            s_off[3 * q] = P.off[3 * q];
            s_off[3 * q + 1] = P.off[3 * q + 1];
            s_off[3 * q + 2] = P.off[3 * q + 2];
        }
        __syncthreads();
        const bool fma = P.arith == ARITH_FMA;
        switch (P.kind) {
            case BK_JPLAIN:
                if (fma) unit_jplain<ARITH_FMA>(P, s_ph, s_unit, s_w, s_off, s_lo);
                else unit_jplain<ARITH_UNFUSED>(P, s_ph, s_unit, s_w, s_off, s_lo);
                break;
            case BK_JBLOCK:
                if (fma) unit_jblock<ARITH_FMA>(P, s_ph, s_unit, s_w, s_off, s_lo, bsm);
                else unit_jblock<ARITH_UNFUSED>(P, s_ph, s_unit, s_w, s_off, s_lo, bsm);
                break;
            case BK_GSTILE:
                if (fma) unit_gstile<ARITH_FMA>(P, s_ph, s_unit, s_w, s_off);
                else unit_gstile<ARITH_UNFUSED>(P, s_ph, s_unit, s_w, s_off);
                break;
            default:
                if (fma) unit_gs1d<ARITH_FMA>(P, s_w, s_off);
                else unit_gs1d<ARITH_UNFUSED>(P, s_w, s_off);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(P.done, 1ull);
        }
    }
}

// ------------------------------------------------------------------ host side

// Everything a batch of a given shape needs on the device, prepared once.
struct BatchEntry {
    cudaGraphExec_t exec = nullptr;  // the captured enqueue (absent until first launched outside a capture)
    char* dev = nullptr;             // descriptors, tables, counters, ticket
    size_t off_probs = 0, off_rpre = 0, off_done = 0, total_bytes = 0, off_ticket = 0;
    int np = 0;
    int64_t maxph = 0, nblk = 1;
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

struct Built {
    std::vector<BProb> probs;
    std::vector<std::vector<int64_t>> dpre;  // per problem (GS tiles)
    std::vector<int64_t> rpre;
    size_t smem = 0;
    int64_t nrounds = 0;
};

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
            P.units = (npts + JCHUNK - 1) / JCHUNK;
            P.nph = T;
        }
        return true;
    }
    if (h->dim == 1) {
        P.kind = BK_GS1D;
        P.units = 1;
        P.nph = T;
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
    return true;
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
        const bool wave = h->method == GAUSS_SEIDEL && plans[i].kernel == STENCIL_KERNEL_WAVEFRONT &&
                          gs_wavefront_supported(h, make_geo(h->dim, gs[i].ext));
        if (!wave && h->K <= BMAXK && describe(h, &gs[i], Ts[i], plans[i], P)) {
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
            snprintf(buf, sizeof buf, "%p,%p,%p,%lld,%lld,%lld,%lld,%d,%d,%lld,%lld,%lld;", (void*)hs[i],
                     (void*)gs[i].data, (void*)gs[i].scratch, (long long)gs[i].ext[0], (long long)gs[i].ext[1],
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
            if (cudaMemsetAsync(e.dev + e.off_done, 0, e.total_bytes - e.off_done, s) != cudaSuccess) return STENCIL_ECUDA;
            k_batch<<<(unsigned)e.nblk, BT, e.smem, s>>>((const BProb*)(e.dev + e.off_probs), e.np,
                                                          (const int64_t*)(e.dev + e.off_rpre), e.maxph,
                                                          (unsigned long long*)(e.dev + e.off_ticket));
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
            int rc = gs_wavefront_prepare(h, make_geo(h->dim, gs[i].ext), Ts[i]);
            if (rc) return rc;
        }
    }
    BatchEntry e;
    e.outside = outside;
    // device block: descriptors, GS schedule tables, round prefix, counters, ticket
    const int np = (int)probs.size();
    e.np = np;
    std::vector<std::vector<int64_t>> dpre(np);
    int64_t maxph = 0;
    size_t smem = 0;
    for (int p = 0; p < np; ++p) {
        BProb& P = probs[p];
        if (P.kind == BK_GSTILE) {
            dpre[p].assign((size_t)P.Dn + 1, 0);
            for (int64_t D = 0; D < P.Dn; ++D) dpre[p][(size_t)D + 1] = dpre[p][(size_t)D] + count_gs_units(P, D);
            P.sweep_units = dpre[p][(size_t)P.Dn];
        }
        if (P.kind == BK_JBLOCK) {
            const int64_t region = (int64_t)P.E0 * P.E1 * P.E2;
            const size_t b = (size_t)(((region + 31) & ~int64_t(31)) + region) * 8;
            if (b > smem) smem = b;
        }
        if (P.nph > maxph) maxph = P.nph;
        if ((P.kind == BK_JPLAIN || P.kind == BK_JBLOCK) && (P.nph & 1)) {
            e.copy_dst.push_back(P.a);
            e.copy_src.push_back(P.b);
            e.copy_bytes.push_back((size_t)(P.g.n0 * P.g.n1 * P.g.n2) * sizeof(double));
        }
    }
    std::vector<int64_t> rpre((size_t)maxph + 1, 0);
    for (int64_t r = 0; r < maxph; ++r) {
        int64_t tot = 0;
        for (int p = 0; p < np; ++p) {
            const BProb& P = probs[p];
            if (r >= P.nph) continue;
            tot += P.kind == BK_GSTILE ? dpre[p][(size_t)(r % P.Dn) + 1] - dpre[p][(size_t)(r % P.Dn)] : P.units;
        }
        rpre[(size_t)r + 1] = rpre[(size_t)r] + tot;
    }
    e.off_probs = 0;
    e.off_rpre = ((size_t)np * sizeof(BProb) + 255) & ~size_t(255);
    const size_t off_dpre = e.off_rpre + ((rpre.size() * 8 + 255) & ~size_t(255));
    std::vector<size_t> dpre_off(np, 0);
    size_t cur = off_dpre;
    for (int p = 0; p < np; ++p) {
        dpre_off[p] = cur;
        cur += (dpre[p].size() * 8 + 255) & ~size_t(255);
    }
    e.off_done = cur;
    e.off_ticket = e.off_done + (((size_t)np * 8 + 255) & ~size_t(255));
    e.total_bytes = e.off_ticket + 256;
    e.maxph = maxph;
    e.smem = smem;
    if (np > 0) {
        if (cudaMalloc(&e.dev, e.total_bytes) != cudaSuccess) {
            cudaGetLastError();
            return STENCIL_ENOMEM;
        }
        for (int p = 0; p < np; ++p) {
            probs[p].dpre = probs[p].kind == BK_GSTILE ? (const int64_t*)(e.dev + dpre_off[p]) : nullptr;
            probs[p].done = (unsigned long long*)(e.dev + e.off_done) + p;
        }
        bool ok = cudaMemcpy(e.dev + e.off_probs, probs.data(), (size_t)np * sizeof(BProb), cudaMemcpyHostToDevice) ==
                      cudaSuccess &&
                  cudaMemcpy(e.dev + e.off_rpre, rpre.data(), rpre.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess;
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
        const int64_t total_units = rpre[(size_t)maxph];
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
