// Time-skewed wavefront Gauss-Seidel: the lanes of a warp hold different sweeps.
//
// Temporal vectorization (Section 3.2, Algorithm 3) puts points with different
// time coordinates into one vector: lane k holds sweep t0+k at a spatial
// position s*k behind lane k-1, so one vector operation advances vl sweeps at
// once. It is legal when the stride s exceeds every forward spatial distance
// a dependence covers in one time step (Section 3.2); for the lexicographic
// Gauss-Seidel update of radius r that means s >= r + 1. The same construction
// applies to Gauss-Seidel stencils by taking the newest-value neighbours from
// the output vectors (Section 3.4).
//
// On GB300 the vector is a warp (vl = 32 sweeps):
//
// 1D. Lane k of the warp for sweep block b updates x = n - s*k at step n
//     (s = r + 2, see k_gs1d_wave).
//     After each step it passes its output one lane up with __shfl_up_sync;
//     that value is exactly the newest previous-sweep value lane k+1 needs
//     next (the rotate + blend of Algorithm 3). Lane 0 loads its
//     previous-sweep values from the grid (the "bottom vector") and the last
//     lane stores the block's final sweep (the "top vector"); the sweeps in
//     between never touch memory. Sweep blocks run concurrently, block b+1
//     trailing block b through a progress word.
//
// 2D/3D. As in the paper, temporal vectorization runs along the outermost
//     space loop (Section 3.2, high-dimensional stencils) and the skewed
//     values of the inner loops go through memory. In block-relative skewed
//     coordinates
//         i2 = i + s*k,  j2 = j + a1*i + b1*k,  k2 = k' + a2*i + c2*j + b2*k
//     (k the lane, i j k' the point) every neighbour a point reads as newest
//     (same sweep) and every neighbour it reads as old (previous sweep, lane
//     k-1) has skewed coordinates no larger than the point's own, and
//     everything that will overwrite a value a point reads has larger ones.
//     The skewed space is cut into tiles of H x HJ x W (2D: H x W); within a
//     tile all lanes walk the skewed rows together (one step per row, the
//     lanes independent within a step), each lane updating W points in order
//     along the fast axis. Tiles form a DAG (a tile depends on its three
//     lower neighbours and on a shifted tile of the previous sweep block: the
//     paper's parallelogram tiling for Gauss-Seidel, Section 3.4); a
//     persistent kernel hands out tiles in diagonal order through a ticket
//     counter, and each tile waits (bounded) for its predecessors' flags.
//
// Every point is computed with the same descending-order sum and rounding as
// the plain kernels, so results are bit-identical to T plain sweeps. Periodic
// boundaries chain the end of each sweep to the start of the next and are left
// to the plain kernel.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace gbst {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SPIN_LIMIT = 1 << 23;  // x ~0.25-0.5 us per poll: a wait gives up after two to four seconds

// Bounded-wait settings of one launch: poll limit, and a tile/block whose
// completion is never published (-1: none; used only by failure-detection tests).
struct WaitCfg {
    int spin;
    int64_t stall;
};

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// --------------------------------------------------------------------- 1D ---

constexpr int PROG_SHIFT = 40;
constexpr unsigned long long PROG_MASK = (1ull << PROG_SHIFT) - 1;

// Wait until the previous block has finalised positions [0, need); returns how many it has (a large
// value after a time-out, which is recorded in status). Run by a whole warp: every lane polls and
// lane 0's value is broadcast, so that the warp never splits around the wait.
__device__ __forceinline__ int64_t wait_progress_warp(const unsigned long long* p, int64_t need, unsigned tag,
                                                      int* status, int spin)
{
    for (int it = 0; it < spin; ++it) {
        const unsigned long long v = __shfl_sync(0xffffffffu, ld_acquire64(p), 0);
        if ((unsigned)(v >> PROG_SHIFT) == tag && (int64_t)(v & PROG_MASK) >= need) return (int64_t)(v & PROG_MASK);
        __nanosleep(500);
    }
    if ((threadIdx.x & 31) == 0) atomicExch(status, DEV_TIMEOUT);
    return INT64_MAX;
}

// Lane k holds sweep t0 + k at x = step - S*k with S = R + 2, one more than
// legality needs: the previous-sweep value a lane receives from lane k-1 at a
// step is already the newest one it needs at the NEXT step, so the partial sum
// over the previous-sweep terms (+R .. 0) is formed one step ahead, and only
// the R newest-value terms (-1 .. -R) remain on the step-to-step chain.
template <int R, int ARITH, class WS>
__global__ void __launch_bounds__(32) k_gs1d_wave(double* __restrict__ u, int64_t n, double c, WS w,
                                                  int64_t T, unsigned long long* progress, int* ticket, int* status,
                                                  unsigned tag, WaitCfg wc)
{
    constexpr int S = R + 2;
    const int lane = threadIdx.x;
    int b = 0;
    if (lane == 0) b = atomicAdd(ticket, 1);
    b = __shfl_sync(FULL, b, 0);
    const int64_t nB = (T + 31) / 32;
    if (b >= nB) return;
    const int L = (int)((T - 32 * (int64_t)b) < 32 ? (T - 32 * (int64_t)b) : 32);
    const bool top = lane == L - 1;
    const unsigned long long* prev = b > 0 ? progress + b - 1 : nullptr;
    unsigned long long* mine = progress + b;
    const bool publish = b != wc.stall;
    const unsigned long long mytag = (unsigned long long)tag << PROG_SHIFT;
    int64_t known = b > 0 ? 0 : INT64_MAX;

    // Lane 0's previous-sweep values (the "bottom vector") arrive in chunks of
    // 32 positions, loaded by the whole warp one chunk ahead of use and handed
    // to lane 0 by shuffle, so no load latency sits on the step's critical path.
    auto need_upto = [&](int64_t upto) {
        // positions [0, upto) must be final in the previous block's output
        if (upto > known) known = wait_progress_warp(prev, upto, tag, status, wc.spin);  // the warp as one
    };
    auto load_chunk = [&](int64_t ch) -> double {
        const int64_t p = ch * 32 + lane;
        return (p >= 0 && p < n) ? __ldcg(u + p) : c;
    };
    int64_t cur_ch = 0;
    need_upto(n < 64 ? n : 64);
    double cur = load_chunk(0), nxt = load_chunk(1);

    // ring[o]: previous-sweep value at x + o (o = 0..R) at the start of a step;
    // nw[a]: this sweep's value at x - 1 - a
    double ring[R + 1], nw[R];
#pragma unroll
    for (int o = 0; o <= R; ++o) {
        const double v = __shfl_sync(FULL, cur, o);
        ring[o] = (lane == 0 && o < n) ? v : c;
    }
#pragma unroll
    for (int a = 0; a < R; ++a) nw[a] = c;
    // Weights of point xx (clamped into the grid: a lane outside it computes a
    // value nobody stores). wcur: point x of this step; wnext: point x + 1,
    // loaded a step ahead so that per-point weights add no load latency to
    // the step. Constant weights fold to immediates.
    auto wat = [&](int q, int64_t xx) -> double { return w.at(q, xx < 0 ? 0 : (xx >= n ? n - 1 : xx)); };
    double wcur[2 * R + 1], wnext[2 * R + 1];
#pragma unroll
    for (int q = 0; q <= 2 * R; ++q) wcur[q] = wat(q, -(int64_t)S * lane);
    // descending canonical order: +R .. +1, 0 (previous sweep), then -1 .. -R (this sweep)
    auto partial = [&](const double* wq) -> double {
        double acc = __dmul_rn(wq[0], ring[R]);
#pragma unroll
        for (int q = 1; q <= R; ++q) acc = acc_step<ARITH>(acc, wq[q], ring[R - q]);
        return acc;
    };
    double pc = partial(wcur);
    double out = c;
    const int64_t steps = n + (int64_t)S * (L - 1);
    for (int64_t step = 0; step < steps; ++step) {
        const int64_t x = step - (int64_t)S * lane;
#pragma unroll
        for (int q = 0; q <= 2 * R; ++q) wnext[q] = wat(q, x + 1);
        const int64_t p = step + R + 1;  // newest previous-sweep position lane 0 takes in this step
        if ((p >> 5) != cur_ch) {
            cur_ch = p >> 5;
            cur = nxt;
            const int64_t upto = (cur_ch + 2) * 32;
            need_upto(upto < n ? upto : n);
            nxt = load_chunk(cur_ch + 1);
        }
        const double bottom = __shfl_sync(FULL, cur, (int)(p & 31));
        double recv = __shfl_up_sync(FULL, out, 1);
        if (lane == 0) recv = p < n ? bottom : c;
        double acc = pc;
#pragma unroll
        for (int a = 1; a <= R; ++a) acc = acc_step<ARITH>(acc, wcur[R + a], nw[a - 1]);
        const bool inside = x >= 0 && x < n;
        out = inside ? acc : c;
#pragma unroll
        for (int a = R - 1; a > 0; --a) nw[a] = nw[a - 1];
        nw[0] = out;
#pragma unroll
        for (int o = 0; o < R; ++o) ring[o] = ring[o + 1];
        ring[R] = recv;
        pc = partial(wnext);
#pragma unroll
        for (int q = 0; q <= 2 * R; ++q) wcur[q] = wnext[q];
        if (top) {
            if (inside) u[x] = acc;
            if (publish && (step & 63) == 63 && x >= 0) {
                __threadfence();
                st_release64(mine, mytag | (unsigned long long)(x + 1 < n ? x + 1 : n));
            }
        }
    }
    if (top && publish) {
        __threadfence();
        st_release64(mine, mytag | (unsigned long long)n);
    }
}

// 1D, radius 1, decoupled: one warp issues only the newest-value FMA chain.
//
// Lane k holds sweep t0 + k at x = j - 33k at step j. With that skew, the two
// previous-sweep terms of a point (lane k - 1's outputs at x and x + 1, made
// at steps j - 33 and j - 32) are known two batches of 16 steps before the
// point is due, so they can be summed away from the chain:
//   warps 1-6 (producers) form P = w(+1) u'(x+1) (+) w(0) u'(x) for the next
//             batch of 16 steps, each warp a share of the steps, all 32 lanes
//             (unrolled, so that their sums overlap);
//   warp 0 (the chain) does the 16 dependent updates u(x) = P (+) w(-1) u(x-1)
//             of the current batch from registers;
// one CTA barrier per batch instead of one per step. The chain's outputs go to
// a shared ring of 3 batches (the producers read the two before the current
// one); lane 0's previous-sweep values are the previous block's outputs, which
// warp 7 fetches from the grid two batches ahead with cp.async (a CTA barrier
// waits for a warp's outstanding register loads, not for cp.async), behind the
// same progress words as above, stores the last lane's outputs (the block's
// final sweep) and publishes this block's progress every 4 batches, with the
// fence at the start of the next batch where it overlaps the chain. The sum keeps the
// descending order and rounding of every other kernel.
constexpr int W4_S = 33, W4_D = 16, W4_ROWS = 3 * W4_D;

// Partial sums of steps D0 .. D1 - 1 of batch m for every lane (k = lane), unrolled so that the
// independent sums of the steps overlap. rbm = (16 m) mod 48, the ring row of the batch's first step.
template <int ARITH, int D0, int D1>
__device__ __forceinline__ void w4_produce(int64_t m, int64_t mmax, int rbm, int L, int64_t n, double c,
                                           const WArr<3>& w, const double (*O)[32], double (*Pb)[W4_D][32],
                                           const double* BOT)
{
    if (m > mmax) return;
    const int k = threadIdx.x & 31;
    const int64_t x0 = W4_D * m - (int64_t)W4_S * k;
#pragma unroll
    for (int d = D0; d < D1; ++d) {
        const int64_t x = x0 + d;
        if (k < L && x >= 0 && x < n) {
            double v0, v1;
            if (k == 0) {
                v0 = BOT[x & 63];
                v1 = x + 1 < n ? BOT[(x + 1) & 63] : c;
            } else {
                // lane k - 1's outputs at steps j - 33 and j - 32: ring rows rbm + d - 33 and - 32 (mod 48)
                int r0 = rbm + d + (W4_ROWS - W4_S), r1 = r0 + 1;
                r0 = r0 >= W4_ROWS ? r0 - W4_ROWS : r0;
                r1 = r1 >= W4_ROWS ? r1 - W4_ROWS : r1;
                v0 = O[r0][k - 1];
                v1 = O[r1][k - 1];  // lane k - 1 wrote c there when x + 1 >= n
            }
            Pb[m & 1][d][k] = acc_step<ARITH>(__dmul_rn(w.w[0], v1), w.w[1], v0);
        }
    }
}

// Warp roles: 0 the chain; 1-6 the partial sums (a warp issues at most one FP64
// instruction per ~64 clocks, so the 32 per batch are spread over six warps);
// 7 lane 0's grid values, the block's final sweep to the grid, and progress.
template <int ARITH>
__global__ void __launch_bounds__(256) k_gs1d_wave4(double* __restrict__ u, int64_t n, double c, WArr<3> w, int64_t T,
                                                    unsigned long long* progress, int* ticket, int* status,
                                                    unsigned tag, WaitCfg wc)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ int s_b;
    __shared__ double O[W4_ROWS][32];      // outputs: row = step mod 48, column = lane
    __shared__ double Pb[2][W4_D][32];     // producers' partial sums: batch parity, step in batch, lane
    __shared__ double BOT[64];             // lane 0's previous-sweep values, by position mod 64
    if (threadIdx.x == 0) s_b = atomicAdd(ticket, 1);
    __syncthreads();
    const int b = s_b;
    const int64_t nB = (T + 31) / 32;
    if (b >= nB) return;
    const int L = (int)((T - 32 * (int64_t)b) < 32 ? (T - 32 * (int64_t)b) : 32);
    const unsigned long long* prev = b > 0 ? progress + b - 1 : nullptr;
    unsigned long long* mine = progress + b;
    const bool publish = b != wc.stall;
    const unsigned long long mytag = (unsigned long long)tag << PROG_SHIFT;
    const int64_t jmax = n - 1 + (int64_t)W4_S * (L - 1), mmax = jmax / W4_D;
    int64_t known = b > 0 ? 0 : INT64_MAX;  // warp 7: positions the previous block has finalised

    // warp 7: positions [16m, 16m + 32) of the previous block's output into BOT by cp.async (the
    // CTA barrier does not wait for it, a register load would hold the barrier for an L2 round trip)
    auto bot_fetch = [&](int64_t m) {
        const int64_t lo = W4_D * m;
        if (lo >= n) return;
        const int64_t need = lo + 32 < n ? lo + 32 : n;
        if (need > known) known = wait_progress_warp(prev, need, tag, status, wc.spin);  // warp 7 as one
        const int64_t x = lo + lane;
        double* dst = BOT + (x & 63);
        if (x < n) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                         "l"(u + x)
                         : "memory");
        } else {
            *dst = c;
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto bot_landed = [&]() { asm volatile("cp.async.wait_all;" ::: "memory"); };
    auto produce = [&](int64_t m) {
        const int rbm = (int)((W4_D * m) % W4_ROWS);
        switch (warp) {
            case 1: w4_produce<ARITH, 0, 3>(m, mmax, rbm, L, n, c, w, O, Pb, BOT); break;
            case 2: w4_produce<ARITH, 3, 6>(m, mmax, rbm, L, n, c, w, O, Pb, BOT); break;
            case 3: w4_produce<ARITH, 6, 9>(m, mmax, rbm, L, n, c, w, O, Pb, BOT); break;
            case 4: w4_produce<ARITH, 9, 12>(m, mmax, rbm, L, n, c, w, O, Pb, BOT); break;
            case 5: w4_produce<ARITH, 12, 14>(m, mmax, rbm, L, n, c, w, O, Pb, BOT); break;
            case 6: w4_produce<ARITH, 14, 16>(m, mmax, rbm, L, n, c, w, O, Pb, BOT); break;
            default: break;
        }
    };

    // prologue: the previous block's first 64 positions, the partial sums of batch 0
    if (warp == 7) {
        bot_fetch(0);
        bot_fetch(1);
        bot_landed();
        bot_fetch(2);
    }
    __syncthreads();
    produce(0);
    __syncthreads();

    double nw = c;         // chain: this lane's previous output (the left neighbour of its next point)
    int64_t pending = -1;  // warp 7: progress to publish at the start of the next batch
    for (int64_t m = 0; m <= mmax + 1; ++m) {
        if (warp == 0) {
            if (m <= mmax) {
                const int k = lane;
                double p[W4_D];
#pragma unroll
                for (int d = 0; d < W4_D; ++d) p[d] = Pb[m & 1][d][k];
                const int row0 = (int)((W4_D * m) % W4_ROWS);
                const int64_t x0 = W4_D * m - (int64_t)W4_S * k;
                if (x0 >= 0 && x0 + W4_D <= n) {
                    // the whole batch inside the grid: no predicate on the chain (lanes >= L compute
                    // values nobody reads, so that the warp does not split between the two paths)
                    // outputs kept in the registers of the sums they replace, stored after the chain
#pragma unroll
                    for (int d = 0; d < W4_D; ++d) {
                        nw = acc_step<ARITH>(p[d], w.w[2], nw);
                        p[d] = nw;
                    }
#pragma unroll
                    for (int d = 0; d < W4_D; ++d) O[row0 + d][k] = p[d];
                } else {
#pragma unroll
                    for (int d = 0; d < W4_D; ++d) {
                        const int64_t x = x0 + d;
                        double o = c;
                        if (k < L && x >= 0 && x < n) {
                            o = acc_step<ARITH>(p[d], w.w[2], nw);
                            nw = o;
                        }
                        O[row0 + d][k] = o;
                    }
                }
            }
        } else if (warp < 7) {
            produce(m + 1);
        } else {
            // progress for the final-sweep stores of earlier batches, first: the fence overlaps the chain
            if (pending >= 0) {
                if (lane == 0) {
                    __threadfence();
                    st_release64(mine, mytag | (unsigned long long)pending);
                }
                pending = -1;
            }
            bot_landed();      // batch m + 2's values (read next iteration) are in BOT
            bot_fetch(m + 3);
            if (m >= 1 && m - 1 <= mmax) {
                // the last lane's outputs of batch m - 1 (the block's final sweep) to the grid;
                // this block's progress every 4 batches, released at the start of the next batch
                if (lane < W4_D) {
                    const int64_t j = W4_D * (m - 1) + lane, x = j - (int64_t)W4_S * (L - 1);
                    if (x >= 0 && x < n) u[x] = O[j % W4_ROWS][L - 1];
                }
                if ((m & 3) == 3 && publish) {
                    __syncwarp();
                    const int64_t xl = W4_D * (m - 1) + W4_D - 1 - (int64_t)W4_S * (L - 1);
                    if (xl >= 0) pending = xl + 1 < n ? xl + 1 : n;
                }
            }
        }
        __syncthreads();
    }
    if (warp == 7) bot_landed();         // no copy into shared memory outlives the CTA
    if (threadIdx.x == 224 && publish) {  // warp 7, after its last stores
        __threadfence();
        st_release64(mine, mytag | (unsigned long long)n);
    }
}

// ------------------------------------------------------------------ 2D/3D ---

struct WaveGeo {
    int s, a1, b1, a2, c2, b2;   // skew (see the file comment); 2D uses s, a1, b1
    int H, HJ;                   // tile extents on i2 and (3D) j2; the fast axis extent is the template W
    int64_t nI, nJ, nK, nB;      // tiles per skewed axis, sweep blocks
    int dI, dJ, dK, db;          // shift of the previous-block dependency, block weight of the diagonal index
    int64_t T, ntiles, nD;
};

__device__ __forceinline__ int64_t count2(int64_t m, int64_t nA, int64_t nB)
{
    // #(A, B) in [0,nA) x [0,nB) with A + B = m
    if (m < 0 || m > nA - 1 + nB - 1) return 0;
    const int64_t lo = m - (nB - 1) > 0 ? m - (nB - 1) : 0;
    const int64_t hi = m < nA - 1 ? m : nA - 1;
    return hi - lo + 1;
}

template <int DIM>
__device__ void decode_tile(int64_t tk, const int64_t* __restrict__ pre, const WaveGeo& wg, int64_t& b, int64_t& I,
                            int64_t& J, int64_t& K)
{
    int64_t lo = 0, hi = wg.nD - 1;  // largest d with pre[d] <= tk
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (pre[mid] <= tk) lo = mid; else hi = mid - 1;
    }
    const int64_t d = lo;
    int64_t r = tk - pre[d];
    b = I = J = K = 0;
    for (int64_t bb = 0; bb < wg.nB; ++bb) {
        const int64_t m = d - bb * wg.db;
        if (m < 0) break;
        if (DIM == 2) {
            const int64_t cnt = count2(m, wg.nI, wg.nJ);
            if (r < cnt) {
                b = bb;
                I = (m - (wg.nJ - 1) > 0 ? m - (wg.nJ - 1) : 0) + r;
                J = m - I;
                return;
            }
            r -= cnt;
        } else {
            for (int64_t ii = 0; ii < wg.nI && ii <= m; ++ii) {
                const int64_t cnt = count2(m - ii, wg.nJ, wg.nK);
                if (r < cnt) {
                    b = bb;
                    I = ii;
                    J = ((m - ii) - (wg.nK - 1) > 0 ? (m - ii) - (wg.nK - 1) : 0) + r;
                    K = m - ii - J;
                    return;
                }
                r -= cnt;
            }
        }
    }
}

__device__ __forceinline__ bool wait_flag(const int* f, int tag, int spin)
{
    // poll tightly at first (a predecessor is usually about to finish), then back off
    for (int it = 0; it < spin; ++it) {
        if (ld_acquire(f) == tag) return true;
        __nanosleep(it < 64 ? 32 : 256);
    }
    return false;
}

__device__ __forceinline__ bool wait_flag_ge(const int* f, int tag, int spin)
{
    for (int it = 0; it < spin; ++it) {
        if (ld_acquire(f) >= tag) return true;
        __nanosleep(it < 64 ? 32 : 256);
    }
    return false;
}

// Flag f of a table of n flags; the checked build skips a wait or a release outside the table.
__device__ __forceinline__ bool wait_flag_at(const int* flags, int64_t f, int64_t n, int tag, int spin)
{
    return GBST_IN(f, n) ? wait_flag(flags + f, tag, spin) : true;
}

__device__ __forceinline__ bool wait_flag_ge_at(const int* flags, int64_t f, int64_t n, int tag, int spin)
{
    return GBST_IN(f, n) ? wait_flag_ge(flags + f, tag, spin) : true;
}

__device__ __forceinline__ void release_flag_at(int* flags, int64_t f, int64_t n, int tag)
{
    if (GBST_IN(f, n)) st_release(flags + f, tag);
}

// The same wait run by a whole warp: every lane polls, and lane 0's value is broadcast, so that all
// lanes leave the loop together and the warp never splits around the wait (a warp whose lane 0 alone
// polled while the others waited at a barrier was measured to run its following work several times
// slower).
__device__ __forceinline__ bool wait_flag_ge_warp_at(const int* flags, int64_t f, int64_t n, int tag, int spin)
{
    if (!GBST_IN(f, n)) return true;
    for (int it = 0; it < spin; ++it) {
        if (__shfl_sync(FULL, ld_acquire(flags + f), 0) >= tag) return true;
        __nanosleep(it < 64 ? 32 : 256);
    }
    return false;
}

// Which window cells a point update reads: every cell for a box; for a star
// the centre row in full and the other rows only above/below the points.
template <int SHAPE, int R, int W>
__host__ __device__ constexpr bool needed(int r0, int r1, int cc)
{
    return SHAPE == BOX || (r0 == 0 && r1 == 0) || ((r0 == 0 || r1 == 0) && cc >= R && cc < W + R);
}

// One step of one lane: W points along the fast axis starting at (p0, p1, p2).
// The window of neighbour values is loaded first (nothing this step writes is
// read through it except the same-row left values, which come from regs).
template <int DIM, int SHAPE, int R, int ARITH, int W, class WS>
__device__ __forceinline__ void lane_step(double* __restrict__ u, const Geo& g, double c, const WS& w, int64_t p0,
                                          int64_t p1, int64_t p2)
{
    using St = Stn<DIM, SHAPE, R>;
    constexpr int NR0 = DIM == 3 ? 2 * R + 1 : 1;
    constexpr int NR1 = 2 * R + 1;
    constexpr int NC = W + 2 * R;
    double win[NR0][NR1][NC];
#pragma unroll
    for (int a = 0; a < NR0; ++a)
#pragma unroll
        for (int bq = 0; bq < NR1; ++bq)
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) {
                const int r0 = DIM == 3 ? a - R : 0;
                const int r1 = bq - R;
                if (needed<SHAPE, R, W>(r0, r1, cc)) {
                    const int64_t q0 = p0 + r0, q1 = p1 + r1, q2 = p2 + cc - R;
                    const bool in = q0 >= 0 && q0 < g.n0 && q1 >= 0 && q1 < g.n1 && q2 >= 0 && q2 < g.n2;
                    win[a][bq][cc] = in ? __ldcg(u + (q0 * g.n1 + q1) * g.n2 + q2) : c;
                }
            }
    const int64_t row = (p0 * g.n1 + p1) * g.n2;
#pragma unroll
    for (int m = 0; m < W; ++m) {
        const int64_t q2 = p2 + m;
        const int64_t pw = row + (q2 < 0 ? 0 : (q2 >= g.n2 ? g.n2 - 1 : q2));  // weights' point (clamped)
        double v[St::K];
#pragma unroll
        for (int q = 0; q < St::K; ++q) {
            const int o0 = St::o(q, 0), o1 = St::o(q, 1), o2 = St::o(q, 2);
            v[q] = win[DIM == 3 ? o0 + R : 0][o1 + R][m + o2 + R];
        }
        double acc = __dmul_rn(w.at(0, pw), v[0]);
#pragma unroll
        for (int q = 1; q < St::K; ++q) acc = acc_step<ARITH>(acc, w.at(q, pw), v[q]);
        if (q2 >= 0 && q2 < g.n2) {
            st_in(u, row + q2, g.n0 * g.n1 * g.n2, acc);
            win[DIM == 3 ? R : 0][R][m + R] = acc;  // newest value, read by the next points as a left neighbour
        }
    }
}

template <int DIM, int SHAPE, int R, int ARITH, int W, class WS>
__global__ void __launch_bounds__(128) k_gs_wave(double* __restrict__ u, Geo g, double c, WS w, WaveGeo wg,
                                                 const int64_t* __restrict__ pre, int* __restrict__ flags,
                                                 int* __restrict__ ticket, int* status, int tag, WaitCfg wc)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int64_t tk = 0;
        if (lane == 0) tk = atomicAdd((unsigned long long*)ticket, 1ull);
        tk = __shfl_sync(FULL, tk, 0);
        if (tk >= wg.ntiles) return;
        int64_t b, I, J, K;
        decode_tile<DIM>(tk, pre, wg, b, I, J, K);
        const int64_t fidx = ((b * wg.nI + I) * wg.nJ + J) * wg.nK + K;
        // predecessors: the three lower neighbours in this block, the shifted tile of the previous block
        bool ok = true;
        if (I > 0) ok &= wait_flag_at(flags, fidx - wg.nJ * wg.nK, wg.ntiles, tag, wc.spin);
        if (J > 0) ok &= wait_flag_at(flags, fidx - wg.nK, wg.ntiles, tag, wc.spin);
        if (K > 0) ok &= wait_flag_at(flags, fidx - 1, wg.ntiles, tag, wc.spin);
        if (b > 0) {
            const int64_t pI = I + wg.dI < wg.nI - 1 ? I + wg.dI : wg.nI - 1;
            const int64_t pJ = J + wg.dJ < wg.nJ - 1 ? J + wg.dJ : wg.nJ - 1;
            const int64_t pK = K + wg.dK < wg.nK - 1 ? K + wg.dK : wg.nK - 1;
            ok &= wait_flag_at(flags, (((b - 1) * wg.nI + pI) * wg.nJ + pJ) * wg.nK + pK, wg.ntiles, tag, wc.spin);
        }
        if (!ok && lane == 0) atomicExch(status, DEV_TIMEOUT);
        __syncwarp();
        const int64_t L = wg.T - 32 * b < 32 ? wg.T - 32 * b : 32;
        const bool active = ok && lane < L;
        const int nsteps = DIM == 3 ? wg.H * wg.HJ : wg.H;
        // the points (p0, p1, p2 .. p2 + W - 1) this lane updates at step st; false if none is in the grid
        auto coords = [&](int st, int64_t& p0, int64_t& p1, int64_t& p2) -> bool {
            if (DIM == 2) {
                p0 = 0;
                p1 = I * wg.H + st - (int64_t)wg.s * lane;
                if (p1 < 0 || p1 >= g.n1) return false;
                p2 = J * W - (int64_t)wg.a1 * p1 - (int64_t)wg.b1 * lane;
            } else {
                p0 = I * wg.H + st / wg.HJ - (int64_t)wg.s * lane;
                if (p0 < 0 || p0 >= g.n0) return false;
                p1 = J * wg.HJ + st % wg.HJ - (int64_t)wg.a1 * p0 - (int64_t)wg.b1 * lane;
                if (p1 < 0 || p1 >= g.n1) return false;
                p2 = K * W - (int64_t)wg.a2 * p0 - (int64_t)wg.c2 * p1 - (int64_t)wg.b2 * lane;
            }
            return p2 + W > 0 && p2 < g.n2;
        };
        for (int st = 0; st < nsteps; ++st) {
            if (active) {
                int64_t p0, p1, p2;
                if (coords(st, p0, p1, p2)) lane_step<DIM, SHAPE, R, ARITH, W>(u, g, c, w, p0, p1, p2);
            }
            __syncwarp();
        }
        if (lane == 0 && fidx != wc.stall) {
            __threadfence();
            release_flag_at(flags, fidx, wg.ntiles, tag);
        }
        __syncwarp();
    }
}

// 2D 5-point star (radius 1), constant boundary, one weight per term: the
// decoupled tile. In the one-warp tile above a lane-step of 16 points is 80
// FP64 instructions, and a warp issues at most one per ~64 clocks, so a tile
// on the DAG's critical path takes ~5100 clocks per step even when it has
// the SM's FP64 pipe to itself. Here a CTA works on one tile at a time and
// splits each point's sum, in the same descending order and rounding:
//   producer warps (GD_NP, a share of the 16 points each) form
//     P = w(+1,0) u'(i+1,j) (+) w(0,+1) u'(i,j+1) (+) w(0,0) u'(i,j)
//   from the previous sweep's values for the NEXT step of every lane;
//   the chain warp does u(i,j) = (P (+) w(0,-1) u(i,j-1)) (+) w(-1,0) u(i-1,j),
//   the two newest-value terms, 32 dependent instructions per step;
//   the scheduler warp takes the next tile's ticket, finds the tile and
//   waits for its predecessors while the current tile computes.
// Lanes are GD_S = 3 rows apart (one more than the one-warp tile), so the
// previous-sweep values a producer reads for step st + 1 were written by
// lane k - 1 at steps st - 2 and st - 1, and none of them is overwritten
// before step st + 1: one barrier per step orders the two roles. The newest
// value left of a lane's first point (tile J - 1) and the row above its
// first step (tile I - 1) come from finished tiles; the row above every
// later step is the chain's own output of the step before, kept in registers.
// Measured: bit-exact, and level with the one-warp tile at best (3-4 CTAs per
// SM, 32-row tiles); the per-step barrier is its main stall, with the
// producers' L2 loads behind it. A fixed wavefront plan selects it
// (tile[2] = 1); the one-warp tile stays the default.
constexpr int GD_W = 16;  // points per lane and step
constexpr int GD_S = 3;   // rows between consecutive lanes (sweeps)
constexpr int GD_NP = 4;  // producer warps
constexpr int GD_THREADS = 32 * (GD_NP + 2);

template <int ARITH, int M0, int M1>
__device__ __forceinline__ void gd_produce(const double* __restrict__ u, const Geo& g, double c, const WArr<5>& w,
                                           int64_t q, int64_t p2, double* __restrict__ P)
{
    const int64_t rq = q * g.n2;
    double below[M1 - M0], right[M1 - M0], centre[M1 - M0];
#pragma unroll
    for (int m = M0; m < M1; ++m) {
        const int64_t col = p2 + m;
        const bool in = col >= 0 && col < g.n2;
        below[m - M0] = in && q + 1 < g.n1 ? __ldcg(u + rq + g.n2 + col) : c;
        right[m - M0] = in && col + 1 < g.n2 ? __ldcg(u + rq + col + 1) : c;
        centre[m - M0] = in ? __ldcg(u + rq + col) : c;
    }
#pragma unroll
    for (int m = M0; m < M1; ++m) {
        double acc = __dmul_rn(w.w[0], below[m - M0]);
        acc = acc_step<ARITH>(acc, w.w[1], right[m - M0]);
        P[m] = acc_step<ARITH>(acc, w.w[2], centre[m - M0]);
    }
}

template <int ARITH>
__global__ void __launch_bounds__(GD_THREADS) k_gs2d_dec(double* __restrict__ u, Geo g, double c, WArr<5> w,
                                                         WaveGeo wg, const int64_t* __restrict__ pre,
                                                         int* __restrict__ flags, int* __restrict__ ticket,
                                                         int* status, int tag, WaitCfg wc)
{
    __shared__ double Ps[2][32][GD_W + 1];  // P of a step, per lane (padded: conflict-free lane-strided reads)
    __shared__ double L0s[2][32];           // newest value left of the lane's first point, per step
    __shared__ double A0s[32][GD_W + 1];    // newest row above the tile's first step
    __shared__ long long nxt[4];            // the next tile: ticket, b, I, J
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int NCOMP = 32 * (GD_NP + 1);  // chain + producers: the per-step barrier
    constexpr int SCHED = GD_NP + 1;
    bool ok = true;

    // scheduler: the next tile's ticket and coordinates; returns once its predecessors are done
    auto fetch = [&]() {
        if (lane == 0) {
            const int64_t tk = (int64_t)atomicAdd((unsigned long long*)ticket, 1ull);
            int64_t b = 0, I = 0, J = 0, K = 0;
            if (tk < wg.ntiles) {
                decode_tile<2>(tk, pre, wg, b, I, J, K);
                const int64_t fidx = (b * wg.nI + I) * wg.nJ + J;
                if (I > 0) ok &= wait_flag_at(flags, fidx - wg.nJ, wg.ntiles, tag, wc.spin);
                if (J > 0) ok &= wait_flag_at(flags, fidx - 1, wg.ntiles, tag, wc.spin);
                if (b > 0) {
                    const int64_t pI = I + wg.dI < wg.nI - 1 ? I + wg.dI : wg.nI - 1;
                    const int64_t pJ = J + wg.dJ < wg.nJ - 1 ? J + wg.dJ : wg.nJ - 1;
                    ok &= wait_flag_at(flags, ((b - 1) * wg.nI + pI) * wg.nJ + pJ, wg.ntiles, tag, wc.spin);
                }
            }
            nxt[0] = tk;
            nxt[1] = b;
            nxt[2] = I;
            nxt[3] = J;
        }
        __syncwarp();
    };

    if (warp == SCHED) fetch();
    __syncthreads();
    for (;;) {
        const int64_t tk = nxt[0], b = nxt[1], I = nxt[2], J = nxt[3];
        __syncthreads();  // every warp has the tile before the scheduler overwrites nxt
        if (tk >= wg.ntiles) break;
        if (warp == SCHED) {
            fetch();
        } else {
            const int64_t L = wg.T - 32 * b < 32 ? wg.T - 32 * b : 32;
            const bool lact = lane < L;
            const int64_t p2 = J * GD_W - (int64_t)wg.b1 * lane;  // a1 = 0: the same columns at every step
            const int64_t r0 = I * wg.H - (int64_t)GD_S * lane;   // the lane's row at step 0
            // producers: P of step sn for every lane into slot sn & 1 (and the newest left value;
            // at sn = 0 also the row above)
            auto produce = [&](int sn) {
                const int64_t q = r0 + sn;
                if (!lact || q < 0 || q >= g.n1) return;
                double* P = Ps[sn & 1][lane];
                switch (warp) {
                    case 1: gd_produce<ARITH, 0, 4>(u, g, c, w, q, p2, P); break;
                    case 2: gd_produce<ARITH, 4, 8>(u, g, c, w, q, p2, P); break;
                    case 3: gd_produce<ARITH, 8, 12>(u, g, c, w, q, p2, P); break;
                    default: gd_produce<ARITH, 12, 16>(u, g, c, w, q, p2, P); break;
                }
                if (warp == 1)
                    L0s[sn & 1][lane] = p2 - 1 >= 0 && p2 - 1 < g.n2 ? __ldcg(u + q * g.n2 + p2 - 1) : c;
                if (sn == 0) {
                    const int m0 = (warp - 1) * 4;
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        const int64_t col = p2 + m0 + d;
                        A0s[lane][m0 + d] = q >= 1 && col >= 0 && col < g.n2 ? __ldcg(u + (q - 1) * g.n2 + col) : c;
                    }
                }
            };
            if (warp >= 1) produce(0);
            asm volatile("bar.sync 1, %0;" ::"r"(NCOMP) : "memory");
            double above[GD_W];
#pragma unroll
            for (int m = 0; m < GD_W; ++m) above[m] = c;
            for (int st = 0; st < wg.H; ++st) {
                if (warp == 0) {
                    const int64_t q = r0 + st;
                    if (lact && q >= 0 && q < g.n1) {
                        const double* P = Ps[st & 1][lane];
                        double left = L0s[st & 1][lane];
                        double* row = u + q * g.n2;
#pragma unroll
                        for (int m = 0; m < GD_W; ++m) {
                            const int64_t col = p2 + m;
                            if (col >= 0 && col < g.n2) {
                                const double a = st == 0 ? A0s[lane][m] : (q == 0 ? c : above[m]);
                                const double t = acc_step<ARITH>(P[m], w.w[3], left);
                                const double o = acc_step<ARITH>(t, w.w[4], a);
                                row[col] = o;
                                left = o;
                                above[m] = o;
                            } else {
                                left = c;
                            }
                        }
                    }
                } else if (st + 1 < wg.H) {
                    produce(st + 1);
                }
                asm volatile("bar.sync 1, %0;" ::"r"(NCOMP) : "memory");
            }
            const int64_t fidx = (b * wg.nI + I) * wg.nJ + J;
            if (tid == 0 && fidx != wc.stall) {
                __threadfence();
                release_flag_at(flags, fidx, wg.ntiles, tag);
            }
        }
        __syncthreads();
    }
    if (warp == SCHED && lane == 0 && !ok) atomicExch(status, DEV_TIMEOUT);
}

// Schedule table: pre[d] = number of tiles on diagonals before d (tiles on
// diagonal d: b*db + I + J + K = d). Counts in parallel, prefix sum by one thread.
template <int DIM>
__global__ void k_wave_prefix(WaveGeo wg, int64_t* pre)
{
    for (int64_t d = threadIdx.x; d < wg.nD; d += blockDim.x) {
        int64_t cnt = 0;
        for (int64_t b = 0; b < wg.nB; ++b) {
            const int64_t m = d - b * wg.db;
            if (m < 0) break;
            if (DIM == 2) {
                cnt += count2(m, wg.nI, wg.nJ);
            } else {
                for (int64_t ii = 0; ii < wg.nI && ii <= m; ++ii) cnt += count2(m - ii, wg.nJ, wg.nK);
            }
        }
        pre[d + 1] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        pre[0] = 0;
        for (int64_t d = 0; d < wg.nD; ++d) pre[d + 1] += pre[d];
    }
}

// ------------------------------------------------------- 2D: rows as lanes ---
//
// The same hyperplane order with the roles of the loops exchanged: the lanes
// of a warp hold 32 consecutive rows of ONE sweep, and the sweeps are
// pipelined across warps. At step t, lane k updates the four columns of group
// G = t - SK k (columns 4G .. 4G + 3) of row 32b + k, left to right; lane
// k - 1 produced the newest values above them (and, for a box, the columns
// on either side) SK to SK + 1 steps before and hands them over by shuffle,
// and lane k + 1, which trails by SK groups, has not yet overwritten the old
// values below them and hands those over too from the groups it holds ahead
// of use. SK = 1 for the star, 2 for the box (whose above-right neighbour is
// one group further on). A lane's only memory traffic is its own row: one
// group of four columns loaded (one 32-byte sector, through L2) and one stored
// per step, so every sector a warp instruction touches is used whole. Lane 0
// reads the newest values of the row above the band from the band above,
// lane 31 the old values of the row below it from the band below in the
// previous sweep.
//
// A task (s, b) is sweep s over band b. It waits (bounded) for the progress
// words of (s, b - 1) (the row above, this sweep), (s - 1, b) (its own rows,
// previous sweep) and (s - 1, b + 1) (the row below, previous sweep), once
// per chunk of CH steps, for exactly the groups the chunk reads, and
// publishes its own steps after each chunk. In-place updates are safe: a
// value is overwritten only by a task that has waited for every reader of the
// older value (the readers are the tasks it waits for, directly or through
// them). Tasks are handed out in the order (s + b, s), in which every task a
// task waits for comes earlier, so a persistent kernel whose warps claim
// tasks from a ticket counter cannot deadlock. The sweeps need no blocking,
// so no lane idles on a partial block of sweeps; the sum keeps the
// descending order and rounding of every other kernel. Rows of a multiple of
// four columns only (whole 32-byte-aligned groups).
constexpr int GR_CHUNK = 8;    // default steps between progress waits and publications (CH)
constexpr int GR_THREADS = 128;
constexpr int GR_PSTRIDE = 32;  // ints between two tasks' progress words: one 128-byte line each

struct RowGeo {
    int64_t n0, n1;   // rows, columns (a multiple of 4)
    int64_t nb;       // bands of 32 rows
    int64_t T;        // sweeps of this launch
    int64_t ntasks;   // T * nb
    int64_t steps;    // steps of a task: n1 / 4 + 31 SK, rounded up to the chunk
};

// The task of ticket tk in the order (s + b, s): (e, pe) is the caller's cursor (anti-diagonal e,
// pe tickets before it); tickets only grow, so the cursor only moves forward.
__device__ __forceinline__ void rows_decode(int64_t tk, const RowGeo& g, int64_t& e, int64_t& pe, int64_t& s,
                                            int64_t& b)
{
    for (;;) {
        const int64_t lo = e - g.nb + 1 > 0 ? e - g.nb + 1 : 0;
        const int64_t hi = e < g.T - 1 ? e : g.T - 1;
        const int64_t cnt = hi - lo + 1;
        if (tk < pe + cnt) {
            s = lo + (tk - pe);
            b = e - s;
            return;
        }
        pe += cnt;
        ++e;
    }
}

// Wait until *p >= need (all lanes of the warp); known caches the last value seen. False after a
// time-out. The
// sleep between polls follows the distance still to go (about 0.25 us per missing step, 64 ns to
// 4 us): a producer a step or two short is seen soon after it publishes, while the thousands of
// warps whose producers are far behind poll rarely and leave the L2 slices alone.
__device__ __forceinline__ bool rows_wait(const int* p, int need, int& known, int spin)
{
    if (known >= need) return true;
    for (int it = 0; it < spin; ++it) {
        known = __shfl_sync(FULL, ld_acquire(p), 0);  // lane 0's value: the loop stays uniform
        if (known >= need) return true;
        const int gap = need - known;
        __nanosleep(gap < 1 ? 64u : (gap > 16 ? 4096u : 256u * (unsigned)gap));
    }
    return false;
}

// Four consecutive doubles (a 32-byte-aligned group, one sector) of a row through L2, or four times
// c where ok is false. Every lane loads (the group index clamped into the row), so that no lane's
// predicate splits the warp; the value is then selected. Groups move as whole sectors (256-bit
// accesses): a sector written in two halves by separate stores was measured to make its later
// reads several times slower.
struct Q4 {
    double v[4];
};

__device__ __forceinline__ Q4 ld_group(const double* rowp, int grp, int ng, bool ok, double c)
{
    const int gc = grp < 0 ? 0 : (grp >= ng ? ng - 1 : grp);
    const double* p = rowp + 4 * (int64_t)gc;
    double a, b2, e, d;
    asm volatile("ld.global.cg.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(a), "=d"(b2), "=d"(e), "=d"(d) : "l"(p) : "memory");
    Q4 q;
    q.v[0] = ok ? a : c;
    q.v[1] = ok ? b2 : c;
    q.v[2] = ok ? e : c;
    q.v[3] = ok ? d : c;
    return q;
}

__device__ __forceinline__ void st_group(double* p, const Q4& q)
{
    asm volatile("st.global.cg.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(q.v[0]), "d"(q.v[1]), "d"(q.v[2]),
                 "d"(q.v[3])
                 : "memory");
}

__device__ __forceinline__ Q4 shfl_down4(const Q4& q, int d = 1)
{
    Q4 r;
#pragma unroll
    for (int e = 0; e < 4; ++e) r.v[e] = __shfl_down_sync(FULL, q.v[e], d);
    return r;
}

__device__ __forceinline__ Q4 shfl_up4(const Q4& q, int d = 1)
{
    Q4 r;
#pragma unroll
    for (int e = 0; e < 4; ++e) r.v[e] = __shfl_up_sync(FULL, q.v[e], d);
    return r;
}

// FIELD: per-point weights (the 5-point star only), fld holding the 5 planes of n0 x n1 weights in
// canonical term order; each lane loads its own row's weights a step ahead of use.
// R = 2: the 9-point star of radius 2; lanes 0 and 31 then hold a second row beyond the band (RY),
// and lanes 1 and 30 take their outer neighbour row from lane 0's and lane 31's first ring.
template <int SHAPE, int ARITH, int CH, bool FIELD = false, int R = 1>
__global__ void __launch_bounds__(GR_THREADS, (FIELD || R == 2) ? 2 : 3) k_gs2d_rows(double* __restrict__ u, RowGeo g, double c,
                                                          WArr<Stn<2, SHAPE, R>::K> w, int* __restrict__ prog,
                                                          int* __restrict__ ticket, int* status, WaitCfg wc,
                                                          const double* __restrict__ fld = nullptr)
{
    static_assert(!FIELD || (SHAPE == STAR && R == 1), "per-point weights: the 5-point star only");
    static_assert(R == 1 || (SHAPE == STAR && !FIELD), "radius 2: the star with one weight per term");
    constexpr int SK = SHAPE == STAR ? 1 : 2;   // groups lane k trails lane k - 1
    constexpr int QX0 = (SHAPE == STAR && R == 1) ? 0 : -1;  // first group of the x-row rings, relative to G
    constexpr int LX = QX0 + 4;                  // group the x-row ring loads at a step, relative to G
    const int lane = threadIdx.x & 31;
    const int64_t nprog = g.T * g.nb;  // progress words (bounds of the checked build)
    (void)nprog;
    const int ng = (int)(g.n1 / 4);
    const int smax = ng + 31 * SK;  // steps after which every lane has finished its row
    const int steps = (int)g.steps;
    int64_t e = 0, pe = 0;
    bool timed_out = false;  // after a time-out this warp stops waiting (its results are void anyway)
    for (;;) {
        int64_t tk = 0;
        if (lane == 0) tk = (int64_t)atomicAdd((unsigned long long*)ticket, 1ull);
        tk = __shfl_sync(FULL, tk, 0);
        if (tk >= g.ntasks) break;
        int64_t s = 0, b = 0;
        if (lane == 0) rows_decode(tk, g, e, pe, s, b);
        s = __shfl_sync(FULL, s, 0);
        b = __shfl_sync(FULL, b, 0);
        const bool publish = tk != wc.stall;
        const int64_t i = b * 32 + lane;
        const bool row_ok = i < g.n0;
        double* const row = u + (row_ok ? i : 0) * g.n1;
        // lane 0: the row above the band (this sweep); lane 31: the row below it (previous sweep)
        const int64_t ix = lane == 0 ? b * 32 - 1 : b * 32 + 32;
        const bool x_ok = (lane == 0 || lane == 31) && ix >= 0 && ix < g.n0;
        const double* xrow = x_ok ? u + ix * g.n1 : row;  // other lanes load (and drop) their own row
        // R = 2: lane 0's second row above (32 b - 2), lane 31's second row below (32 b + 33)
        const int64_t iy = lane == 0 ? b * 32 - 2 : b * 32 + 33;
        const bool y_ok = R == 2 && (lane == 0 || lane == 31) && iy >= 0 && iy < g.n0;
        const double* yrow = y_ok ? u + iy * g.n1 : row;
        const int64_t f = s * g.nb + b;
        const int64_t fA = f - 1, fO = f - g.nb, fB = f - g.nb + 1;  // above / own / below predecessors
        const bool hasA = b > 0, hasO = s > 0, hasB = s > 0 && b + 1 < g.nb;
        int kA = 0, kO = 0, kB = 0;
        // grid values written by other SMs are read through L2 (ld.global.cg), never from a stale L1 line
        auto ld_row = [&](int grp) -> Q4 {
            return ld_group(row, grp, ng, row_ok && (unsigned)grp < (unsigned)ng && GBST_IN(grp, ng), c);
        };
        auto ld_x = [&](int grp) -> Q4 {
            return ld_group(xrow, grp, ng, x_ok && (unsigned)grp < (unsigned)ng && GBST_IN(grp, ng), c);
        };
        auto ld_y = [&](int grp) -> Q4 {
            return ld_group(yrow, grp, ng, y_ok && (unsigned)grp < (unsigned)ng && GBST_IN(grp, ng), c);
        };
        // RO[(m + q) & 3]: old values of this lane's row, group G + q (q = 0..3), G the group of step m;
        // RX[(m + q) & 3]: lane 0 the newest row above, lane 31 the old row below, group G + q
        //                  (q = QX0 .. QX0 + 3);
        // O[m & 3]: this lane's outputs of step m (c outside the grid)
        Q4 RO[4], RX[4], O[4], RY[R == 2 ? 4 : 1];
#pragma unroll
        for (int q = 0; q < 4; ++q) O[q].v[0] = O[q].v[1] = O[q].v[2] = O[q].v[3] = c;
        // FIELD: WR[m & 1][q] the weights of term q (summation order) at group G of step m
        Q4 WR[FIELD ? 2 : 1][FIELD ? 5 : 1];
        const int64_t fpl = g.n0 * g.n1;  // points per weight plane
        auto ld_w = [&](int grp, Q4* dst) {
            if constexpr (FIELD) {
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    dst[q] = ld_group(fld + (int64_t)(4 - q) * fpl + (row - u), grp, ng,
                                      row_ok && (unsigned)grp < (unsigned)ng && GBST_IN(grp, ng), 0.0);
            }
        };
        for (int t0 = 0; t0 < steps; t0 += CH) {
            // every lane polls (one warp-wide load of one word, the same value to all lanes), so that
            // the warp never splits around the wait; timed_out stays uniform
            if (!timed_out) {
                bool ok = true;
                const int nA = t0 + CH + LX + 31 * SK, nO = t0 + CH + 4, nB = t0 + CH - 31 * SK + LX + (R - 1);
                if (hasA && GBST_IN(fA, nprog))
                    ok &= rows_wait(prog + fA * GR_PSTRIDE, nA < smax ? nA : smax, kA, wc.spin);
                if (ok && hasO && GBST_IN(fO, nprog))
                    ok &= rows_wait(prog + fO * GR_PSTRIDE, nO < smax ? nO : smax, kO, wc.spin);
                if (ok && hasB && nB > 0 && GBST_IN(fB, nprog))
                    ok &= rows_wait(prog + fB * GR_PSTRIDE, nB < smax ? nB : smax, kB, wc.spin);
                ok = __all_sync(FULL, ok);
                if (!ok) {
                    if (lane == 0) atomicExch(status, DEV_TIMEOUT);
                    timed_out = true;
                }
            }
            __syncwarp();
            if (t0 == 0) {
                const int G0 = -SK * lane;
#pragma unroll
                for (int q = 0; q < 4; ++q) RO[q] = ld_row(G0 + q);
#pragma unroll
                for (int q = QX0; q < QX0 + 4; ++q) RX[q & 3] = ld_x(G0 + q);
                if constexpr (R == 2) {
#pragma unroll
                    for (int q = QX0; q < QX0 + 4; ++q) RY[q & 3] = ld_y(G0 + q);
                }
                ld_w(G0, WR[0]);
            }
            for (int tg = t0; tg < t0 + CH; tg += 4) {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int G = tg + m - SK * lane;
                    Q4 out;
                    if constexpr (R == 2) {
                        // below: rows i + 1 (lane k + 1's q = 1) and i + 2 (lane k + 2's q = 2); above: lane
                        // k - 1's output of step m - 1 and lane k - 2's of step m - 2 (both group G). Beyond
                        // the band: lane 31 takes rows 32 b + 32 / 33 from its rings (q = 0), lane 30 the
                        // first of them from lane 31's (its q = +1); lane 0 takes rows 32 b - 1 / - 2 from its
                        // rings, lane 1 the first from lane 0's (its q = -1)
                        Q4 b1 = shfl_down4(RO[(m + 1) & 3]);
                        Q4 b2 = shfl_down4(RO[(m + 2) & 3], 2);
                        const Q4 x31 = shfl_down4(RX[(m + 1) & 3]);
                        Q4 a1 = shfl_up4(O[(m + 3) & 3]);
                        Q4 a2 = shfl_up4(O[(m + 2) & 3], 2);
                        const Q4 x0 = shfl_up4(RX[(m + 3) & 3]);
                        if (lane == 30) b2 = x31;
                        if (lane == 31) {
                            b1 = RX[m & 3];
                            b2 = RY[m & 3];
                        }
                        if (lane == 1) a2 = x0;
                        if (lane == 0) {
                            a1 = RX[m & 3];
                            a2 = RY[m & 3];
                        }
                        double l1 = O[(m + 3) & 3].v[3], l2 = O[(m + 3) & 3].v[2];
#pragma unroll
                        for (int x = 0; x < 4; ++x) {
                            // (+2,0) (+1,0) (0,+2) (0,+1) (0,0) (0,-1) (0,-2) (-1,0) (-2,0)
                            const double r1 = x < 3 ? RO[m & 3].v[x + 1] : RO[(m + 1) & 3].v[0];
                            const double r2 = x < 2 ? RO[m & 3].v[x + 2] : RO[(m + 1) & 3].v[x - 2];
                            double acc = __dmul_rn(w.w[0], b2.v[x]);
                            acc = acc_step<ARITH>(acc, w.w[1], b1.v[x]);
                            acc = acc_step<ARITH>(acc, w.w[2], r2);
                            acc = acc_step<ARITH>(acc, w.w[3], r1);
                            acc = acc_step<ARITH>(acc, w.w[4], RO[m & 3].v[x]);
                            acc = acc_step<ARITH>(acc, w.w[5], l1);
                            acc = acc_step<ARITH>(acc, w.w[6], l2);
                            acc = acc_step<ARITH>(acc, w.w[7], a1.v[x]);
                            acc = acc_step<ARITH>(acc, w.w[8], a2.v[x]);
                            out.v[x] = acc;
                            l2 = l1;
                            l1 = acc;
                        }
                    } else if (SHAPE == STAR) {
                        // below: lane k + 1's own-row group G (its q = 1); above: lane k - 1's outputs of
                        // step m - 1 (its group then was G); lanes 31 and 0 take the x row's group G
                        Q4 bel = shfl_down4(RO[(m + 1) & 3]);
                        Q4 abv = shfl_up4(O[(m + 3) & 3]);
                        if (lane == 31) bel = RX[m & 3];
                        if (lane == 0) abv = RX[m & 3];
                        double left = O[(m + 3) & 3].v[3];
                        if constexpr (FIELD) ld_w(tg + m - SK * lane + 1, WR[(m + 1) & 1]);  // next step's
#pragma unroll
                        for (int x = 0; x < 4; ++x) {
                            // (+1,0) (0,+1) (0,0) (0,-1) (-1,0)
                            auto wt = [&](int q) -> double {
                                if constexpr (FIELD) return WR[m & 1][q].v[x];
                                return w.w[q];
                            };
                            const double rgt = x < 3 ? RO[m & 3].v[x + 1] : RO[(m + 1) & 3].v[0];
                            double acc = __dmul_rn(wt(0), bel.v[x]);
                            acc = acc_step<ARITH>(acc, wt(1), rgt);
                            acc = acc_step<ARITH>(acc, wt(2), RO[m & 3].v[x]);
                            acc = acc_step<ARITH>(acc, wt(3), left);
                            acc = acc_step<ARITH>(acc, wt(4), abv.v[x]);
                            out.v[x] = acc;
                            left = acc;
                        }
                    } else {
                        // bv[x + 1], av[x + 1]: old row below, newest row above, at column 4G + x
                        // (x = -1..4); lane k + 1 holds groups G - 1 .. G + 1 as its q = 1..3, lane k - 1
                        // produced them at steps m - 3 .. m - 1
                        double bv[6], av[6];
                        {
                            const Q4 bc = shfl_down4(RO[(m + 2) & 3]);
                            const Q4 ac = shfl_up4(O[(m + 2) & 3]);
                            bv[0] = __shfl_down_sync(FULL, RO[(m + 1) & 3].v[3], 1);
                            bv[5] = __shfl_down_sync(FULL, RO[(m + 3) & 3].v[0], 1);
                            av[0] = __shfl_up_sync(FULL, O[(m + 1) & 3].v[3], 1);
                            av[5] = __shfl_up_sync(FULL, O[(m + 3) & 3].v[0], 1);
#pragma unroll
                            for (int x = 0; x < 4; ++x) {
                                bv[x + 1] = bc.v[x];
                                av[x + 1] = ac.v[x];
                            }
                        }
                        if (lane == 31) {
                            bv[0] = RX[(m + 3) & 3].v[3];
                            bv[5] = RX[(m + 1) & 3].v[0];
#pragma unroll
                            for (int x = 0; x < 4; ++x) bv[x + 1] = RX[m & 3].v[x];
                        }
                        if (lane == 0) {
                            av[0] = RX[(m + 3) & 3].v[3];
                            av[5] = RX[(m + 1) & 3].v[0];
#pragma unroll
                            for (int x = 0; x < 4; ++x) av[x + 1] = RX[m & 3].v[x];
                        }
                        double left = O[(m + 3) & 3].v[3];
#pragma unroll
                        for (int x = 0; x < 4; ++x) {
                            // (+1,+1) (+1,0) (+1,-1) (0,+1) (0,0) (0,-1) (-1,+1) (-1,0) (-1,-1)
                            const double rgt = x < 3 ? RO[m & 3].v[x + 1] : RO[(m + 1) & 3].v[0];
                            double acc = __dmul_rn(w.w[0], bv[x + 2]);
                            acc = acc_step<ARITH>(acc, w.w[1], bv[x + 1]);
                            acc = acc_step<ARITH>(acc, w.w[2], bv[x]);
                            acc = acc_step<ARITH>(acc, w.w[3], rgt);
                            acc = acc_step<ARITH>(acc, w.w[4], RO[m & 3].v[x]);
                            acc = acc_step<ARITH>(acc, w.w[5], left);
                            acc = acc_step<ARITH>(acc, w.w[6], av[x + 2]);
                            acc = acc_step<ARITH>(acc, w.w[7], av[x + 1]);
                            acc = acc_step<ARITH>(acc, w.w[8], av[x]);
                            out.v[x] = acc;
                            left = acc;
                        }
                    }
                    const bool gin = (unsigned)G < (unsigned)ng;
#pragma unroll
                    for (int x = 0; x < 4; ++x) out.v[x] = gin ? out.v[x] : c;
                    O[m & 3] = out;
                    if (gin && row_ok && GBST_IN(G, ng)) st_group(row + 4 * (int64_t)G, out);
                    RO[m & 3] = ld_row(G + 4);
                    RX[(m + QX0) & 3] = ld_x(G + LX);
                    if constexpr (R == 2) RY[(m + QX0) & 3] = ld_y(G + LX);
                }
            }
            __syncwarp();
            if (lane == 0 && publish && GBST_IN(f, nprog)) {
                __threadfence();
                st_release(prog + f * GR_PSTRIDE, t0 + CH);
            }
        }
    }
}

// ---------------------------------------------------- periodic: in-sweep DAG ---
//
// With a periodic boundary, sweep t+1 reads (through the wrap) values sweep t
// writes last, so sweeps cannot overlap (no time skew is legal). Inside a
// sweep the parallelogram tiling of the plain kernel still applies: in
// (i, sigma, theta) coordinates every newest-value dependence points to a
// tile with all coordinates <= (and not all equal), every old-value read to
// one with all coordinates >=. Instead of one launch per tile diagonal, one
// persistent launch runs all T sweeps: tiles are handed out in (sweep,
// diagonal) order, each waits (bounded) for its three lower neighbours of the
// same sweep and for every tile of the previous sweep, computes its points in
// theta order (one CTA barrier per theta), and publishes its flag. A tile of sweep s waits only for
// the tiles of sweep s - 1 it depends on (sweep_dag_prev_waits), so about three sweeps can be in
// flight at once: the wrap makes a sweep's first points depend on the previous sweep's last
// hyperplanes of each axis, a lag of about one extent per axis, not a whole sweep.

struct SweepDag {
    int b0, b1, bs, cp0, cp1, skew;   // tile extents in (i, sigma, theta), hyperplane weights, sigma skew
    int64_t nt0, nt1, nts, Dn, sweep_units, T;
};

__device__ __forceinline__ int64_t count_tiles_on(const SweepDag& t, int64_t D)
{
    int64_t n = 0;
    for (int64_t t0 = 0; t0 < t.nt0; ++t0) {
        int64_t lo = D - t0 - t.nts + 1, hi = D - t0;
        if (lo < 0) lo = 0;
        if (hi > t.nt1 - 1) hi = t.nt1 - 1;
        if (hi >= lo) n += hi - lo + 1;
    }
    return n;
}

__global__ void k_sweepdag_prefix(SweepDag t, int64_t* pre)
{
    for (int64_t d = threadIdx.x; d < t.Dn; d += blockDim.x) pre[d + 1] = count_tiles_on(t, d);
    __syncthreads();
    if (threadIdx.x == 0) {
        pre[0] = 0;
        for (int64_t d = 0; d < t.Dn; ++d) pre[d + 1] += pre[d];
    }
}

// Tiles of the previous sweep a tile (T0, T1, TS) must wait for (flag indices; returns how many).
// A tile's completion implies that of every tile of its sweep with no larger coordinates, so one
// "highest" tile stands for a set:
//   (a) the tile beyond this one by the radius in every coordinate: every point within the radius of
//       this tile's points, whose old values it reads and which read, in the previous sweep, the
//       values this tile overwrites;
//   (b) for points within r of the low face of an axis, the tiles holding the wrapped neighbours at
//       the high end of that axis: they must hold the previous sweep's values when read, and they
//       read this tile's points (their wrapped + neighbours) in the previous sweep before these are
//       overwritten.
// Everything else a point reads is of its own sweep and is ordered by the in-sweep waits.
template <int DIM, int R>
__device__ __forceinline__ int sweep_dag_prev_waits(const SweepDag& t, const Geo& g, int64_t T0, int64_t T1,
                                                    int64_t TS, int64_t* out)
{
    auto cdiv = [](int64_t a, int64_t b) { return (a + b - 1) / b; };
    auto idx = [&](int64_t a, int64_t b, int64_t c) {
        a = a < t.nt0 - 1 ? a : t.nt0 - 1;
        b = b < t.nt1 - 1 ? b : t.nt1 - 1;
        c = c < t.nts - 1 ? c : t.nts - 1;
        return (a * t.nt1 + b) * t.nts + c;
    };
    int n = 0;
    out[n++] = idx(T0 + cdiv(R, t.b0), T1 + cdiv(R, t.b1), TS + cdiv(R, t.bs));
    // extents of the tile's points (the star has no sigma skew)
    const int64_t i_lo = T0 * t.b0, i_hi = (T0 + 1) * t.b0 - 1 < g.n0 - 1 ? (T0 + 1) * t.b0 - 1 : g.n0 - 1;
    const int64_t j_lo = T1 * t.b1, j_hi = (T1 + 1) * t.b1 - 1 < g.n1 - 1 ? (T1 + 1) * t.b1 - 1 : g.n1 - 1;
    const int64_t th_lo = TS * t.bs, th_hi = th_lo + t.bs - 1;
    // the fast axis: points with k < R exist where theta - cp0 i - cp1 j < R
    if (th_lo < (int64_t)t.cp0 * i_hi + (int64_t)t.cp1 * j_hi + R)
        out[n++] = idx(T0, T1, ((int64_t)t.cp0 * i_hi + (int64_t)t.cp1 * j_hi + (g.n2 - 1)) / t.bs);
    // axis 1: rows j < R; their wrapped neighbours sit in the last row tile, theta up to
    // cp0 i + cp1 (n1 - 1) + k with k <= theta - cp0 i
    if (j_lo < R)
        out[n++] = idx(T0, t.nt1 - 1, ((int64_t)t.cp1 * (g.n1 - 1) + th_hi) / t.bs);
    // axis 0 (3D): planes i < R; wrapped neighbours in the last plane tile, theta up to cp0 (n0 - 1) + theta
    if (DIM == 3 && i_lo < R) out[n++] = idx(t.nt0 - 1, T1, ((int64_t)t.cp0 * (g.n0 - 1) + th_hi) / t.bs);
    return n;
}

template <int DIM, int SHAPE, int R, int ARITH, class WS>
__global__ void __launch_bounds__(256) k_gs_sweepdag(double* __restrict__ u, Geo g, int bc, double c, WS w, SweepDag t,
                                                     const int64_t* __restrict__ pre, int* __restrict__ flags,
                                                     unsigned long long* __restrict__ ctr, int* status, WaitCfg wc)
{
    __shared__ long long s_T0, s_T1, s_TS, s_sw;
    __shared__ int s_go;
    unsigned long long* ticket = ctr;
    unsigned long long* finished = ctr + 1;
    const int64_t total = t.sweep_units * t.T;
    const int64_t s1 = g.n2, s0 = g.n1 * g.n2;
    for (;;) {
        if (threadIdx.x < 32) {
            // warp 0 claims the next tile and waits for it, all of its lanes together
            const int lane = threadIdx.x;
            long long tk = 0;
            if (lane == 0) tk = (long long)atomicAdd(ticket, 1ull);
            tk = __shfl_sync(FULL, tk, 0);
            if (lane == 0) s_go = tk < total;
            if (tk < total) {
                const int64_t sw = tk / t.sweep_units, rem = tk % t.sweep_units;
                int64_t lo = 0, hi = t.Dn - 1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) / 2;
                    if (pre[mid] <= rem) lo = mid; else hi = mid - 1;
                }
                const int64_t D = lo;
                int64_t r = rem - pre[D], T0 = 0, T1 = 0;
                for (int64_t t0 = 0; t0 < t.nt0; ++t0) {
                    int64_t a = D - t0 - t.nts + 1, b = D - t0;
                    if (a < 0) a = 0;
                    if (b > t.nt1 - 1) b = t.nt1 - 1;
                    const int64_t cnt = b >= a ? b - a + 1 : 0;
                    if (r < cnt) {
                        T0 = t0;
                        T1 = a + r;
                        break;
                    }
                    r -= cnt;
                }
                const int64_t TS = D - T0 - T1;
                if (lane == 0) {
                    s_T0 = T0;
                    s_T1 = T1;
                    s_TS = TS;
                    s_sw = sw;
                }
                // the three lower neighbours of this sweep, then what this tile needs of the previous
                // sweep (sweep_dag_prev_waits)
                bool ok = true;
                const int tag = (int)sw + 1;
                const int64_t f = (T0 * t.nt1 + T1) * t.nts + TS;
                if (sw > 0) {
                    int64_t pw[4];
                    const int np = sweep_dag_prev_waits<DIM, R>(t, g, T0, T1, TS, pw);
                    for (int q = 0; q < np; ++q)
                        ok &= wait_flag_ge_warp_at(flags, pw[q], t.sweep_units, (int)sw, wc.spin);
                }
                if (T0 > 0) ok &= wait_flag_ge_warp_at(flags, f - t.nt1 * t.nts, t.sweep_units, tag, wc.spin);
                if (T1 > 0) ok &= wait_flag_ge_warp_at(flags, f - t.nts, t.sweep_units, tag, wc.spin);
                if (TS > 0) ok &= wait_flag_ge_warp_at(flags, f - 1, t.sweep_units, tag, wc.spin);
                if (!ok && lane == 0) atomicExch(status, DEV_TIMEOUT);
                __threadfence();
            }
        }
        __syncthreads();
        if (!s_go) return;
        const int l1 = threadIdx.x % t.b1, l0 = threadIdx.x / t.b1;
        const int64_t i = s_T0 * t.b0 + l0;
        const int64_t j = s_T1 * t.b1 + l1 - (int64_t)t.skew * i;
        const bool owner = l0 < t.b0 && i < g.n0 && j >= 0 && j < g.n1;
        const int64_t kb = s_TS * t.bs - (int64_t)t.cp0 * i - (int64_t)t.cp1 * j;
        const bool in01 = (DIM < 3 || (i >= R && i < g.n0 - R)) && (j >= R && j < g.n1 - R);
        for (int ls = 0; ls < t.bs; ++ls) {
            const int64_t k = kb + ls;
            if (owner && k >= 0 && k < g.n2) {
                const int64_t p = i * s0 + j * s1 + k;
                st_in(u, p, g.n0 * s0,
                      (in01 && k >= R && k < g.n2 - R)
                          ? update_interior<DIM, SHAPE, R, ARITH, false>(u, p, s0, s1, w, g.n0 * s0)
                          : update_bc<DIM, SHAPE, R, ARITH>(u, i, j, k, g, bc, c, w));
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const int64_t f = (s_T0 * t.nt1 + s_T1) * t.nts + s_TS;
            __threadfence();
            if (s_sw * t.sweep_units + f != wc.stall) release_flag_at(flags, f, t.sweep_units, (int)s_sw + 1);
            atomicAdd(finished, 1ull);
        }
    }
}

// ------------------------------------------------------------------- host ---

bool gs_wavefront_supported(const stencil_handle_s* h, const Geo& g)
{
    (void)g;
    if (h->method != GAUSS_SEIDEL) return false;
    if (h->bc == BC_PERIODIC)  // in-sweep tile DAG: stars in 2D/3D (a periodic box has no hyperplane order)
        return h->dim >= 2 && h->shape == STAR && h->r <= 2;
    if (h->dim == 1) return h->r >= 1 && h->r <= 4;
    if (h->dim == 2) return h->r <= 2;
    return h->r == 1;
}

// Grow the handle's wavefront workspace to at least bytes (zeroed when grown).
static int wave_workspace(stencil_handle_s* h, size_t bytes, cudaStream_t st)
{
    if (h->wave_ws_bytes >= bytes) return STENCIL_OK;
    (void)st;
    if (h->wave_ws) {
        cudaDeviceSynchronize();
        cudaFree(h->wave_ws);
        h->wave_ws = nullptr;
        h->wave_ws_bytes = 0;
    }
    size_t want = bytes + bytes / 4 + 4096;
    if (cudaMalloc(&h->wave_ws, want) != cudaSuccess) {
        cudaGetLastError();
        return STENCIL_ENOMEM;
    }
    if (cudaMemset(h->wave_ws, 0, want) != cudaSuccess) return STENCIL_ECUDA;
    h->wave_ws_bytes = want;
    h->wave_epoch = 0;
    return STENCIL_OK;
}

static WaitCfg take_wait_cfg(stencil_handle_s* h)
{
    WaitCfg wc{h->debug_spin > 0 ? h->debug_spin : SPIN_LIMIT, h->debug_stall_tile};
    h->debug_stall_tile = -1;
    h->debug_spin = 0;
    return wc;
}

template <int R, class WS>
static void launch_gs1d_wave(const RunCtx& ctx, double* u, int64_t T, const WS& w, unsigned long long* progress,
                             int* ticket, unsigned tag, const WaitCfg& wc)
{
    const stencil_handle_s* h = ctx.h;
    const unsigned nB = (unsigned)((T + 31) / 32);
    if (h->arith == ARITH_FMA)
        k_gs1d_wave<R, ARITH_FMA, WS><<<nB, 32, 0, ctx.st>>>(u, ctx.g.n2, h->c, w, T, progress, ticket, h->d_status,
                                                             tag, wc);
    else
        k_gs1d_wave<R, ARITH_UNFUSED, WS><<<nB, 32, 0, ctx.st>>>(u, ctx.g.n2, h->c, w, T, progress, ticket,
                                                                 h->d_status, tag, wc);
}

template <int R>
static int wave_1d(const RunCtx& ctx, double* u, int64_t T, bool prepare_only = false)
{
    stencil_handle_s* h = ctx.h;
    WArr<2 * R + 1> w;
    for (int q = 0; q < 2 * R + 1; ++q) w.w[q] = h->w_desc[q];
    const int64_t nB = (T + 31) / 32;
    const size_t bytes = 64 + (size_t)nB * sizeof(unsigned long long);
    int rc = wave_workspace(h, bytes, ctx.st);
    if (rc || prepare_only) return rc;
    int* ticket = (int*)h->wave_ws;
    unsigned long long* progress = (unsigned long long*)((char*)h->wave_ws + 64);
    // stream-ordered reset of the ticket and progress words: replays of a captured graph start clean
    const unsigned tag = 1;
    if (cudaMemsetAsync(h->wave_ws, 0, bytes, ctx.st) != cudaSuccess) return STENCIL_ECUDA;
    const WaitCfg wc = take_wait_cfg(h);
    if (ctx.sd.field) {  // per-point weights: the single-warp kernel
        launch_gs1d_wave<R>(ctx, u, T, WField<2 * R + 1>{ctx.sd.field, ctx.sd.npts}, progress, ticket, tag, wc);
    } else if (R == 1) {
        WArr<3> w3;
        for (int q = 0; q < 3; ++q) w3.w[q] = w.w[q];
        if (h->arith == ARITH_FMA)
            k_gs1d_wave4<ARITH_FMA><<<(unsigned)nB, 256, 0, ctx.st>>>(u, ctx.g.n2, h->c, w3, T, progress, ticket,
                                                                       h->d_status, tag, wc);
        else
            k_gs1d_wave4<ARITH_UNFUSED><<<(unsigned)nB, 256, 0, ctx.st>>>(u, ctx.g.n2, h->c, w3, T, progress, ticket,
                                                                           h->d_status, tag, wc);
    } else {
        launch_gs1d_wave<R>(ctx, u, T, w, progress, ticket, tag, wc);
    }
    g_launches++;
    return cuda_rc(cudaGetLastError());
}

template <int DIM, int SHAPE, int R, int W, class WS>
static int launch_wave(const RunCtx& ctx, double* u, const WS& w, const WaveGeo& wg, const int64_t* dpre, int* flags,
                       int* ticket, int tag);
template <int DIM, int SHAPE, int R, class WS>
static int launch_sweepdag(const RunCtx& ctx, double* u, const WS& w, const SweepDag& t, const int64_t* dpre,
                           int* flags, unsigned long long* ctr);

template <int ARITH>
static int launch_gs2d_dec(const RunCtx& ctx, double* u, const WaveGeo& wg, const int64_t* dpre, int* flags,
                           int* ticket, int tag);

// dec: the decoupled tile (k_gs2d_dec; 2D 5-point star with one weight per term only)
template <int DIM, int SHAPE, int R, int W>
static int wave_tiles(const RunCtx& ctx, double* u, int64_t T, int lanes, bool prepare_only = false, bool dec = false)
{
    (void)lanes;
    stencil_handle_s* h = ctx.h;
    const Geo& g = ctx.g;
    const bool box = SHAPE == BOX;
    WaveGeo wg;
    wg.s = dec ? GD_S : R + 1;
    if (DIM == 2) {
        wg.a1 = box ? R : 0;
        wg.b1 = R * (1 + wg.a1);
        wg.a2 = wg.c2 = wg.b2 = 0;
        // skewed rows per tile: 16, or what the wavefront plan asks for (tile[1], 2..64)
        const int64_t hp = ctx.wtile[1];
        wg.H = hp >= 2 && hp <= 64 ? (int)hp : 16;
        wg.HJ = 1;
    } else {
        wg.a1 = box ? R : 0;
        wg.b1 = R * (1 + wg.a1);
        wg.c2 = box ? R : 0;
        wg.a2 = box ? R * (1 + R) : 0;
        wg.b2 = R * (1 + wg.a2 + wg.c2);
        wg.H = 4;
        wg.HJ = 4;
    }
    const int64_t L = 32;
    int64_t extI, extJ, extK;
    if (DIM == 2) {
        extI = g.n1 + wg.s * (L - 1);
        extJ = g.n2 + wg.a1 * (g.n1 - 1) + wg.b1 * (L - 1);
        wg.nI = (extI + wg.H - 1) / wg.H;
        wg.nJ = (extJ + W - 1) / W;
        wg.nK = 1;
        wg.dI = (R + wg.s * (int)(L - 1)) / wg.H + 2;
        wg.dJ = (R * (1 + wg.a1) + wg.b1 * (int)(L - 1)) / W + 2;
        wg.dK = 0;
    } else {
        extI = g.n0 + wg.s * (L - 1);
        extJ = g.n1 + wg.a1 * (g.n0 - 1) + wg.b1 * (L - 1);
        extK = g.n2 + wg.a2 * (g.n0 - 1) + wg.c2 * (g.n1 - 1) + wg.b2 * (L - 1);
        wg.nI = (extI + wg.H - 1) / wg.H;
        wg.nJ = (extJ + wg.HJ - 1) / wg.HJ;
        wg.nK = (extK + W - 1) / W;
        wg.dI = (R + wg.s * (int)(L - 1)) / wg.H + 2;
        wg.dJ = (R * (1 + wg.a1) + wg.b1 * (int)(L - 1)) / wg.HJ + 2;
        wg.dK = (R * (1 + wg.a2 + wg.c2) + wg.b2 * (int)(L - 1)) / W + 2;
    }
    wg.nB = (T + 31) / 32;
    wg.T = T;
    wg.db = wg.dI + wg.dJ + wg.dK + 1;
    wg.nD = (wg.nI - 1) + (wg.nJ - 1) + (wg.nK - 1) + (wg.nB - 1) * wg.db + 1;
    wg.ntiles = wg.nB * wg.nI * wg.nJ * wg.nK;
    if (wg.ntiles > (int64_t)1 << 31) return STENCIL_EUNSUPPORTED;
    const size_t pre_bytes = (size_t)(wg.nD + 1) * sizeof(int64_t);
    const size_t flag_off = 256 + ((pre_bytes + 255) & ~size_t(255));
    const size_t bytes = flag_off + (size_t)wg.ntiles * sizeof(int);
    int rc = wave_workspace(h, bytes, ctx.st);
    if (rc || prepare_only) return rc;
    int* ticket = (int*)h->wave_ws;  // 8 bytes used (64-bit counter)
    int64_t* dpre = (int64_t*)((char*)h->wave_ws + 256);
    int* flags = (int*)((char*)h->wave_ws + flag_off);
    // stream-ordered reset of ticket and flags, schedule table built on the device:
    // nothing here waits on the host, so the run can be captured into a graph and replayed
    const int tag = 1;
    if (cudaMemsetAsync(ticket, 0, 8, ctx.st) != cudaSuccess) return STENCIL_ECUDA;
    if (cudaMemsetAsync(flags, 0, (size_t)wg.ntiles * sizeof(int), ctx.st) != cudaSuccess) return STENCIL_ECUDA;
    k_wave_prefix<DIM><<<1, 256, 0, ctx.st>>>(wg, dpre);
    g_launches++;
    if constexpr (DIM == 2 && SHAPE == STAR && R == 1 && W == GD_W) {
        if (dec)
            return h->arith == ARITH_FMA ? launch_gs2d_dec<ARITH_FMA>(ctx, u, wg, dpre, flags, ticket, tag)
                                         : launch_gs2d_dec<ARITH_UNFUSED>(ctx, u, wg, dpre, flags, ticket, tag);
    }
    constexpr int K = Stn<DIM, SHAPE, R>::K;
    if (ctx.sd.field)
        return launch_wave<DIM, SHAPE, R, W>(ctx, u, WField<K>{ctx.sd.field, ctx.sd.npts}, wg, dpre, flags, ticket, tag);
    WArr<K> w;
    for (int q = 0; q < K; ++q) w.w[q] = h->w_desc[q];
    return launch_wave<DIM, SHAPE, R, W>(ctx, u, w, wg, dpre, flags, ticket, tag);
}

template <int DIM, int SHAPE, int R, int W, class WS>
static int launch_wave(const RunCtx& ctx, double* u, const WS& w, const WaveGeo& wg, const int64_t* dpre, int* flags,
                       int* ticket, int tag)
{
    stencil_handle_s* h = ctx.h;
    auto kern = h->arith == ARITH_FMA ? k_gs_wave<DIM, SHAPE, R, ARITH_FMA, W, WS>
                                      : k_gs_wave<DIM, SHAPE, R, ARITH_UNFUSED, W, WS>;
    int nsm = 0, per_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0);
    // two CTAs (8 worker warps) per SM by default: more tiles in flight would slow the tiles on
    // the DAG's critical path (they share the FP64 pipe); fewer leave it idle. A fixed wavefront
    // plan may ask for another count (tile[0]).
    const int want = ctx.wtile[0] > 0 ? (int)ctx.wtile[0] : 2;
    int64_t nblk = (int64_t)nsm * (per_sm > want ? want : (per_sm > 0 ? per_sm : 1));
    const int64_t need = (wg.ntiles + 3) / 4;
    if (nblk > need) nblk = need;
    const WaitCfg wc = take_wait_cfg(h);
    kern<<<(unsigned)nblk, 128, 0, ctx.st>>>(u, ctx.g, h->c, w, wg, dpre, flags, ticket, h->d_status, tag, wc);
    g_launches++;
    return cuda_rc(cudaGetLastError());
}

template <int ARITH>
static int launch_gs2d_dec(const RunCtx& ctx, double* u, const WaveGeo& wg, const int64_t* dpre, int* flags,
                           int* ticket, int tag)
{
    stencil_handle_s* h = ctx.h;
    WArr<5> w;
    for (int q = 0; q < 5; ++q) w.w[q] = h->w_desc[q];
    auto kern = k_gs2d_dec<ARITH>;
    int nsm = 0, per_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GD_THREADS, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return STENCIL_ECUDA;
    }
    // every CTA waits on tiles other CTAs hold: all of them must be resident (the count is capped
    // at the occupancy); 2 per SM by default, or what the wavefront plan asks for (tile[0])
    const int want = ctx.wtile[0] > 0 ? (int)ctx.wtile[0] : 2;
    int64_t nblk = (int64_t)nsm * (per_sm < want ? per_sm : want);
    if (nblk > wg.ntiles) nblk = wg.ntiles;
    const WaitCfg wc = take_wait_cfg(h);
    kern<<<(unsigned)nblk, GD_THREADS, 0, ctx.st>>>(u, ctx.g, h->c, w, wg, dpre, flags, ticket, h->d_status, tag, wc);
    g_launches++;
    return cuda_rc(cudaGetLastError());
}

template <int DIM, int SHAPE, int R>
static int sweep_dag(const RunCtx& ctx, double* u, int64_t T, bool prepare_only)
{
    stencil_handle_s* h = ctx.h;
    const Geo& g = ctx.g;
    const bool box = SHAPE == BOX;
    SweepDag t;
    t.cp1 = box ? 1 + R : 1;
    t.cp0 = DIM == 3 ? (box ? 1 + R * (t.cp1 + 1) : 1) : 0;
    t.skew = (DIM == 3 && box) ? R : 0;
    // small tiles: a sweep's critical path is about nt0 + nt1 + nts tiles long. The plan may set
    // the lines per tile along axes 0 and 1 (tile[0], tile[1]; one thread each, at most 256 in
    // all) and the hyperplane steps per tile (tile[2]).
    if (DIM == 3) {
        t.b0 = 8; t.b1 = 16; t.bs = 8;  // measured best on 512^3: 24.5 GStencil/s (8 x 8 x 16: 22.4)
    } else {
        t.b0 = 1; t.b1 = 64; t.bs = 32;
    }
    if (DIM == 3 && ctx.wtile[0] > 0) t.b0 = (int)std::min<int64_t>(ctx.wtile[0], 256);
    if (ctx.wtile[1] > 0) t.b1 = (int)std::min<int64_t>(ctx.wtile[1], 256);
    if (ctx.wtile[2] > 0) t.bs = (int)std::min<int64_t>(ctx.wtile[2], 1024);
    if (t.b0 * t.b1 > 256) t.b1 = 256 / t.b0;
    const int64_t thmax = t.cp0 * (g.n0 - 1) + t.cp1 * (g.n1 - 1) + (g.n2 - 1);
    t.nt0 = (g.n0 + t.b0 - 1) / t.b0;
    t.nt1 = (g.n1 + t.skew * (g.n0 - 1) + t.b1 - 1) / t.b1;
    t.nts = thmax / t.bs + 1;
    t.Dn = (t.nt0 - 1) + (t.nt1 - 1) + (t.nts - 1) + 1;
    t.sweep_units = t.nt0 * t.nt1 * t.nts;
    t.T = T;
    if (t.sweep_units > (int64_t)1 << 30) return STENCIL_EUNSUPPORTED;
    const size_t pre_bytes = (size_t)(t.Dn + 1) * sizeof(int64_t);
    const size_t flag_off = 256 + ((pre_bytes + 255) & ~size_t(255));
    const size_t bytes = flag_off + (size_t)t.sweep_units * sizeof(int);
    int rc = wave_workspace(h, bytes, ctx.st);
    if (rc || prepare_only) return rc;
    unsigned long long* ctr = (unsigned long long*)h->wave_ws;  // ticket, finished
    int64_t* dpre = (int64_t*)((char*)h->wave_ws + 256);
    int* flags = (int*)((char*)h->wave_ws + flag_off);
    if (cudaMemsetAsync(ctr, 0, 16, ctx.st) != cudaSuccess) return STENCIL_ECUDA;
    if (cudaMemsetAsync(flags, 0, (size_t)t.sweep_units * sizeof(int), ctx.st) != cudaSuccess) return STENCIL_ECUDA;
    k_sweepdag_prefix<<<1, 256, 0, ctx.st>>>(t, dpre);
    g_launches++;
    constexpr int K = Stn<DIM, SHAPE, R>::K;
    if (ctx.sd.field)
        return launch_sweepdag<DIM, SHAPE, R>(ctx, u, WField<K>{ctx.sd.field, ctx.sd.npts}, t, dpre, flags, ctr);
    WArr<K> w;
    for (int q = 0; q < K; ++q) w.w[q] = h->w_desc[q];
    return launch_sweepdag<DIM, SHAPE, R>(ctx, u, w, t, dpre, flags, ctr);
}

template <int DIM, int SHAPE, int R, class WS>
static int launch_sweepdag(const RunCtx& ctx, double* u, const WS& w, const SweepDag& t, const int64_t* dpre,
                           int* flags, unsigned long long* ctr)
{
    stencil_handle_s* h = ctx.h;
    const int64_t T = t.T;
    auto kern = h->arith == ARITH_FMA ? k_gs_sweepdag<DIM, SHAPE, R, ARITH_FMA, WS>
                                      : k_gs_sweepdag<DIM, SHAPE, R, ARITH_UNFUSED, WS>;
    int nsm = 0, per_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // whole warps (warp 0 claims and waits as one warp); threads past the tile's lines own no line
    const int nthr = (t.b0 * t.b1 + 31) / 32 * 32;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nthr, 0);
    int64_t nblk = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
    if (nblk > t.sweep_units * T) nblk = t.sweep_units * T;
    const WaitCfg wc = take_wait_cfg(h);
    kern<<<(unsigned)nblk, nthr, 0, ctx.st>>>(u, ctx.g, h->bc, h->c, w, t, dpre, flags, ctr, h->d_status, wc);
    g_launches++;
    return cuda_rc(cudaGetLastError());
}

// 2D Gauss-Seidel, rows as lanes (k_gs2d_rows): constant boundary, radius 1, constant weights (or a
// weight field for the star), rows of a multiple of four columns on a 32-byte-aligned grid and field
// (the dispatcher checks).
// Sweeps go to launches of at most GR_MAX_TASKS tasks (progress words) each.
constexpr int64_t GR_MAX_TASKS = (int64_t)1 << 18;  // 32 MiB of progress words at most

template <int SHAPE, int CH, int R>
static int gs2d_rows(const RunCtx& ctx, double* u, int64_t T, bool prepare_only)
{
    stencil_handle_s* h = ctx.h;
    RowGeo g;
    g.n0 = ctx.g.n1;
    g.n1 = ctx.g.n2;
    g.nb = (g.n0 + 31) / 32;
    constexpr int SK = SHAPE == STAR ? 1 : 2;
    g.steps = (g.n1 / 4 + 31 * SK + CH - 1) / CH * CH;
    if (g.n1 / 4 + 31 * SK + CH > INT32_MAX) return STENCIL_EUNSUPPORTED;  // progress words are int
    const int64_t tmax = GR_MAX_TASKS / g.nb > 0 ? GR_MAX_TASKS / g.nb : 1;
    const int64_t tl = T < tmax ? T : tmax;  // sweeps per launch
    const size_t bytes = 256 + (size_t)(tl * g.nb) * GR_PSTRIDE * sizeof(int);
    int rc = wave_workspace(h, bytes, ctx.st);
    if (rc || prepare_only) return rc;
    int* ticket = (int*)h->wave_ws;
    int* prog = (int*)((char*)h->wave_ws + 256);
    constexpr int K = Stn<2, SHAPE, R>::K;
    WArr<K> w;
    for (int q = 0; q < K; ++q) w.w[q] = h->w_desc[q];
    const bool field = ctx.sd.field != nullptr;
    auto kern = h->arith == ARITH_FMA ? k_gs2d_rows<SHAPE, ARITH_FMA, CH, false, R>
                                      : k_gs2d_rows<SHAPE, ARITH_UNFUSED, CH, false, R>;
    if constexpr (SHAPE == STAR && R == 1) {
        if (field)
            kern = h->arith == ARITH_FMA ? k_gs2d_rows<SHAPE, ARITH_FMA, CH, true>
                                         : k_gs2d_rows<SHAPE, ARITH_UNFUSED, CH, true>;
    }
    int nsm = 0, per_sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, GR_THREADS, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return STENCIL_ECUDA;
    }
    // CTAs of four worker warps per SM: 4 by default, or what the wavefront plan asks for (tile[0])
    const int want = ctx.wtile[0] > 0 ? (int)ctx.wtile[0] : 4;
    const WaitCfg wc = take_wait_cfg(h);
    for (int64_t s0 = 0; s0 < T; s0 += tl) {
        g.T = T - s0 < tl ? T - s0 : tl;
        g.ntasks = g.T * g.nb;
        int64_t nblk = (int64_t)nsm * (per_sm < want ? per_sm : want);
        const int64_t need = (g.ntasks + GR_THREADS / 32 - 1) / (GR_THREADS / 32);
        if (nblk > need) nblk = need;
        if (cudaMemsetAsync(ticket, 0, 8, ctx.st) != cudaSuccess) return STENCIL_ECUDA;
        if (cudaMemsetAsync(prog, 0, (size_t)g.ntasks * GR_PSTRIDE * sizeof(int), ctx.st) != cudaSuccess)
            return STENCIL_ECUDA;
        kern<<<(unsigned)nblk, GR_THREADS, 0, ctx.st>>>(u, g, h->c, w, prog, ticket, h->d_status, wc, ctx.sd.field);
        g_launches++;
        if (cudaGetLastError() != cudaSuccess) return STENCIL_ECUDA;
    }
    return STENCIL_OK;
}

// steps per chunk of the rows pipeline: 8, or 16 / 64 / 128 when the wavefront plan asks (tile[1])
template <int SHAPE, int R>
static int gs2d_rows(const RunCtx& ctx, double* u, int64_t T, bool prepare_only)
{
    if (ctx.wtile[1] == 16) return gs2d_rows<SHAPE, 16, R>(ctx, u, T, prepare_only);
    if (ctx.wtile[1] == 64) return gs2d_rows<SHAPE, 64, R>(ctx, u, T, prepare_only);
    if (ctx.wtile[1] == 128) return gs2d_rows<SHAPE, 128, R>(ctx, u, T, prepare_only);
    return gs2d_rows<SHAPE, GR_CHUNK, R>(ctx, u, T, prepare_only);  // 8 steps
}

static int wave_dispatch(const RunCtx& ctx, double* u, int64_t T, int lanes, bool prep)
{
    const stencil_handle_s* h = ctx.h;
    if (h->bc == BC_PERIODIC) {  // sweeps cannot overlap: one persistent launch, tiles in a DAG per sweep
        if (h->dim == 2 && h->shape == STAR && h->r == 1) return sweep_dag<2, STAR, 1>(ctx, u, T, prep);
        if (h->dim == 2 && h->shape == STAR && h->r == 2) return sweep_dag<2, STAR, 2>(ctx, u, T, prep);
        if (h->dim == 3 && h->shape == STAR && h->r == 1) return sweep_dag<3, STAR, 1>(ctx, u, T, prep);
        if (h->dim == 3 && h->shape == STAR && h->r == 2) return sweep_dag<3, STAR, 2>(ctx, u, T, prep);
        return STENCIL_EUNSUPPORTED;
    }
    if (h->dim == 1) {
        switch (h->r) {
            case 1: return wave_1d<1>(ctx, u, T, prep);
            case 2: return wave_1d<2>(ctx, u, T, prep);
            case 3: return wave_1d<3>(ctx, u, T, prep);
            case 4: return wave_1d<4>(ctx, u, T, prep);
        }
        return STENCIL_EUNSUPPORTED;
    }
    if (h->dim == 2) {
        // points per lane and step: 16, or 8 when the wavefront plan asks for it (tile[2] = 8);
        // tile[2] = 1 selects the decoupled tile for the 5-point star with one weight per term
        // (measured level with the one-warp tile at best, so not the default)
        const int64_t pw = ctx.wtile[2];
        const bool w8 = pw == 8;
        // tile[2] = 0 (default) or 2: rows as lanes where they apply (radius 1 with constant weights or
        // the star's weight field, the radius-2 star with constant weights; rows of whole 32-byte
        // groups of four columns); 16 or 8: the one-warp
        // tiles with that many points per lane and step; 1: the decoupled tile. Other grids take the
        // one-warp tiles.
        const bool rows_ok =
            ctx.g.n2 % 4 == 0 && ((uintptr_t)u & 31) == 0 &&
            ((h->r == 1 && (!ctx.sd.field || (h->shape == STAR && ((uintptr_t)ctx.sd.field & 31) == 0))) ||
             (h->r == 2 && h->shape == STAR && !ctx.sd.field));
        if ((pw == 0 || pw == 2) && rows_ok) {
            if (h->r == 2) return gs2d_rows<STAR, 2>(ctx, u, T, prep);
            return h->shape == STAR ? gs2d_rows<STAR, 1>(ctx, u, T, prep) : gs2d_rows<BOX, 1>(ctx, u, T, prep);
        }
        if (h->shape == STAR && h->r == 1)
            return w8 ? wave_tiles<2, STAR, 1, 8>(ctx, u, T, lanes, prep)
                      : wave_tiles<2, STAR, 1, 16>(ctx, u, T, lanes, prep, pw == 1 && !ctx.sd.field);
        if (h->shape == BOX && h->r == 1)
            return w8 ? wave_tiles<2, BOX, 1, 8>(ctx, u, T, lanes, prep)
                      : wave_tiles<2, BOX, 1, 16>(ctx, u, T, lanes, prep);
        if (h->shape == STAR && h->r == 2) return wave_tiles<2, STAR, 2, 8>(ctx, u, T, lanes, prep);
        if (h->shape == BOX && h->r == 2) return wave_tiles<2, BOX, 2, 8>(ctx, u, T, lanes, prep);
    } else {
        if (h->shape == STAR && h->r == 1) return wave_tiles<3, STAR, 1, 8>(ctx, u, T, lanes, prep);
        if (h->shape == BOX && h->r == 1) return wave_tiles<3, BOX, 1, 4>(ctx, u, T, lanes, prep);
    }
    return STENCIL_EUNSUPPORTED;
}

int gs_wavefront_run(const RunCtx& ctx, double* u, int64_t T, int lanes)
{
    return wave_dispatch(ctx, u, T, lanes, false);
}

int gs_wavefront_prepare(stencil_handle_s* h, const Geo& g, int64_t T, const int64_t wtile[3])
{
    if (!gs_wavefront_supported(h, g) || T <= 0) return STENCIL_OK;
    RunCtx ctx;
    ctx.h = h;
    ctx.g = g;
    ctx.st = 0;
    ctx.sd = make_sd(h, g.n0 * g.n1 * g.n2);
    for (int d = 0; d < 3; ++d) ctx.wtile[d] = wtile ? wtile[d] : 0;
    return wave_dispatch(ctx, nullptr, T, 0, true);
}

}  // namespace gbst
