// Longest common subsequence (Section 3.4, "Longest common subsequence") as
// a 1D Gauss-Seidel wavefront: x (over A) is time, y (over B) is space.
//
// Both kernels use the temporal-vectorisation layout of the Gauss-Seidel
// wavefront: a warp takes a strip of consecutive rows of A; lane k holds
// rows one step behind lane k - 1 (spatial skew s = 1, the legality bound the
// paper gives LCS), so at every step lane k receives from lane k - 1, by warp
// shuffle, the value of the row above at the column it is about to update.
// Lane 0 reads the row above the strip (written by the previous strip) in
// chunks of 32 values, loaded one chunk ahead by the whole warp and handed
// to lane 0 by shuffle; the top lane writes the strip's last row for the
// next strip and publishes its progress. Strips are handed out in order by a
// ticket counter to a persistent grid of warps, and their row buffers form a
// ring of (warps + 1) rows: a strip overwrites a buffer only after every
// strip still reading it has passed that column (each strip waits on its
// predecessor's progress, so by induction on all earlier ones).
//
//   k_lcs_dp    one cell per lane and step: lcs = diag + 1 where A[x] ==
//               B[y], else max(up, left) (the paper's blend of the equality
//               mask). B[y] travels down the lanes with the values.
//   k_lcs_bits  64 cells per lane and step, Q rows of A per lane: a row is
//               the bit vector V of its differences (bit y clear iff
//               lcs[x][y+1] - lcs[x][y] = 1); one row of A advances V by
//               U = V & M[a], V = (V + U + carry) | (V & ~U), the addition
//               carried from word to word along the row (Allison and Dix
//               1986; Hyyro 2004). M[a] is the bit mask of the positions of
//               symbol a in B. The final row is recovered from V by prefix
//               counts of its clear bits.
//
// Every wait is bounded: a wait that gives up records STENCIL_ETIMEOUT in the
// workspace's status word and the kernel runs on to its end.
#include <cstdint>
#include <cstdio>

#include "lcs.h"
#include "internal.h"

namespace gbst {

namespace {

constexpr unsigned FULL32 = 0xffffffffu;
constexpr int LCS_WARPS_PER_CTA = 4;
constexpr int LCS_SPIN = 1 << 22;   // polls before a wait gives up (each poll sleeps up to ~0.5 us)
constexpr int LCS_PUBLISH = 32;     // the top lane publishes its progress every this many steps
constexpr int LCS_BITS_Q = 16;      // rows of A per lane in k_lcs_bits (measured: 4 -> 45 ms, 8 -> 27, 16 -> 23, 32 -> 24 at 200000^2)
constexpr int64_t LCS_MAX_LEN = (int64_t)1 << 30;  // longest A or B (32-bit step counters)

enum { LCS_DEV_OK = 0, LCS_DEV_TIMEOUT = 1 };

// Header of the workspace: the strip ticket and the status word.
struct LcsHeader {
    unsigned long long ticket;
    int status;
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Wait (bounded) until *p >= need. Polls with relaxed loads and takes one acquire load once the
// value is there: an acquire at GPU scope invalidates the SM's L1, so polling with it would keep
// flushing the L1 under every warp of the SM. Returns the value seen, or 0 if the wait gave up.
__device__ unsigned long long wait_at_least(const unsigned long long* p, unsigned long long need)
{
    for (int it = 0; it < LCS_SPIN; ++it) {
        if (ld_relaxed_u64(p) >= need) return ld_acquire_u64(p);
        __nanosleep(it < 16 ? 64 : 256);
    }
    return 0;
}

// One row of the bit-parallel update on a 64-bit word: u = v & m, s = v + u + carry (the carry of the
// previous word of this row; the carry out is returned in carry), v = s | (v & ~u). The add is one
// carry chain over the two 32-bit halves: the first add sets the carry flag from the saved carry.
__device__ __forceinline__ uint64_t bits_row(uint64_t v, uint64_t m, uint32_t& carry)
{
    const uint64_t u = v & m;
    uint32_t s0, s1;
    asm("{\n\t"
        ".reg .u32 t;\n\t"
        "add.cc.u32 t, %2, 0xffffffff;\n\t"
        "addc.cc.u32 %0, %3, %5;\n\t"
        "addc.cc.u32 %1, %4, %6;\n\t"
        "addc.u32 %2, 0, 0;\n\t"
        "}"
        : "=r"(s0), "=r"(s1), "+r"(carry)
        : "r"((uint32_t)v), "r"((uint32_t)(v >> 32)), "r"((uint32_t)u), "r"((uint32_t)(u >> 32)));
    const uint64_t s = ((uint64_t)s1 << 32) | s0;
    return s | (v & ~u);
}

struct LcsGeo {
    int64_t na, nb;
    int64_t nstrips;   // strips of rows
    int64_t ring;      // row buffers in the ring
    int64_t rowlen;    // elements per row buffer (nb for DP, words for BITS)
};

// ------------------------------------------------------------------- DP ---

// Strip b = rows 32 b .. 32 b + 31 of A (0-based); lane k holds row x = 32 b + k
// and at step j updates column y = j - k (0-based; lcs column y + 1).
// rows: the ring of row buffers (g.ring x g.nb); the last strip writes into
// out_row + 1 instead (lcs[na][1..nb]).
__global__ void __launch_bounds__(32 * LCS_WARPS_PER_CTA) k_lcs_dp(const uint8_t* __restrict__ A,
                                                                   const uint8_t* __restrict__ B, LcsGeo g,
                                                                   int32_t* __restrict__ rows,
                                                                   int32_t* __restrict__ out_row,
                                                                   unsigned long long* __restrict__ progress,
                                                                   LcsHeader* hdr)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(&hdr->ticket, 1ull);
        const int64_t b = (int64_t)__shfl_sync(FULL32, tk, 0);
        if (b >= g.nstrips) return;
        const int L = (int)(g.na - 32 * b < 32 ? g.na - 32 * b : 32);
        const int top = L - 1;
        const uint8_t a = lane < L ? A[32 * b + lane] : 0;
        const int32_t* above = b > 0 ? rows + ((b - 1) % g.ring) * g.nb : nullptr;
        int32_t* below = b == g.nstrips - 1 ? out_row + 1 : rows + (b % g.ring) * g.nb;
        const unsigned long long* prev = b > 0 ? progress + b - 1 : nullptr;
        unsigned long long* mine = progress + b;
        int64_t known = b > 0 ? 0 : INT64_MAX;  // columns of the row above known to be final
        // columns [0, upto) of the row above must be final before lane 0's chunk loads
        auto need = [&](int64_t upto) {
            if (lane == 0 && upto > known) {
                const unsigned long long seen = wait_at_least(prev, (unsigned long long)upto);
                if (seen >= (unsigned long long)upto) {
                    known = (int64_t)seen;
                } else {
                    atomicExch(&hdr->status, LCS_DEV_TIMEOUT);
                    known = INT64_MAX;
                }
            }
            __syncwarp();
        };
        auto load_up = [&](int64_t ch) -> int32_t {
            const int64_t p = ch * 32 + lane;
            return (above && p < g.nb) ? __ldcg(above + p) : 0;
        };
        auto load_b = [&](int64_t ch) -> int {
            const int64_t p = ch * 32 + lane;
            return p < g.nb ? (int)B[p] : -1;
        };
        int cur_ch = 0;
        const int nb = (int)g.nb;
        need(nb < 64 ? nb : 64);
        int32_t cur_up = load_up(0), nxt_up = load_up(1);
        int cur_b = load_b(0), nxt_b = load_b(1);
        int32_t out = 0;   // this lane's value at its last column: lcs[x][y - 1] when it starts column y
        int32_t diag = 0;  // lcs[x - 1][y - 1]
        int bsym = -1;     // B[y] of this lane's last column, passed to the next lane
        // lane 0 enters chunk c (warp-uniform): the next chunk's loads go out
        auto enter_chunk = [&](int c) {
            cur_ch = c;
            cur_up = nxt_up;
            cur_b = nxt_b;
            const int upto = (c + 2) * 32;
            need(upto < nb ? upto : nb);
            nxt_up = load_up(c + 1);
            nxt_b = load_b(c + 1);
        };
        // one step: lane 0 takes column j from the chunks (lane src = j & 31), the others from lane - 1
        auto step = [&](int j, int src, bool all_inside) {
            const int32_t up0 = __shfl_sync(FULL32, cur_up, src);
            const int b0 = __shfl_sync(FULL32, cur_b, src);
            int32_t up = __shfl_up_sync(FULL32, out, 1);
            int bb = __shfl_up_sync(FULL32, bsym, 1);
            up = lane == 0 ? up0 : up;
            bb = lane == 0 ? b0 : bb;
            const int y = j - lane;
            // the blend of the equality mask: diag + 1 where the symbols match, else max(up, left);
            // lanes outside [0, nb) keep their state (selects, no divergent branch)
            const int32_t v = ((int)a == bb) ? diag + 1 : (up > out ? up : out);
            const bool act = all_inside || (unsigned)y < (unsigned)nb;
            out = act ? v : out;
            diag = act ? up : diag;
            bsym = act ? bb : bsym;
            if (act && lane == top) below[y] = v;
        };
        auto publish = [&](int done) {
            if (lane == top) st_release_u64(mine, (unsigned long long)done);
        };
        const int steps = nb + top;
        int j = 0;
        // chunks in which every lane of a full strip is inside the row: unrolled by 32, the chunk
        // position of each step known at compile time; the top lane publishes once per chunk
        const int full_end = top == 31 ? ((nb - 31) >> 5) : 0;  // chunks 1 .. full_end - 1
        for (; j < 32 && j < steps; ++j) {
            step(j, j & 31, false);
            const int done = j - top + 1;
            if (done > 0 && ((done & (LCS_PUBLISH - 1)) == 0 || done == nb)) publish(done);
        }
        for (int c = 1; c < full_end; ++c) {
            enter_chunk(c);
#pragma unroll
            for (int t = 0; t < 32; ++t) step(32 * c + t, t, true);
            // after step 32 c + 31 the top lane has finished columns [0, 32 c + 1); publish the multiple of 32
            publish(32 * c);
        }
        if (full_end > 1) j = 32 * full_end;
        for (; j < steps; ++j) {
            if ((j & 31) == 0) enter_chunk(j >> 5);
            step(j, j & 31, false);
            const int done = j - top + 1;
            if (done > 0 && ((done & (LCS_PUBLISH - 1)) == 0 || done == nb)) publish(done);
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------------- BITS ---

// M[a * nw + w]: bit i set iff B[64 w + i] == a (a = 0..255).
__global__ void k_lcs_masks(const uint8_t* __restrict__ B, int64_t nb, int64_t nw, uint64_t* __restrict__ M)
{
    const int64_t total = 256 * nw;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(q / nw);
        const int64_t w = q - (int64_t)a * nw;
        uint64_t m = 0;
        const int64_t p0 = w * 64;
        const int n = nb - p0 < 64 ? (int)(nb - p0) : 64;
        for (int i = 0; i < n; ++i) m |= (uint64_t)(__ldg(B + p0 + i) == a) << i;
        M[q] = m;
    }
}

// Strip b = rows 32 Q b .. 32 Q (b + 1) - 1 of A; lane k holds rows 32 Q b + Q k + r
// (r = 0..Q-1) and at step j advances word w = j - k of each of them in turn.
// rows: the ring of difference vectors (g.ring x nw words); the last strip
// writes the final vector into vfinal.
template <int Q>
__global__ void __launch_bounds__(32 * LCS_WARPS_PER_CTA) k_lcs_bits(const uint8_t* __restrict__ A,
                                                                     const uint64_t* __restrict__ M, LcsGeo g,
                                                                     uint64_t* __restrict__ rows,
                                                                     uint64_t* __restrict__ vfinal,
                                                                     unsigned long long* __restrict__ progress,
                                                                     LcsHeader* hdr)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = g.rowlen;
    for (;;) {
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(&hdr->ticket, 1ull);
        const int64_t b = (int64_t)__shfl_sync(FULL32, tk, 0);
        if (b >= g.nstrips) return;
        const int64_t x0 = 32 * Q * b;
        const int64_t nrows = g.na - x0 < 32 * Q ? g.na - x0 : 32 * Q;
        const int top = (int)((nrows + Q - 1) / Q) - 1;  // last lane holding a row
        const uint64_t* mrow[Q];
        bool valid[Q];
#pragma unroll
        for (int r = 0; r < Q; ++r) {
            const int64_t x = x0 + (int64_t)Q * lane + r;
            valid[r] = x < g.na;
            mrow[r] = M + (valid[r] ? (int64_t)A[x] : 0) * nw;
        }
        const uint64_t* above = b > 0 ? rows + ((b - 1) % g.ring) * nw : nullptr;
        uint64_t* below = b == g.nstrips - 1 ? vfinal : rows + (b % g.ring) * nw;
        const unsigned long long* prev = b > 0 ? progress + b - 1 : nullptr;
        unsigned long long* mine = progress + b;
        int64_t known = b > 0 ? 0 : INT64_MAX;
        auto need = [&](int64_t upto) {
            if (lane == 0 && upto > known) {
                const unsigned long long seen = wait_at_least(prev, (unsigned long long)upto);
                if (seen >= (unsigned long long)upto) {
                    known = (int64_t)seen;
                } else {
                    atomicExch(&hdr->status, LCS_DEV_TIMEOUT);
                    known = INT64_MAX;
                }
            }
            __syncwarp();
        };
        // the vector above the first strip is all ones: no differences yet (row 0 is all zero)
        auto load_up = [&](int64_t ch) -> uint64_t {
            const int64_t p = ch * 32 + lane;
            return (above && p < nw) ? __ldcg(above + p) : ~0ull;
        };
        int64_t cur_ch = 0;
        need(nw < 64 ? nw : 64);
        uint64_t cur_up = load_up(0), nxt_up = load_up(1);
        uint64_t out = ~0ull;
        uint32_t carry[Q];
#pragma unroll
        for (int r = 0; r < Q; ++r) carry[r] = 0;
        // mask words of this lane's rows at word ww (0 outside the row): loaded one step ahead of
        // use, so that their latency overlaps a step's carry chain instead of lengthening it
        auto load_masks = [&](int64_t ww, uint64_t* m) {
            const bool in = ww >= 0 && ww < nw && lane <= top;
#pragma unroll
            for (int r = 0; r < Q; ++r) m[r] = (in && valid[r]) ? __ldg(mrow[r] + ww) : 0ull;
        };
        uint64_t mcur[Q], mnxt[Q];
        load_masks(-(int64_t)lane, mcur);
        const int nwi = (int)nw;
        const int steps = nwi + top;
        for (int j = 0; j < steps; ++j) {
            load_masks(j - lane + 1, mnxt);
            if ((j & 15) == 0 && lane <= top) {  // the next cache line of each row, into L1
                const int ww = j - lane + 16;
                if (ww >= 0 && ww < nwi) {
#pragma unroll
                    for (int r = 0; r < Q; ++r)
                        if (valid[r]) asm volatile("prefetch.global.L1 [%0];" ::"l"(mrow[r] + ww));
                }
            }
            if ((j & 31) == 0 && j > 0) {  // warp-uniform: lane 0 enters chunk j / 32
                cur_ch = j >> 5;
                cur_up = nxt_up;
                const int64_t upto = (cur_ch + 2) * 32;
                need(upto < nw ? upto : nw);
                nxt_up = load_up(cur_ch + 1);
            }
            const uint64_t up0 = __shfl_sync(FULL32, cur_up, j & 31);
            uint64_t v = __shfl_up_sync(FULL32, out, 1);
            if (lane == 0) v = up0;
            // rows outside the strip and words outside [0, nw) have an all-zero mask, for which the
            // update is the identity (u = 0, the carry stays 0): no branch on validity
#pragma unroll
            for (int r = 0; r < Q; ++r) v = bits_row(v, mcur[r], carry[r]);
            out = v;
            const int w = j - lane;
            if (lane == top && (unsigned)w < (unsigned)nwi) below[w] = v;
            const int done = j - top + 1;  // words the top lane has finished (warp-uniform)
            if (done > 0 && ((done & (LCS_PUBLISH - 1)) == 0 || done == nwi)) {
                if (lane == top) st_release_u64(mine, (unsigned long long)done);
            }
#pragma unroll
            for (int r = 0; r < Q; ++r) mcur[r] = mnxt[r];
        }
        __syncwarp();
    }
}

// counts[w] = clear bits of the final vector's word w (within the nb valid bits).
__global__ void k_lcs_count(const uint64_t* __restrict__ v, int64_t nb, int64_t nw, int32_t* __restrict__ counts)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t nbits = nb - w * 64 < 64 ? nb - w * 64 : 64;
        const uint64_t valid = nbits == 64 ? ~0ull : ((1ull << nbits) - 1);
        counts[w] = __popcll(~v[w] & valid);
    }
}

// In-place exclusive prefix sum of counts[0..n) with counts[n] = the total (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) k_lcs_scan(int32_t* __restrict__ counts, int64_t n)
{
    __shared__ int32_t warp_sums[32];
    __shared__ int32_t carry_in;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_in = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int32_t c = i < n ? counts[i] : 0;
        int32_t incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t o = __shfl_up_sync(FULL32, incl, d);
            if (lane >= d) incl += o;
        }
        if (lane == 31) warp_sums[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int32_t s = warp_sums[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t o = __shfl_up_sync(FULL32, s, d);
                if (lane >= d) s += o;
            }
            warp_sums[lane] = s;  // inclusive over warps
        }
        __syncthreads();
        const int32_t before = carry_in + (wid > 0 ? warp_sums[wid - 1] : 0) + incl - c;
        if (i < n) counts[i] = before;
        __syncthreads();
        if (threadIdx.x == 0) carry_in += warp_sums[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[n] = carry_in;
}

// row[y] = clear bits of the final vector among bits [0, y), y = 0..nb.
__global__ void k_lcs_row(const uint64_t* __restrict__ v, const int32_t* __restrict__ pre, int64_t nb, int64_t nw,
                          int32_t* __restrict__ row)
{
    for (int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; y <= nb; y += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = y >> 6;
        const int bit = (int)(y & 63);
        row[y] = w >= nw ? pre[nw] : pre[w] + __popcll(~v[w] & ((1ull << bit) - 1));
    }
}

// ------------------------------------------------------------------- host ---

struct LcsLayout {
    LcsGeo g;
    int kernel;
    int64_t warps;  // persistent warps
    size_t off_progress, off_ring, off_masks, off_final, off_counts, total;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int lcs_layout(int64_t na, int64_t nb, int kernel, LcsLayout& L)
{
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        nsm = 152;
    }
    L.kernel = kernel == LCS_KERNEL_AUTO ? LCS_KERNEL_BITS : kernel;
    LcsGeo& g = L.g;
    g.na = na;
    g.nb = nb;
    const int64_t rows_per_strip = L.kernel == LCS_KERNEL_DP ? 32 : 32 * LCS_BITS_Q;
    g.nstrips = (na + rows_per_strip - 1) / rows_per_strip;
    g.rowlen = L.kernel == LCS_KERNEL_DP ? nb : (nb + 63) / 64;
    // strips in flight are bounded by the row length over the lag between strips; more warps only wait
    const int64_t cap = L.kernel == LCS_KERNEL_DP ? (int64_t)nsm * 16 : (int64_t)nsm * LCS_WARPS_PER_CTA;
    L.warps = g.nstrips < cap ? g.nstrips : cap;
    if (L.warps < 1) L.warps = 1;
    L.warps = (L.warps + LCS_WARPS_PER_CTA - 1) / LCS_WARPS_PER_CTA * LCS_WARPS_PER_CTA;
    g.ring = L.warps + 1;
    const size_t elt = L.kernel == LCS_KERNEL_DP ? sizeof(int32_t) : sizeof(uint64_t);
    L.off_progress = 256;
    L.off_ring = L.off_progress + align256((size_t)(g.nstrips > 0 ? g.nstrips : 1) * 8);
    L.off_masks = L.off_ring + align256((size_t)g.ring * (size_t)(g.rowlen > 0 ? g.rowlen : 1) * elt);
    if (L.kernel == LCS_KERNEL_BITS) {
        L.off_final = L.off_masks + align256((size_t)256 * (size_t)(g.rowlen > 0 ? g.rowlen : 1) * 8);
        L.off_counts = L.off_final + align256((size_t)(g.rowlen > 0 ? g.rowlen : 1) * 8);
        L.total = L.off_counts + align256((size_t)(g.rowlen + 1) * 4);
    } else {
        L.off_final = L.off_counts = L.off_masks;
        L.total = L.off_masks;
    }
    return STENCIL_OK;
}

}  // namespace

}  // namespace gbst

using namespace gbst;

extern "C" {

int lcs_workspace_bytes(int64_t na, int64_t nb, int kernel, size_t* bytes)
{
    if (!bytes || na < 0 || nb < 0 || na > LCS_MAX_LEN || nb > LCS_MAX_LEN) return STENCIL_EINVAL;
    if (kernel != LCS_KERNEL_AUTO && kernel != LCS_KERNEL_DP && kernel != LCS_KERNEL_BITS) return STENCIL_EINVAL;
    LcsLayout L;
    lcs_layout(na, nb, kernel, L);
    *bytes = L.total;
    return STENCIL_OK;
}

int lcs_run(const uint8_t* A, int64_t na, const uint8_t* B, int64_t nb, int32_t* row, int kernel, void* workspace,
            void* cuda_stream)
{
    if (na < 0 || nb < 0 || na > LCS_MAX_LEN || nb > LCS_MAX_LEN || !row) return STENCIL_EINVAL;
    if ((na > 0 && !A) || (nb > 0 && !B)) return STENCIL_EINVAL;
    if (kernel != LCS_KERNEL_AUTO && kernel != LCS_KERNEL_DP && kernel != LCS_KERNEL_BITS) return STENCIL_EINVAL;
    if (workspace && ((uintptr_t)workspace & 15)) return STENCIL_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (na == 0 || nb == 0) return cuda_rc(cudaMemsetAsync(row, 0, (size_t)(nb + 1) * sizeof(int32_t), st));
    LcsLayout L;
    lcs_layout(na, nb, kernel, L);
    bool owned = false;
    if (!workspace) {
        if (cudaMallocAsync(&workspace, L.total, st) != cudaSuccess) {
            cudaGetLastError();
            return STENCIL_ENOMEM;
        }
        owned = true;
    }
    char* ws = (char*)workspace;
    LcsHeader* hdr = (LcsHeader*)ws;
    unsigned long long* progress = (unsigned long long*)(ws + L.off_progress);
    int rc = cuda_rc(cudaMemsetAsync(ws, 0, L.off_ring, st));  // ticket, status, progress words
    const unsigned nblk = (unsigned)(L.warps / LCS_WARPS_PER_CTA);
    if (rc == STENCIL_OK && L.kernel == LCS_KERNEL_DP) {
        rc = cuda_rc(cudaMemsetAsync(row, 0, sizeof(int32_t), st));
        if (rc == STENCIL_OK) {
            k_lcs_dp<<<nblk, 32 * LCS_WARPS_PER_CTA, 0, st>>>(A, B, L.g, (int32_t*)(ws + L.off_ring), row, progress,
                                                              hdr);
            g_launches++;
            rc = cuda_rc(cudaGetLastError());
        }
    } else if (rc == STENCIL_OK) {
        const int64_t nw = L.g.rowlen;
        uint64_t* M = (uint64_t*)(ws + L.off_masks);
        uint64_t* vfinal = (uint64_t*)(ws + L.off_final);
        int32_t* counts = (int32_t*)(ws + L.off_counts);
        const int64_t mblk = (256 * nw + 255) / 256;
        k_lcs_masks<<<(unsigned)(mblk < 152 * 32 ? mblk : 152 * 32), 256, 0, st>>>(B, nb, nw, M);
        k_lcs_bits<LCS_BITS_Q><<<nblk, 32 * LCS_WARPS_PER_CTA, 0, st>>>(A, M, L.g, (uint64_t*)(ws + L.off_ring),
                                                                          vfinal, progress, hdr);
        const int64_t cblk = (nw + 255) / 256;
        k_lcs_count<<<(unsigned)(cblk < 152 * 32 ? cblk : 152 * 32), 256, 0, st>>>(vfinal, nb, nw, counts);
        k_lcs_scan<<<1, 1024, 0, st>>>(counts, nw);
        const int64_t rblk = (nb + 1 + 255) / 256;
        k_lcs_row<<<(unsigned)(rblk < 152 * 32 ? rblk : 152 * 32), 256, 0, st>>>(vfinal, counts, nb, nw, row);
        g_launches += 5;
        rc = cuda_rc(cudaGetLastError());
    }
    if (owned) {
        int s = 0;
        if (rc == STENCIL_OK) {
            rc = cuda_rc(cudaMemcpyAsync(&s, &hdr->status, sizeof(int), cudaMemcpyDeviceToHost, st));
            if (rc == STENCIL_OK) rc = cuda_rc(cudaStreamSynchronize(st));
        }
        cudaFreeAsync(workspace, st);
        if (rc == STENCIL_OK && s != LCS_DEV_OK) rc = STENCIL_ETIMEOUT;
    }
    return rc;
}

int lcs_status(void* workspace, void* cuda_stream)
{
    if (!workspace) return STENCIL_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) return STENCIL_ECUDA;
    LcsHeader* hdr = (LcsHeader*)workspace;
    int s = 0;
    if (cudaMemcpy(&s, &hdr->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return STENCIL_ECUDA;
    if (s != LCS_DEV_OK && cudaMemset(&hdr->status, 0, sizeof(int)) != cudaSuccess) return STENCIL_ECUDA;
    return s == LCS_DEV_OK ? STENCIL_OK : STENCIL_ETIMEOUT;
}

}  // extern "C"
