// Game of Life (Section 3.4, "Game of life"): a 2D Jacobi stencil over the
// 3 x 3 box on 0/1 cells, here on bit-packed grids.
//
// Layout: 32 cells per 32-bit word, bit b of word w of row i = cell
// (i, 32 w + b); rows of W = ceil(n1 / 32) words; the bits of the last word
// beyond n1 are kept 0. An 8000^2 grid is 8 MB, so both packed grids stay in
// L2 for the whole run.
//
// Per word, the 8 neighbour bits of its 32 cells are word-wide vectors: for a
// row with words L, C, R around the cell word C, the west neighbours are
// (C << 1) | (L >> 31) and the east neighbours (C >> 1) | (R << 31), one
// funnel shift each. Their sum (0..8) is formed in four bit planes by a tree
// of full adders (sum = a ^ b ^ c, carry = majority(a, b, c): one 3-input
// logic instruction each), and the birth/survival rule reads the planes:
// B2S23 and B3S23 in one or two logic instructions, any other rule through
// the nine count masks. About 20 integer instructions per 32 cells and step.
//
// Kernels: k_life_pack / k_life_unpack convert between bytes and words (one
// warp ballot per word). k_life_step advances one step (each thread walks a
// column of rows with a three-row window in registers). k_life_blocked
// advances tb steps per launch: a CTA stages a tile with tb halo rows and one
// halo word on each side in shared memory, runs tb steps there (the valid
// region shrinks by a row per step; a halo word covers 32 cells, so
// tb <= 32) and writes its interior back: the overlapped temporal tiles the
// FP64 Jacobi kernel uses, on an integer stencil.
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "life.h"
#include "internal.h"

namespace gbst {

namespace {

constexpr unsigned FULLMASK = 0xffffffffu;
constexpr int LIFE_ROWS = 8;       // rows per thread in k_life_step
constexpr int LIFE_MAX_TB = 32;    // one halo word of 32 cells bounds the steps per launch
constexpr int LIFE_THREADS = 256;  // threads per CTA of k_life_blocked

enum { RULE_B2S23 = 0, RULE_B3S23 = 1, RULE_ANY = 2 };

struct LifeGeo {
    int64_t n0, n1, W;   // rows, cells per row, words per row
    int bc;
    int m;               // valid bits in the last word of a row (1..32)
    uint32_t last_mask;  // mask of those bits
};

__device__ __forceinline__ void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t& s, uint32_t& cy)
{
    s = a ^ b ^ c;
    cy = (a & b) | (c & (a ^ b));
}

// New state of the 32 cells of a word from the west/centre/east vectors of
// the rows above (a*) and below (b*), the west/east vectors of its own row
// and its current cells.
template <int RULE>
__device__ __forceinline__ uint32_t life_word(uint32_t aw, uint32_t ac, uint32_t ae, uint32_t mw, uint32_t me,
                                              uint32_t alive, uint32_t bw, uint32_t bc, uint32_t be,
                                              uint32_t birth, uint32_t survive)
{
    uint32_t sa, ca, sb, cb;
    full_add(aw, ac, ae, sa, ca);
    full_add(bw, bc, be, sb, cb);
    const uint32_t sm = mw ^ me, cm = mw & me;
    uint32_t x0, k1, y1, k2;
    full_add(sa, sb, sm, x0, k1);  // x0: weight 1; k1: weight 2
    full_add(ca, cb, cm, y1, k2);  // y1: weight 2; k2: weight 4
    const uint32_t z1 = k1 ^ y1, k2b = k1 & y1;
    const uint32_t b2 = k2 ^ k2b, b3 = k2 & k2b;  // count = x0 + 2 z1 + 4 b2 + 8 b3
    if (RULE == RULE_B2S23) return z1 & ~b2 & (~x0 | alive);  // count 2, or count 3 and live (8 has z1 = 0)
    if (RULE == RULE_B3S23) return z1 & ~b2 & (x0 | alive);   // count 3, or count 2 and live
    uint32_t out = 0;
#pragma unroll
    for (int n = 0; n <= 8; ++n) {
        const uint32_t e = ((n & 1) ? x0 : ~x0) & ((n & 2) ? z1 : ~z1) & ((n & 4) ? b2 : ~b2) & ((n & 8) ? b3 : ~b3);
        if ((birth >> n) & 1u) out |= e & ~alive;
        if ((survive >> n) & 1u) out |= e & alive;
    }
    return out;
}

// West and east neighbour vectors of a word c with left word l and right word r.
__device__ __forceinline__ uint32_t west_of(uint32_t l, uint32_t c) { return __funnelshift_l(l, c, 1); }
__device__ __forceinline__ uint32_t east_of(uint32_t c, uint32_t r) { return __funnelshift_r(c, r, 1); }

// ---------------------------------------------------------------- packing ---

// One warp per word: lane l reads cell 32 w + l of its row (32 consecutive bytes), one ballot.
__global__ void k_life_pack(const uint8_t* __restrict__ cells, uint32_t* __restrict__ bits, LifeGeo g)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = g.n0 * g.W;
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < total; q += nwarps) {
        const int64_t i = q / g.W, w = q - (q / g.W) * g.W;
        const int64_t j = w * 32 + lane;
        const bool v = j < g.n1 && cells[i * g.n1 + j] != 0;
        const unsigned word = __ballot_sync(FULLMASK, v);
        if (lane == 0) bits[q] = word;
    }
}

__global__ void k_life_unpack(const uint32_t* __restrict__ bits, uint8_t* __restrict__ cells, LifeGeo g)
{
    const int64_t total = g.n0 * g.n1;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = p / g.n1, j = p - (p / g.n1) * g.n1;
        cells[p] = (uint8_t)((bits[i * g.W + (j >> 5)] >> (j & 31)) & 1u);
    }
}

// -------------------------------------------------------------- one step ---

// West / centre / east vectors of row i at word w under the boundary rule.
__device__ __forceinline__ void row_vectors(const uint32_t* __restrict__ a, const LifeGeo& g, int64_t i, int64_t w,
                                            uint32_t& vw, uint32_t& vc, uint32_t& ve)
{
    if (i < 0 || i >= g.n0) {
        if (g.bc == BC_CONSTANT) {
            vw = vc = ve = 0;
            return;
        }
        i = i < 0 ? i + g.n0 : i - g.n0;
    }
    const uint32_t* r = a + i * g.W;
    const uint32_t c = __ldg(r + w);
    uint32_t l = 0, rr = 0, extra = 0;
    if (w > 0)
        l = __ldg(r + w - 1);
    else if (g.bc == BC_PERIODIC)
        l = __ldg(r + g.W - 1) << (32 - g.m);  // bit 31 = cell n1 - 1
    if (w < g.W - 1)
        rr = __ldg(r + w + 1);
    else if (g.bc == BC_PERIODIC)
        extra = (__ldg(r) & 1u) << (g.m - 1);  // cell 0, east of cell n1 - 1 (bit m - 1)
    vw = west_of(l, c);
    vc = c;
    ve = east_of(c, rr) | extra;
}

template <int RULE>
__global__ void __launch_bounds__(256) k_life_step(const uint32_t* __restrict__ a, uint32_t* __restrict__ b, LifeGeo g,
                                                   uint32_t birth, uint32_t survive)
{
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= g.W) return;
    const uint32_t keep = w == g.W - 1 ? g.last_mask : FULLMASK;
    const int64_t stride = (int64_t)gridDim.y * blockDim.y * LIFE_ROWS;
    for (int64_t i0 = ((int64_t)blockIdx.y * blockDim.y + threadIdx.y) * LIFE_ROWS; i0 < g.n0; i0 += stride) {
        uint32_t aw, ac, ae, mw, mc, me;
        row_vectors(a, g, i0 - 1, w, aw, ac, ae);
        row_vectors(a, g, i0, w, mw, mc, me);
#pragma unroll
        for (int r = 0; r < LIFE_ROWS; ++r) {
            const int64_t i = i0 + r;
            if (i >= g.n0) break;
            uint32_t bw, bc, be;
            row_vectors(a, g, i + 1, w, bw, bc, be);
            b[i * g.W + w] = life_word<RULE>(aw, ac, ae, mw, me, mc, bw, bc, be, birth, survive) & keep;
            aw = mw; ac = mc; ae = me;
            mw = bw; mc = bc; me = be;
        }
    }
}

// ---------------------------------------------------- temporally blocked ---

constexpr int LIFE_TILE_ROWS = 64;  // largest interior rows per tile
constexpr int LIFE_MAX_COLS = 128;  // tile columns (interior words + 2 halo words)

struct LifeTile {
    int tb;      // steps per launch (2..32)
    int tr;      // interior rows per tile
    int tw;      // interior words per tile
    int cols;    // tw + 2: one halo word on each side
    int rows;    // tr + 2 tb
    int stride;  // cols + 2: a zero guard word at each end of a shared-memory row
    int groups;  // row groups per column (threads = cols * groups)
};

// Supports the constant boundary (any n1) and the periodic boundary when n1
// is a multiple of 32 (then a halo word is a whole word of the grid).
template <int RULE>
__global__ void __launch_bounds__(LIFE_THREADS) k_life_blocked(const uint32_t* __restrict__ a,
                                                               uint32_t* __restrict__ b, LifeGeo g, LifeTile t,
                                                               uint32_t birth, uint32_t survive)
{
    extern __shared__ uint32_t smem[];
    const int64_t ntr = (g.n0 + t.tr - 1) / t.tr;
    const int64_t tj = blockIdx.x;
    const int64_t gw0 = tj * t.tw - 1;  // grid word of tile column 0
    const int nthr = blockDim.x;
    const int col = threadIdx.x % t.cols;
    const int grp = threadIdx.x / t.cols;
    const bool worker = grp < t.groups;
    const int64_t gw = gw0 + col;
    const bool wvalid = g.bc == BC_PERIODIC || (gw >= 0 && gw < g.W);
    const uint32_t keep = !wvalid ? 0u : (g.bc == BC_CONSTANT && gw == g.W - 1 ? g.last_mask : FULLMASK);
    const int plane = t.rows * t.stride;
    for (int64_t ti = blockIdx.y; ti < ntr; ti += gridDim.y) {
        const int64_t gi0 = ti * t.tr - t.tb;  // grid row of tile row 0
        // stage the tile and its halo into buffer 0; out-of-grid rows and words are dead (constant)
        // or wrapped (periodic); the guard words of both buffers are zero
        for (int q = threadIdx.x; q < t.rows * t.stride; q += nthr) {
            const int r = q / t.stride, sc = q - (q / t.stride) * t.stride;
            uint32_t v = 0;
            if (sc >= 1 && sc <= t.cols) {
                int64_t i = gi0 + r, w = gw0 + sc - 1;
                if (g.bc == BC_PERIODIC) {
                    i = ((i % g.n0) + g.n0) % g.n0;
                    w = ((w % g.W) + g.W) % g.W;
                    v = __ldg(a + i * g.W + w);
                } else if (i >= 0 && i < g.n0 && w >= 0 && w < g.W) {
                    v = __ldg(a + i * g.W + w);
                }
            } else {
                smem[plane + q] = 0;
            }
            smem[q] = v;
        }
        // tile rows inside the grid (the others stay dead under the constant boundary)
        int rlo = 0, rhi = t.rows;
        if (g.bc == BC_CONSTANT) {
            rlo = gi0 < 0 ? (int)(-gi0) : 0;
            rhi = g.n0 - gi0 < t.rows ? (int)(g.n0 - gi0) : t.rows;
        }
        __syncthreads();
        // 32-bit offsets into the shared array keep every access a plain shared-memory load/store
        int src = 0, dst = plane;
        for (int s = 1; s <= t.tb; ++s) {
            const int lo = s, hi = t.rows - s;  // rows valid after step s: [lo, hi)
            const int per = (hi - lo + t.groups - 1) / t.groups;
            const int r0 = lo + grp * per;
            const int r1 = r0 + per < hi ? r0 + per : hi;
            if (worker && r0 < r1) {
                int o = src + (r0 - 1) * t.stride + col + 1;
                uint32_t aw = west_of(smem[o - 1], smem[o]), ac = smem[o], ae = east_of(smem[o], smem[o + 1]);
                o += t.stride;
                uint32_t mw = west_of(smem[o - 1], smem[o]), mc = smem[o], me = east_of(smem[o], smem[o + 1]);
                int od = dst + r0 * t.stride + col + 1;
#pragma unroll 2
                for (int r = r0; r < r1; ++r) {
                    o += t.stride;
                    const uint32_t bw = west_of(smem[o - 1], smem[o]), bcv = smem[o], be = east_of(smem[o], smem[o + 1]);
                    const uint32_t nv = life_word<RULE>(aw, ac, ae, mw, me, mc, bw, bcv, be, birth, survive);
                    smem[od] = (r >= rlo && r < rhi) ? (nv & keep) : 0u;
                    od += t.stride;
                    aw = mw; ac = mc; ae = me;
                    mw = bw; mc = bcv; me = be;
                }
            }
            __syncthreads();
            const int tmp = src;
            src = dst;
            dst = tmp;
        }
        // write the interior
        for (int q = threadIdx.x; q < t.tr * t.tw; q += nthr) {
            const int r = q / t.tw, cc = q - (q / t.tw) * t.tw;
            const int64_t i = ti * t.tr + r, w = tj * t.tw + cc;
            if (i < g.n0 && w < g.W) b[i * g.W + w] = smem[src + (r + t.tb) * t.stride + cc + 2];
        }
        __syncthreads();  // the next tile's staging overwrites the buffers
    }
}

// ------------------------------------------------------------------- host ---

LifeGeo make_life_geo(const int64_t ext[2], int bc)
{
    LifeGeo g;
    g.n0 = ext[0];
    g.n1 = ext[1];
    g.W = (ext[1] + 31) / 32;
    g.bc = bc;
    g.m = (int)(ext[1] - (g.W - 1) * 32);
    g.last_mask = g.m == 32 ? FULLMASK : ((1u << g.m) - 1u);
    return g;
}

size_t packed_bytes(const LifeGeo& g) { return ((size_t)(g.n0 * g.W) * 4 + 255) & ~size_t(255); }

int rule_kind(uint32_t birth, uint32_t survive)
{
    if (birth == (1u << 2) && survive == ((1u << 2) | (1u << 3))) return RULE_B2S23;
    if (birth == (1u << 3) && survive == ((1u << 2) | (1u << 3))) return RULE_B3S23;
    return RULE_ANY;
}

// Tile shape: as few tile columns as fit LIFE_MAX_COLS, the words split evenly among them; tr
// interior rows.
LifeTile make_tile(const LifeGeo& g, int tb, int tr)
{
    LifeTile t;
    t.tb = tb;
    const int64_t nt = (g.W + (LIFE_MAX_COLS - 2) - 1) / (LIFE_MAX_COLS - 2);
    t.tw = (int)((g.W + nt - 1) / nt);
    t.cols = t.tw + 2;
    t.stride = t.cols + 2;
    t.tr = tr;
    t.rows = t.tr + 2 * tb;
    t.groups = LIFE_THREADS / t.cols;
    return t;
}

template <int RULE>
int life_steps(const LifeGeo& g, uint32_t*& a, uint32_t*& b, int64_t T, int tb, uint32_t birth, uint32_t survive,
               cudaStream_t st)
{
    const bool blocked_ok = g.bc == BC_CONSTANT || g.m == 32;
    int64_t t = 0;
    if (tb > 1 && blocked_ok) {
        const int tbc = tb > LIFE_MAX_TB ? LIFE_MAX_TB : tb;
        LifeTile tl = make_tile(g, tbc, LIFE_TILE_ROWS);
        size_t smem = 2 * (size_t)tl.rows * tl.stride * sizeof(uint32_t);
        if (smem > 227 * 1024) return STENCIL_EUNSUPPORTED;
        if (cudaFuncSetAttribute(k_life_blocked<RULE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) !=
            cudaSuccess)
            return STENCIL_ECUDA;
        // Tile height: the tiles of one pass fill whole waves of resident CTAs, so that no SM runs
        // two tiles while another idles (a pass costs as much as its busiest SM).
        int dev = 0, nsm = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_life_blocked<RULE>, LIFE_THREADS, smem);
        const int64_t ntc = (g.W + tl.tw - 1) / tl.tw;
        const int64_t row_tiles_per_wave = (int64_t)nsm * (per_sm > 0 ? per_sm : 1) / ntc;
        if (row_tiles_per_wave > 0) {
            const int64_t waves = (g.n0 + LIFE_TILE_ROWS * row_tiles_per_wave - 1) / (LIFE_TILE_ROWS * row_tiles_per_wave);
            const int64_t tr = (g.n0 + waves * row_tiles_per_wave - 1) / (waves * row_tiles_per_wave);
            if (tr >= 16 && tr < LIFE_TILE_ROWS) {
                tl = make_tile(g, tbc, (int)tr);
                smem = 2 * (size_t)tl.rows * tl.stride * sizeof(uint32_t);
            }
        }
        const int64_t ntr = (g.n0 + tl.tr - 1) / tl.tr;
        const dim3 grid((unsigned)((g.W + tl.tw - 1) / tl.tw), (unsigned)(ntr < 65535 ? ntr : 65535));
        for (; T - t >= tl.tb; t += tl.tb) {
            k_life_blocked<RULE><<<grid, LIFE_THREADS, smem, st>>>(a, b, g, tl, birth, survive);
            g_launches++;
            if (cudaGetLastError() != cudaSuccess) return STENCIL_ECUDA;
            uint32_t* tmp = a;
            a = b;
            b = tmp;
        }
    }
    int bx = 32;
    while (bx < 128 && bx < g.W) bx *= 2;
    const dim3 block(bx, 256 / bx);
    const int64_t gy = (g.n0 + (int64_t)LIFE_ROWS * block.y - 1) / ((int64_t)LIFE_ROWS * block.y);
    const dim3 grid((unsigned)((g.W + bx - 1) / bx), (unsigned)(gy < 65535 ? gy : 65535));
    for (; t < T; ++t) {
        k_life_step<RULE><<<grid, block, 0, st>>>(a, b, g, birth, survive);
        g_launches++;
        if (cudaGetLastError() != cudaSuccess) return STENCIL_ECUDA;
        uint32_t* tmp = a;
        a = b;
        b = tmp;
    }
    return STENCIL_OK;
}

}  // namespace

}  // namespace gbst

using namespace gbst;

extern "C" {

int life_workspace_bytes(const int64_t ext[2], size_t* bytes)
{
    if (!ext || !bytes || ext[0] < 1 || ext[1] < 1) return STENCIL_EINVAL;
    if (ext[0] > ((int64_t)1 << 40) / ext[1]) return STENCIL_EINVAL;
    *bytes = 2 * packed_bytes(make_life_geo(ext, BC_CONSTANT));
    return STENCIL_OK;
}

int life_run(uint8_t* cells, const int64_t ext[2], int boundary, uint32_t birth_mask, uint32_t survive_mask, int64_t T,
             int tb, void* workspace, void* cuda_stream)
{
    if (!cells || !ext || T < 0 || tb < 0 || birth_mask > 0x1FFu || survive_mask > 0x1FFu) return STENCIL_EINVAL;
    if (boundary != STENCIL_BC_CONSTANT && boundary != STENCIL_BC_PERIODIC) return STENCIL_EINVAL;
    size_t ws_bytes = 0;
    int rc = life_workspace_bytes(ext, &ws_bytes);
    if (rc) return rc;
    if (boundary == STENCIL_BC_PERIODIC && (ext[0] < 3 || ext[1] < 3)) return STENCIL_EINVAL;
    if (workspace && ((uintptr_t)workspace & 15)) return STENCIL_EINVAL;
    if (T == 0) return STENCIL_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const LifeGeo g = make_life_geo(ext, boundary);
    bool owned = false;
    if (!workspace) {
        if (cudaMallocAsync(&workspace, ws_bytes, st) != cudaSuccess) {
            cudaGetLastError();
            return STENCIL_ENOMEM;
        }
        owned = true;
    }
    uint32_t* a = (uint32_t*)workspace;
    uint32_t* b = (uint32_t*)((char*)workspace + packed_bytes(g));
    const int64_t pack_blocks = (g.n0 * g.W + 7) / 8;
    k_life_pack<<<(unsigned)(pack_blocks < 152 * 16 ? pack_blocks : 152 * 16), 256, 0, st>>>(cells, a, g);
    g_launches++;
    rc = cuda_rc(cudaGetLastError());
    if (tb == 0) tb = 16;
    if (rc == STENCIL_OK) {
        switch (rule_kind(birth_mask, survive_mask)) {
            case RULE_B2S23: rc = life_steps<RULE_B2S23>(g, a, b, T, tb, birth_mask, survive_mask, st); break;
            case RULE_B3S23: rc = life_steps<RULE_B3S23>(g, a, b, T, tb, birth_mask, survive_mask, st); break;
            default: rc = life_steps<RULE_ANY>(g, a, b, T, tb, birth_mask, survive_mask, st); break;
        }
    }
    if (rc == STENCIL_OK) {
        const int64_t unpack_blocks = (g.n0 * g.n1 + 255) / 256;
        k_life_unpack<<<(unsigned)(unpack_blocks < 152 * 32 ? unpack_blocks : 152 * 32), 256, 0, st>>>(a, cells, g);
        g_launches++;
        rc = cuda_rc(cudaGetLastError());
    }
    if (owned) cudaFreeAsync(workspace, st);
    return rc;
}

}  // extern "C"
