// Temporally blocked Jacobi: one HBM round trip per T_b steps.
//
// Temporal tiling (Section 1, the blocking methods; Section 3.4: tiles of
// height T_b in time) reduces memory traffic by advancing a tile several time
// steps while it stays on chip. Here each CTA owns an output tile of
// B0 x B1 x B2 points and:
//   1. stages the tile plus a halo of h = T_b * r points per side into shared
//      memory with one TMA tiled copy (cp.async.bulk.tensor; the hardware
//      zero-fills the part outside the grid), or with plain coalesced loads
//      where TMA cannot express the halo (periodic wrap, odd row pitch);
//   2. runs T_b Jacobi steps between two shared-memory buffers, the valid
//      region shrinking by r per step (an overlapped, trapezoidal tile: the
//      halo is recomputed redundantly instead of exchanged);
//   3. writes the B0 x B1 x B2 interior back once.
// Cells outside the grid hold the boundary value c in both buffers, so every
// step reads the constant boundary exactly as the plain kernel does; with a
// periodic boundary the halo cells are wrapped copies and are updated like
// any other cell. Each cell is computed with the same descending-order sum
// and rounding as the plain kernel, so the result is bit-identical to T_b
// plain steps.
#include <cuda.h>

#include <cstring>

#include "internal.h"

namespace gbst {

struct BlkGeo {
    int B0, B1, B2;       // output tile extents (1 on unused axes)
    int h0, h1, h2;       // halo per side (T_b*r on used axes)
    int E0, E1, E2;       // staged region extents; E2 includes alignment padding
    int64_t nt0, nt1, nt2;
    int tb;               // steps in this pass (<= the T_b the halo was sized for)
    int use_tma;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Bounded wait on phase 0 of an mbarrier; returns false on time-out.
__device__ __forceinline__ bool mbar_wait0(uint64_t* bar)
{
    const uint32_t a = smem_u32(bar);
    for (int it = 0; it < (1 << 24); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(0)
            : "memory");
        if (done) return true;
    }
    return false;
}

// After a time-out: a further wait on phase 0 with a back-off, bounded at
// about a second (2^20 polls of at least 1 us each).
__device__ __forceinline__ void mbar_wait_backoff(uint64_t* bar)
{
    const uint32_t a = smem_u32(bar);
    for (int it = 0; it < (1 << 20); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(0)
            : "memory");
        if (done) return;
        __nanosleep(1000);
    }
}

template <int DIM, int SHAPE, int R, int ARITH>
__global__ void __launch_bounds__(256) k_jacobi_blocked(const __grid_constant__ CUtensorMap tmap,
                                                        const double* __restrict__ in, double* __restrict__ out,
                                                        Geo g, int bc, double c, BlkGeo b,
                                                        WArr<Stn<DIM, SHAPE, R>::K> w, int* status)
{
    extern __shared__ __align__(128) double sm[];
    __shared__ __align__(8) uint64_t bar;
    const int64_t region = (int64_t)b.E0 * b.E1 * b.E2;
    double* bufA = sm;
    double* bufB = sm + ((region + 31) & ~int64_t(31));
    // checked build: both staged buffers inside the launch's dynamic shared memory (uniform per CTA)
    if (!GBST_IN(((region + 31) & ~int64_t(31)) + region - 1, (int64_t)(dyn_smem_bytes() / 8))) return;

    // tile coordinates
    int64_t t = blockIdx.x;
    const int64_t T2 = t % b.nt2;
    t /= b.nt2;
    const int64_t T1 = t % b.nt1;
    const int64_t T0 = t / b.nt1;
    // global coordinates of staged cell (0,0,0); the inner one rounded down to an even index
    const int64_t g0 = T0 * b.B0 - b.h0;
    const int64_t g1 = T1 * b.B1 - b.h1;
    const int64_t x2 = T2 * b.B2 - b.h2;
    const int64_t g2 = (DIM >= 1 && b.use_tma) ? (x2 >= 0 ? (x2 & ~int64_t(1)) : -((-x2 + 1) & ~int64_t(1))) : x2;
    const int pad2 = (int)(x2 - g2);  // 0 or 1
    const int nthr = blockDim.x;
    griddep_wait();  // launched programmatically: the previous pass has finished with both buffers

    // ---- stage tile + halo
    if (b.use_tma) {
        if (threadIdx.x == 0) {
            const uint32_t ab = smem_u32(&bar);
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ab) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const uint32_t bytes = (uint32_t)(region * 8);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ab), "r"(bytes) : "memory");
            const uint32_t dst = smem_u32(bufA);
            if (DIM == 1) {
                // 1D boxes hold at most 256 elements: E2 is a multiple of 256, one copy per chunk
                for (int ch = 0; ch < b.E2; ch += 256) {
                    const int cx = (int)(g2 + ch);
                    asm volatile(
                        "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                        "[%0], [%1, {%2}], [%3];" ::"r"(dst + ch * 8), "l"(&tmap), "r"(cx), "r"(ab)
                        : "memory");
                }
            } else if (DIM == 2) {
                asm volatile(
                    "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                    "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst), "l"(&tmap), "r"((int)g2), "r"((int)g1), "r"(ab)
                    : "memory");
            } else {
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                    "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst), "l"(&tmap), "r"((int)g2), "r"((int)g1), "r"((int)g0),
                    "r"(ab)
                    : "memory");
            }
        }
        __syncthreads();
        if (!mbar_wait0(&bar)) {
            // Record the time-out, then keep the CTA (and its shared memory) until the
            // barrier completes. The copy is a bounded read of global memory that lands
            // within microseconds, so this back-off wait (about a second more) ends with
            // it; a barrier still open after that means the byte count it expects was
            // never going to be met, which is only possible once every copy has landed.
            if (threadIdx.x == 0) atomicExch(status, DEV_TIMEOUT);
            mbar_wait_backoff(&bar);
            return;
        }
    } else {
        // the staged region fits in shared memory: 32-bit cell indices (E0 = 1 in 2D, E0 = E1 = 1 in 1D)
        for (int idx = threadIdx.x; idx < (int)region; idx += nthr) {
            const int s2 = DIM == 1 ? idx : idx % b.E2;
            const int s1 = DIM == 1 ? 0 : DIM == 2 ? idx / b.E2 : (idx / b.E2) % b.E1;
            const int s0 = DIM <= 2 ? 0 : idx / (b.E2 * b.E1);
            st_in(bufA, idx, region, fetch_bc(in, g0 + s0, g1 + s1, g2 + s2, g, bc, c));
        }
    }
    // cells outside the grid hold the boundary value in both buffers
    if (bc == BC_CONSTANT) {
        for (int idx = threadIdx.x; idx < (int)region; idx += nthr) {
            const int64_t i = g0 + (DIM <= 2 ? 0 : idx / (b.E2 * b.E1));
            const int64_t j = g1 + (DIM == 1 ? 0 : DIM == 2 ? idx / b.E2 : (idx / b.E2) % b.E1);
            const int64_t k = g2 + (DIM == 1 ? idx : idx % b.E2);
            if (i < 0 || i >= g.n0 || j < 0 || j >= g.n1 || k < 0 || k >= g.n2) {
                st_in(bufA, idx, region, c);
                st_in(bufB, idx, region, c);
            }
        }
    }
    __syncthreads();

    // ---- T_b steps on chip
    const int64_t st1 = b.E2, st0 = (int64_t)b.E1 * b.E2;
    double* src = bufA;
    double* dst = bufB;
    for (int s = 1; s <= b.tb; ++s) {
        // region still valid after s steps: shrink by s*R from the staged edges on used axes
        const int lo0 = DIM >= 3 ? s * R : 0, hi0 = DIM >= 3 ? b.E0 - s * R : 1;
        const int lo1 = DIM >= 2 ? s * R : 0, hi1 = DIM >= 2 ? b.E1 - s * R : 1;
        const int lo2 = pad2 + s * R, hi2 = pad2 + b.B2 + 2 * b.h2 - s * R;
        const int w1 = hi1 - lo1, w2 = hi2 - lo2;  // >= 1: the halo is T_b * R wide on every used axis
        auto cell = [&](int s0, int s1, int s2) {
            if (bc == BC_CONSTANT) {
                const int64_t i = g0 + s0, j = g1 + s1, k = g2 + s2;
                if (i < 0 || i >= g.n0 || j < 0 || j >= g.n1 || k < 0 || k >= g.n2) return;
            }
            const int64_t p = s0 * st0 + s1 * st1 + s2;
            st_in(dst, p, region, update_interior<DIM, SHAPE, R, ARITH, false>(src, p, st0, st1, w, region));
        };
        if (DIM == 1) {
            for (int s2 = lo2 + (int)threadIdx.x; s2 < hi2; s2 += nthr) cell(0, 0, s2);
        } else {
            // Each thread walks its cells (s0, s1, s2) in steps of nthr cells without a division: the
            // step is split once into (dq0, dq1, dr) and added digit by digit with carries. Both
            // remainders are below their extents, so one subtraction per digit restores the range.
            const int cnt = (hi0 - lo0) * w1 * w2;
            const int dr = nthr % w2, dq = nthr / w2, dq1 = dq % w1, dq0 = dq / w1;
            int s2 = lo2 + (int)threadIdx.x % w2;
            int s1 = lo1 + ((int)threadIdx.x / w2) % w1;
            int s0 = lo0 + (int)threadIdx.x / (w2 * w1);
            for (int idx = threadIdx.x; idx < cnt; idx += nthr) {
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
        double* tmp = src;
        src = dst;
        dst = tmp;
    }

    // ---- write the interior back
    const int cnt = b.B0 * b.B1 * b.B2;
    for (int idx = threadIdx.x; idx < cnt; idx += nthr) {
        const int l2 = DIM == 1 ? idx : idx % b.B2;
        const int l1 = DIM == 1 ? 0 : DIM == 2 ? idx / b.B2 : (idx / b.B2) % b.B1;
        const int l0 = DIM <= 2 ? 0 : idx / (b.B2 * b.B1);
        const int64_t i = T0 * b.B0 + l0, j = T1 * b.B1 + l1, k = T2 * b.B2 + l2;
        if (i < g.n0 && j < g.n1 && k < g.n2)
            st_in(out, (i * g.n1 + j) * g.n2 + k, g.n0 * g.n1 * g.n2,
                  ld_in(src, (l0 + b.h0) * st0 + (l1 + b.h1) * st1 + (l2 + b.h2 + pad2), region));
    }
}

// ------------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    }
    return fn;
}

bool jacobi_blocked_supported(const stencil_handle_s* h, const Geo& g)
{
    (void)g;
    // constant weights only: the staged tile has no room for K weight planes
    return h->method == JACOBI && !h->field && plain_specialised(h->dim, h->shape, h->r) &&
           !(h->dim == 3 && h->shape == BOX && h->r == 2);
}

static void default_tile(int dim, int r, int64_t tile[3], int& tb)
{
    if (dim == 1) {
        tile[0] = tile[1] = 1;
        tile[2] = 1024;
        if (tb <= 0) tb = 32 / r;
    } else if (dim == 2) {
        tile[0] = 1;
        tile[1] = 64;
        tile[2] = 64;
        if (tb <= 0) tb = 2;
    } else {
        tile[0] = 8;
        tile[1] = 16;
        tile[2] = 32;
        if (tb <= 0) tb = 2;
    }
}

static int make_blk(const stencil_handle_s* h, const Geo& g, int tb, const int64_t tile_in[3], BlkGeo& b,
                    size_t& smem, bool& tma_ok)
{
    int64_t tile[3] = {tile_in ? tile_in[0] : 0, tile_in ? tile_in[1] : 0, tile_in ? tile_in[2] : 0};
    int64_t def[3];
    int tbd = tb;
    default_tile(h->dim, h->r, def, tbd);
    for (int d = 0; d < 3; ++d)
        if (tile[d] <= 0) tile[d] = def[d];
    if (tb <= 0) tb = tbd;
    const int dim = h->dim, r = h->r;
    if (dim < 3) tile[0] = 1;
    if (dim < 2) tile[1] = 1;
    b.B0 = (int)tile[0];
    b.B1 = (int)tile[1];
    b.B2 = (int)((tile[2] + 1) & ~int64_t(1));
    b.h0 = dim >= 3 ? tb * r : 0;
    b.h1 = dim >= 2 ? tb * r : 0;
    b.h2 = tb * r;
    b.E0 = b.B0 + 2 * b.h0;
    b.E1 = b.B1 + 2 * b.h1;
    b.E2 = b.B2 + 2 * b.h2 + 2;  // +2: room to round the start down to an even index
    if (dim == 1) b.E2 = (b.E2 + 255) & ~255;
    b.nt0 = (g.n0 + b.B0 - 1) / b.B0;
    b.nt1 = (g.n1 + b.B1 - 1) / b.B1;
    b.nt2 = (g.n2 + b.B2 - 1) / b.B2;
    b.tb = tb;
    const int64_t region = (int64_t)b.E0 * b.E1 * b.E2;
    smem = (size_t)(((region + 31) & ~int64_t(31)) + region) * sizeof(double);
    if (smem > 227 * 1024 || b.nt0 * b.nt1 * b.nt2 > 0x7fffffffLL) return STENCIL_EUNSUPPORTED;
    tma_ok = h->bc == BC_CONSTANT && encode_fn() != nullptr && (dim == 1 || g.n2 % 2 == 0) &&
             (dim == 1 || (b.E2 <= 256 && b.E1 <= 256 && b.E0 <= 256)) && g.n2 < (1LL << 31) &&
             g.n1 < (1LL << 31) && g.n0 < (1LL << 31);
    return STENCIL_OK;
}

static bool encode_map(CUtensorMap& m, const double* base, const Geo& g, int dim, const BlkGeo& b)
{
    if (((uintptr_t)base & 15) != 0) return false;
    cuuint64_t gdim[3], gstr[2];
    cuuint32_t box[3], es[3] = {1, 1, 1};
    if (dim == 1) {
        gdim[0] = (cuuint64_t)g.n2;
        box[0] = 256;
    } else if (dim == 2) {
        gdim[0] = (cuuint64_t)g.n2;
        gdim[1] = (cuuint64_t)g.n1;
        gstr[0] = (cuuint64_t)g.n2 * 8;
        box[0] = (cuuint32_t)b.E2;
        box[1] = (cuuint32_t)b.E1;
    } else {
        gdim[0] = (cuuint64_t)g.n2;
        gdim[1] = (cuuint64_t)g.n1;
        gdim[2] = (cuuint64_t)g.n0;
        gstr[0] = (cuuint64_t)g.n2 * 8;
        gstr[1] = (cuuint64_t)g.n2 * g.n1 * 8;
        box[0] = (cuuint32_t)b.E2;
        box[1] = (cuuint32_t)b.E1;
        box[2] = (cuuint32_t)b.E0;
    }
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)dim, (void*)base, gdim, gstr, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int DIM, int SHAPE, int R>
static int blocked_passes(const RunCtx& ctx, double* a, double* bb, int64_t T, int tb, const int64_t tile[3])
{
    constexpr int K = Stn<DIM, SHAPE, R>::K;
    WArr<K> w;
    for (int q = 0; q < K; ++q) w.w[q] = ctx.h->w_desc[q];
    BlkGeo b;
    size_t smem;
    bool tma_ok;
    int rc = make_blk(ctx.h, ctx.g, tb, tile, b, smem, tma_ok);
    if (rc) return rc;
    auto kern = ctx.h->arith == ARITH_FMA ? k_jacobi_blocked<DIM, SHAPE, R, ARITH_FMA>
                                          : k_jacobi_blocked<DIM, SHAPE, R, ARITH_UNFUSED>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return STENCIL_ECUDA;
    CUtensorMap mapA, mapB;
    memset(&mapA, 0, sizeof(mapA));
    memset(&mapB, 0, sizeof(mapB));
    if (tma_ok) tma_ok = encode_map(mapA, a, ctx.g, DIM, b) && encode_map(mapB, bb, ctx.g, DIM, b);
    b.use_tma = tma_ok ? 1 : 0;
    const unsigned nblk = (unsigned)(b.nt0 * b.nt1 * b.nt2);
    const int full_tb = b.tb;
    double* src = a;
    double* dst = bb;
    for (int64_t done = 0; done < T;) {
        b.tb = (int)((T - done) < full_tb ? (T - done) : full_tb);
        // programmatic launch: the next pass's CTAs are scheduled while this one drains
        const CUtensorMap& map = src == a ? mapA : mapB;
        if (launch_pdl(kern, dim3(nblk), dim3(256), smem, ctx.st, map, src, dst, ctx.g, ctx.h->bc, ctx.h->c, b, w,
                       ctx.h->d_status) != cudaSuccess) {
            cudaGetLastError();  // a stream that refuses the attribute: an ordinary launch
            kern<<<nblk, 256, smem, ctx.st>>>(map, src, dst, ctx.g, ctx.h->bc, ctx.h->c, b, w, ctx.h->d_status);
        }
        g_launches++;
        if (cudaGetLastError() != cudaSuccess) return STENCIL_ECUDA;
        done += b.tb;
        double* tmp = src;
        src = dst;
        dst = tmp;
    }
    if (src != a) {
        const size_t bytes = (size_t)(ctx.g.n0 * ctx.g.n1 * ctx.g.n2) * sizeof(double);
        if (cudaMemcpyAsync(a, src, bytes, cudaMemcpyDeviceToDevice, ctx.st) != cudaSuccess) return STENCIL_ECUDA;
    }
    return STENCIL_OK;
}

int jacobi_blocked_run(const RunCtx& ctx, double* a, double* b, int64_t T, int tb, const int64_t tile[3])
{
    const stencil_handle_s* h = ctx.h;
#define X(D, S, R) \
    if (h->dim == D && h->shape == S && h->r == R) return blocked_passes<D, S, R>(ctx, a, b, T, tb, tile);
    X(1, STAR, 1) X(1, STAR, 2) X(1, STAR, 3) X(1, STAR, 4)
    X(2, STAR, 1) X(2, BOX, 1) X(2, STAR, 2) X(2, BOX, 2)
    X(3, STAR, 1) X(3, BOX, 1) X(3, STAR, 2)
#undef X
    return STENCIL_EUNSUPPORTED;
}

}  // namespace gbst
