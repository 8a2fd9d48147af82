// Device-side building blocks shared by the stencil kernels.
//
// A stencil point update (Section 1; Algorithm 1) is the weighted sum of the
// neighbours at the canonical offsets, summed in DESCENDING canonical order:
// the offset that is largest lexicographically (slowest dimension first)
// comes first, so that in Gauss-Seidel the newest-value terms (negative
// offsets) come last. Two rounding modes:
//   ARITH_FMA      acc = w0*v0 (rounded), then acc = fma(wq, vq, acc)
//   ARITH_UNFUSED  acc = w0*v0 (rounded), then acc = acc + (wq*vq), each rounded
// The intrinsics __dmul_rn / __fma_rn / __dadd_rn pin every rounding; the
// compiler never contracts them.
//
// Weights come from a weight source: WArr (the same K weights at every point)
// or WField (per-point weights, a variable-coefficient stencil as Section 3.4
// treats LCS's second sequence). Both answer at(q, p), the weight of the q-th
// term in summation order at the point of linear index p.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gbst {

enum { STAR = 0, BOX = 1 };
enum { JACOBI = 0, GAUSS_SEIDEL = 1 };
enum { BC_CONSTANT = 0, BC_PERIODIC = 1 };
enum { ARITH_FMA = 0, ARITH_UNFUSED = 1 };

// Device status word values (mirrored by the C ABI's negative codes).
enum { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BOUNDS = 2 };

// Checked build (compiled with -DSTENCIL_CHECKED into its own library): every
// index the stencil kernels form into a grid, a coefficient field or a staged
// shared-memory tile goes through GBST_IN(i, n), which tests 0 <= i < n. A
// failing test skips the access (a load reads 0), and the first failing index
// is kept in a fault word of the kernel's translation unit; stencil_status
// reads and clears the fault words of every unit and answers STENCIL_EBOUNDS.
// The fault words are process-wide: a fault shows in the next stencil_status
// call, whichever handle it names. In the normal build GBST_IN is the
// constant true and every guarded access compiles to the plain access.
#ifdef STENCIL_CHECKED
static __device__ unsigned long long chk_fault_word;

__device__ __forceinline__ bool chk_in(int64_t i, int64_t n)
{
    if (i >= 0 && i < n) return true;
    // bit 63 marks a fault; the low 62 bits keep the failing index (two's complement, truncated)
    atomicCAS(&chk_fault_word, 0ull, (1ull << 63) | ((unsigned long long)i & ((1ull << 62) - 1)));
    return false;
}
#define GBST_IN(i, n) ::gbst::chk_in((int64_t)(i), (int64_t)(n))

// The library's registry of fault-word readers (abi.cu): each unit adds its own at load time.
void chk_register(unsigned long long (*take)());

static unsigned long long chk_take_fault_word()
{
    unsigned long long v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, chk_fault_word, sizeof(v)) != cudaSuccess) return 0;
    if (v) cudaMemcpyToSymbol(chk_fault_word, &zero, sizeof(zero));
    return v;
}
static const int chk_registered = (chk_register(&chk_take_fault_word), 0);
#else
#define GBST_IN(i, n) true
#endif

// Bytes of dynamic shared memory this CTA was launched with.
__device__ __forceinline__ uint32_t dyn_smem_bytes()
{
    uint32_t v;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

// Guarded element access: a[i] for 0 <= i < n; the checked build tests the index first.
template <class T>
__device__ __forceinline__ T ld_in(const T* a, int64_t i, int64_t n)
{
    return GBST_IN(i, n) ? a[i] : T(0);
}
template <class T>
__device__ __forceinline__ void st_in(T* a, int64_t i, int64_t n, T v)
{
    if (GBST_IN(i, n)) a[i] = v;
}

// Extents padded to three dimensions, slowest first (a 1D grid is 1 x 1 x N).
struct Geo {
    int64_t n0, n1, n2;
};

// Stencil description for kernels that take the offsets at run time.
struct StencilDev {
    int K, r, bc, arith;
    double c;
    const double* w;   // K weights, descending canonical order (device)
    const int* off;    // 3K offset components, descending canonical order (device)
    int* status;       // device status word
    const double* field;  // per-point weights (canonical term-major, K x npts) or nullptr
    int64_t npts;         // points of the grid the field belongs to
};

__host__ __device__ constexpr int stencil_k(int dim, int shape, int r)
{
    return shape == STAR ? 2 * dim * r + 1 : (dim == 1 ? 2 * r + 1 : (dim == 2 ? (2 * r + 1) * (2 * r + 1)
                                                                              : (2 * r + 1) * (2 * r + 1) * (2 * r + 1)));
}

// Component d (0..2, slowest first, padded) of canonical offset q of a star.
// Canonical (lexicographic) order of a star: the negative offsets of each axis
// from the slowest axis to the second fastest, then the fastest axis from -r
// to +r, then the positive offsets from the second fastest axis back to the
// slowest.
__host__ __device__ constexpr int star_off(int dim, int r, int q, int d)
{
    int first = 3 - dim;
    int idx = q;
    for (int a = first; a < 2; ++a) {
        if (idx < r) return d == a ? idx - r : 0;
        idx -= r;
    }
    if (idx < 2 * r + 1) return d == 2 ? idx - r : 0;
    idx -= 2 * r + 1;
    for (int a = 1; a >= first; --a) {
        if (idx < r) return d == a ? idx + 1 : 0;
        idx -= r;
    }
    return 0;
}

// Component d of canonical offset q of a box: q written in base 2r+1, the
// slowest used axis the most significant digit.
__host__ __device__ constexpr int box_off(int dim, int r, int q, int d)
{
    if (d < 3 - dim) return 0;
    int b = 2 * r + 1;
    int v = q;
    for (int i = 0; i < 2 - d; ++i) v /= b;
    return v % b - r;
}

template <int DIM, int SHAPE, int R>
struct Stn {
    static constexpr int K = stencil_k(DIM, SHAPE, R);
    // offset component d of the q-th term in summation (descending) order
    __host__ __device__ static constexpr int o(int q, int d)
    {
        return SHAPE == STAR ? star_off(DIM, R, K - 1 - q, d) : box_off(DIM, R, K - 1 - q, d);
    }
};

template <int K>
struct WArr {
    static constexpr bool per_point = false;
    double w[K];  // descending canonical order
    __device__ __forceinline__ double at(int q, int64_t) const { return w[q]; }
};

// The same weights at every point, read from memory (shared or global).
struct WPtr {
    static constexpr bool per_point = false;
    const double* w;
    __device__ __forceinline__ double at(int q, int64_t) const { return w[q]; }
};

// Per-point weights: f holds K planes of n doubles in CANONICAL term order, so
// the q-th term in summation (descending) order is plane K-1-q. Read through
// the non-coherent path: no kernel writes the field.
template <int K>
struct WField {
    static constexpr bool per_point = true;
    const double* f;
    int64_t n;
    __device__ __forceinline__ double at(int q, int64_t p) const
    {
        return GBST_IN(p, n) ? __ldg(f + (int64_t)(K - 1 - q) * n + p) : 0.0;
    }
};

template <int ARITH>
__device__ __forceinline__ double acc_step(double acc, double w, double v)
{
    if (ARITH == ARITH_FMA) return __fma_rn(w, v, acc);
    return __dadd_rn(acc, __dmul_rn(w, v));
}

__device__ __forceinline__ int64_t wrap_idx(int64_t i, int64_t n)
{
    // |offset| <= r < n for periodic grids, so one correction suffices
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

// Value at (i, j, k) under the boundary rule; u is read with a plain
// (coherent) load so that values written earlier in the same kernel by this
// CTA are seen.
__device__ __forceinline__ double fetch_bc(const double* u, int64_t i, int64_t j, int64_t k, const Geo& g,
                                           int bc, double c)
{
    if (bc == BC_PERIODIC) {
        i = wrap_idx(i, g.n0);
        j = wrap_idx(j, g.n1);
        k = wrap_idx(k, g.n2);
    } else if (i < 0 || i >= g.n0 || j < 0 || j >= g.n1 || k < 0 || k >= g.n2) {
        return c;
    }
    return ld_in(u, (i * g.n1 + j) * g.n2 + k, g.n0 * g.n1 * g.n2);
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialization attribute (launch_pdl) may be scheduled while the
// kernel before it in the stream is still draining its last CTAs, so that its
// own launch latency overlaps that tail. griddepcontrol.wait then holds every
// thread until the previous kernel has completed and its writes are visible;
// such a kernel calls this before it touches memory the previous one may
// write. Without a programmatic predecessor it returns at once.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Full update at (i, j, k) (inside the grid) with compile-time offsets and
// the boundary rule applied to every term.
template <int DIM, int SHAPE, int R, int ARITH, class WS>
__device__ __forceinline__ double update_bc(const double* u, int64_t i, int64_t j, int64_t k, const Geo& g,
                                            int bc, double c, const WS& w)
{
    using S = Stn<DIM, SHAPE, R>;
    const int64_t p = (i * g.n1 + j) * g.n2 + k;
    double v[S::K];
#pragma unroll
    for (int q = 0; q < S::K; ++q) v[q] = fetch_bc(u, i + S::o(q, 0), j + S::o(q, 1), k + S::o(q, 2), g, bc, c);
    double acc = __dmul_rn(w.at(0, p), v[0]);
#pragma unroll
    for (int q = 1; q < S::K; ++q) acc = acc_step<ARITH>(acc, w.at(q, p), v[q]);
    return acc;
}

// Full update at linear index p whose every neighbour is inside the grid (or
// the staged tile) u of n elements.
template <int DIM, int SHAPE, int R, int ARITH, bool RO, class WS>
__device__ __forceinline__ double update_interior(const double* u, int64_t p, int64_t s0, int64_t s1, const WS& w,
                                                  int64_t n)
{
    using S = Stn<DIM, SHAPE, R>;
    double v[S::K];
#pragma unroll
    for (int q = 0; q < S::K; ++q) {
        const int64_t a = p + S::o(q, 0) * s0 + S::o(q, 1) * s1 + S::o(q, 2);
        v[q] = GBST_IN(a, n) ? (RO ? __ldg(u + a) : u[a]) : 0.0;
    }
    double acc = __dmul_rn(w.at(0, p), v[0]);
#pragma unroll
    for (int q = 1; q < S::K; ++q) acc = acc_step<ARITH>(acc, w.at(q, p), v[q]);
    return acc;
}

// Run-time-offset update (any K), the boundary rule applied to every term.
template <int ARITH>
__device__ __forceinline__ double update_rt(const double* u, int64_t i, int64_t j, int64_t k, const Geo& g,
                                            const StencilDev& s)
{
    double acc = 0.0;
    for (int q0 = 0; q0 < s.K; q0 += 8) {
        double v[8];
        double w[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int q = q0 + t;
            if (q < s.K) {
                v[t] = fetch_bc(u, i + s.off[3 * q], j + s.off[3 * q + 1], k + s.off[3 * q + 2], g, s.bc, s.c);
                const int64_t p = (i * g.n1 + j) * g.n2 + k;
                w[t] = s.field ? (GBST_IN(p, s.npts) ? __ldg(s.field + (int64_t)(s.K - 1 - q) * s.npts + p) : 0.0)
                               : s.w[q];
            }
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int q = q0 + t;
            if (q < s.K) acc = (q == 0) ? __dmul_rn(w[t], v[t]) : acc_step<ARITH>(acc, w[t], v[t]);
        }
    }
    return acc;
}

}  // namespace gbst
