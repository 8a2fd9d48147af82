/*
 * CPU oracle for time-iterated Jacobi and Gauss-Seidel stencils.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path links,
 * loads or calls this file; only the tests, the smoke check and the
 * benchmark's CPU-baseline leg do. It shares no code, header or table with
 * the CUDA path.
 *
 * It is the literal definition, written out with no blocking, skewing,
 * vectorisation or reordering:
 *
 *  - The naive (d+1)-loop stencil of Section 1 and Algorithm 1: the outer
 *    loop runs over time, the inner loops update every grid point from the
 *    values of its neighbours.
 *  - Jacobi (Section 1 taxonomy; Algorithm 1): every point of step t+1 is
 *    computed from step-t values only, so two arrays are used.
 *  - Gauss-Seidel (Section 3.4, "Gauss-Seidel stencils"): one array, updated
 *    in place, points visited in increasing lexicographic order with the
 *    slowest dimension outermost (Section 3.2: the innermost loop runs over
 *    space in increasing order), so neighbours that were already visited in
 *    this sweep contribute their newest value.
 *  - Boundary conditions (Section 1 taxonomy, "constant, periodic"): a
 *    constant boundary reads the value c at every index outside the grid
 *    (the fixed a_0 and a_{NX+1} of Algorithm 1, generalised to width r and
 *    to corners); a periodic boundary wraps each index modulo the extent.
 *
 * Readings where the paper is silent (the library follows the same ones):
 *  - Offsets are ordered lexicographically, slowest dimension first, each
 *    component running from -r to +r ("canonical order"). A star keeps the
 *    offsets with at most one non-zero component; a box keeps all of them.
 *    Coefficients are given in that order.
 *  - Terms are summed in DESCENDING canonical order (the offset with the
 *    largest lexicographic value first), so that in Gauss-Seidel the
 *    newest-value terms (negative offsets) enter last.
 *  - ARITH_FMA:      acc = w*u for the first term (one rounding), then
 *                    acc = fma(w, u, acc) for every later term.
 *    ARITH_UNFUSED:  acc = w*u for the first term, then acc = acc + (w*u),
 *                    the product and the sum each rounded.
 *    Built with -ffp-contract=off so that the compiler fuses nothing;
 *    fma() is the C99 correctly rounded fused multiply-add.
 *  - Variable coefficients (Section 3.4 treats LCS's second sequence B as a
 *    variable coefficient): when a coefficient field is given, the weight of
 *    canonical term q at point p is field[q * N + p] (N = grid points)
 *    instead of w[q]; everything else is unchanged.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_STAR 0
#define OR_BOX 1
#define OR_JACOBI 0
#define OR_GAUSS_SEIDEL 1
#define OR_BC_CONSTANT 0
#define OR_BC_PERIODIC 1
#define OR_ARITH_FMA 0
#define OR_ARITH_UNFUSED 1

/* Canonical offsets of a (dim, shape, r) stencil, each stored as three
 * components (slowest first; the unused leading components of a 1D or 2D
 * stencil are 0). Returns K, the number of points, or -1 on bad input. */
int oracle_offsets(int dim, int shape, int r, int* off)
{
    if (dim < 1 || dim > 3 || r < 0 || (shape != OR_STAR && shape != OR_BOX)) return -1;
    int lo0 = (dim >= 3) ? -r : 0, hi0 = (dim >= 3) ? r : 0;
    int lo1 = (dim >= 2) ? -r : 0, hi1 = (dim >= 2) ? r : 0;
    int K = 0;
    for (int a = lo0; a <= hi0; ++a)
        for (int b = lo1; b <= hi1; ++b)
            for (int c = -r; c <= r; ++c) {
                int nz = (a != 0) + (b != 0) + (c != 0);
                if (shape == OR_STAR && nz > 1) continue;
                if (off) { off[3 * K] = a; off[3 * K + 1] = b; off[3 * K + 2] = c; }
                ++K;
            }
    return K;
}

typedef struct {
    int64_t n[3];       /* extents, slowest first, padded with 1 */
    int bc;
    double c;
} grid_t;

/* Value of the array at (i, j, k) after applying the boundary rule. */
static double fetch(const double* u, const grid_t* g, int64_t i, int64_t j, int64_t k)
{
    if (g->bc == OR_BC_PERIODIC) {
        i = ((i % g->n[0]) + g->n[0]) % g->n[0];
        j = ((j % g->n[1]) + g->n[1]) % g->n[1];
        k = ((k % g->n[2]) + g->n[2]) % g->n[2];
    } else if (i < 0 || i >= g->n[0] || j < 0 || j >= g->n[1] || k < 0 || k >= g->n[2]) {
        return g->c;
    }
    return u[(i * g->n[1] + j) * g->n[2] + k];
}

/* Weight of canonical term q at point (i, j, k): w[q], or the field's value. */
static double weight(const double* w, const double* field, const grid_t* g, int q, int64_t i, int64_t j, int64_t k)
{
    if (!field) return w[q];
    int64_t n = g->n[0] * g->n[1] * g->n[2];
    return field[q * n + (i * g->n[1] + j) * g->n[2] + k];
}

/* One point update: the weighted sum over the stencil in descending
 * canonical order, with the rounding of the chosen arithmetic mode. */
static double update(const double* src, const grid_t* g, int64_t i, int64_t j, int64_t k,
                     const int* off, const double* w, const double* field, int K, int arith)
{
    int q = K - 1;
    double acc = weight(w, field, g, q, i, j, k) * fetch(src, g, i + off[3 * q], j + off[3 * q + 1], k + off[3 * q + 2]);
    for (q = K - 2; q >= 0; --q) {
        double v = fetch(src, g, i + off[3 * q], j + off[3 * q + 1], k + off[3 * q + 2]);
        double wq = weight(w, field, g, q, i, j, k);
        if (arith == OR_ARITH_FMA) {
            acc = fma(wq, v, acc);
        } else {
            double prod = wq * v;
            acc = acc + prod;
        }
    }
    return acc;
}

/* Advance u (C order, ext[0] slowest, interior points only) by T steps.
 * field: NULL for the constant weights w, else K * N per-point weights
 * (term-major, canonical order). Returns 0, or -1 on invalid arguments.
 * nthreads <= 0 uses the OpenMP default; the result does not depend on the
 * thread count. */
int oracle_run_field(int dim, int shape, int r, const double* w, const double* field, int K, int method, int bc,
                     double c, int arith, const int64_t* ext, int64_t T, double* u, int nthreads)
{
    int off[3 * 729];
    if (r > 4) return -1;
    int Kc = oracle_offsets(dim, shape, r, off);
    if (Kc < 0 || Kc != K || T < 0) return -1;
    grid_t g;
    g.n[0] = g.n[1] = g.n[2] = 1;
    for (int d = 0; d < dim; ++d) {
        if (ext[d] < 1) return -1;
        g.n[3 - dim + d] = ext[d];
    }
    g.bc = bc;
    g.c = c;
    if (bc == OR_BC_PERIODIC)
        for (int d = 0; d < dim; ++d)
            if (ext[d] < 2 * r + 1) return -1;
    int64_t total = g.n[0] * g.n[1] * g.n[2];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    if (method == OR_JACOBI) {
        double* v = (double*)malloc((size_t)total * sizeof(double));
        if (!v) return -1;
        double* a = u;
        double* b = v;
        for (int64_t t = 0; t < T; ++t) {
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < g.n[0]; ++i)
                for (int64_t j = 0; j < g.n[1]; ++j)
                    for (int64_t k = 0; k < g.n[2]; ++k)
                        b[(i * g.n[1] + j) * g.n[2] + k] = update(a, &g, i, j, k, off, w, field, K, arith);
            double* s = a; a = b; b = s;
        }
        if (a != u) memcpy(u, a, (size_t)total * sizeof(double));
        free(v);
    } else if (method == OR_GAUSS_SEIDEL) {
        for (int64_t t = 0; t < T; ++t)
            for (int64_t i = 0; i < g.n[0]; ++i)
                for (int64_t j = 0; j < g.n[1]; ++j)
                    for (int64_t k = 0; k < g.n[2]; ++k)
                        u[(i * g.n[1] + j) * g.n[2] + k] = update(u, &g, i, j, k, off, w, field, K, arith);
    } else {
        return -1;
    }
    return 0;
}

int oracle_run(int dim, int shape, int r, const double* w, int K, int method, int bc, double c,
               int arith, const int64_t* ext, int64_t T, double* u, int nthreads)
{
    return oracle_run_field(dim, shape, r, w, NULL, K, method, bc, c, arith, ext, T, u, nthreads);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
