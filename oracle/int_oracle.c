/*
 * CPU oracle for the integer stencils: Game of Life (Section 3.4, "Game of
 * life") and the longest common subsequence (Section 3.4, "Longest common
 * subsequence").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path links,
 * loads or calls this file; only the tests, the smoke check and the
 * benchmark's CPU-baseline leg do. It shares no code, header or table with
 * the CUDA path.
 *
 * Game of Life, the literal definition: a 2D Jacobi stencil over the 3 x 3
 * box (Section 3.4 calls it a 2D9P Jacobi stencil whose update depends on
 * the 8 neighbours). Each cell holds 0 (dead) or 1 (live). At every step,
 * for every cell, n = the number of live cells among its 8 neighbours
 * (the cell itself excluded), read from the previous step's grid (two
 * arrays); the new cell is live iff bit n of `survive` is set (live cell)
 * or bit n of `birth` is set (dead cell). The paper's variant B2S23 is
 * birth = 1 << 2, survive = (1 << 2) | (1 << 3); Conway's B3S23 is
 * birth = 1 << 3.
 * Boundary: constant = every cell outside the grid is dead; periodic = the
 * grid is a torus (indices wrap modulo the extents).
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OI_BC_CONSTANT 0
#define OI_BC_PERIODIC 1

static int cell_at(const uint8_t* g, int64_t n0, int64_t n1, int bc, int64_t i, int64_t j)
{
    if (bc == OI_BC_PERIODIC) {
        i = ((i % n0) + n0) % n0;
        j = ((j % n1) + n1) % n1;
    } else if (i < 0 || i >= n0 || j < 0 || j >= n1) {
        return 0;
    }
    return g[i * n1 + j] != 0;
}

/* Advance cells (n0 x n1, C order, one byte per cell) by T steps in place.
 * Returns 0, or -1 on invalid arguments. */
int oracle_life(int64_t n0, int64_t n1, int bc, uint32_t birth, uint32_t survive, int64_t T, uint8_t* cells,
                int nthreads)
{
    if (n0 < 1 || n1 < 1 || T < 0 || !cells || (bc != OI_BC_CONSTANT && bc != OI_BC_PERIODIC)) return -1;
    uint8_t* a = cells;
    uint8_t* b = (uint8_t*)malloc((size_t)(n0 * n1));
    if (!b) return -1;
    if (nthreads > 0) omp_set_num_threads(nthreads);
    for (int64_t t = 0; t < T; ++t) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n0; ++i) {
            for (int64_t j = 0; j < n1; ++j) {
                int n = 0;
                for (int di = -1; di <= 1; ++di)
                    for (int dj = -1; dj <= 1; ++dj)
                        if (di != 0 || dj != 0) n += cell_at(a, n0, n1, bc, i + di, j + dj);
                const int alive = a[i * n1 + j] != 0;
                b[i * n1 + j] = (uint8_t)(((alive ? survive : birth) >> n) & 1u);
            }
        }
        uint8_t* tmp = a;
        a = b;
        b = tmp;
    }
    if (a != cells) {
        memcpy(cells, a, (size_t)(n0 * n1));
        free(a);
    } else {
        free(b);
    }
    return 0;
}

/*
 * Longest common subsequence, the dynamic-programming definition of Section
 * 3.4: lcs[x][y] is the length of the longest common subsequence of
 * A[1..x] and B[1..y]; lcs[0][y] = lcs[x][0] = 0 and, for x, y >= 1,
 *     lcs[x][y] = lcs[x-1][y-1] + 1                  if A[x] == B[y]
 *               = max(lcs[x-1][y], lcs[x][y-1])      otherwise.
 * x (over A) is the time dimension and y (over B) the space dimension, so
 * one row of nb + 1 values is kept and updated in place in increasing y,
 * the 1D Gauss-Seidel form the paper gives it. On return
 * row[y] = lcs[na][y] for y = 0..nb (row[nb] is the LCS length).
 * Returns 0, or -1 on invalid arguments.
 */
int oracle_lcs(const uint8_t* A, int64_t na, const uint8_t* B, int64_t nb, int32_t* row)
{
    if (na < 0 || nb < 0 || !row || (na > 0 && !A) || (nb > 0 && !B)) return -1;
    for (int64_t y = 0; y <= nb; ++y) row[y] = 0;
    for (int64_t x = 1; x <= na; ++x) {
        int32_t diag = 0;  /* lcs[x-1][y-1] */
        for (int64_t y = 1; y <= nb; ++y) {
            const int32_t up = row[y];  /* lcs[x-1][y] */
            const int32_t left = row[y - 1];  /* lcs[x][y-1], already updated */
            row[y] = A[x - 1] == B[y - 1] ? diag + 1 : (up > left ? up : left);
            diag = up;
        }
    }
    return 0;
}
