/*
 * life.h - C ABI of the Game of Life kernels of the GB300-native stencil
 * library.
 *
 * Game of Life (Section 3.4 of "Temporal Vectorization for Stencils",
 * "Game of life"): a 2D Jacobi stencil over the 3 x 3 box whose update of a
 * cell depends on its 8 neighbours. Each cell is 0 (dead) or 1 (live). At
 * every step, for every cell, n = the number of live cells among its 8
 * neighbours in the previous step's grid; the new cell is live iff bit n of
 * survive_mask is set (live cell) or bit n of birth_mask is set (dead
 * cell). The paper's variant B2S23 is birth_mask = 1 << 2 and
 * survive_mask = (1 << 2) | (1 << 3); Conway's B3S23 has birth_mask = 1 << 3.
 *
 * Layout: cells are n0 x n1 bytes (ext[0] = n0 rows, the slow dimension;
 * ext[1] = n1 cells per row, contiguous), C order, DEVICE memory; a byte is
 * read as live iff it is non-zero and written as 0 or 1. Internally the
 * library packs 32 cells per 32-bit word (2 bits of workspace per cell for
 * two packed grids), runs the steps on the packed grids and unpacks the
 * result into the same bytes.
 * Boundary: STENCIL_BC_CONSTANT = every cell outside the grid is dead;
 * STENCIL_BC_PERIODIC = the grid is a torus (every extent must be >= 3).
 * Return codes, streams and asynchrony as in stencil.h.
 */
#ifndef GB300_LIFE_H
#define GB300_LIFE_H

#include <stddef.h>
#include <stdint.h>

#include "stencil.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Bytes of workspace life_run needs for ext (two packed grids, 16-byte aligned). */
int life_workspace_bytes(const int64_t ext[2], size_t* bytes);

/*
 * Advance cells (device pointer, ext[0] x ext[1] bytes) by T >= 0 steps on
 * stream (a cudaStream_t; NULL = legacy default stream).
 *   boundary      STENCIL_BC_CONSTANT or STENCIL_BC_PERIODIC.
 *   birth_mask    bit n set: a dead cell with n live neighbours becomes live (n = 0..8).
 *   survive_mask  bit n set: a live cell with n live neighbours stays live.
 *   tb            steps per launch: 0 = the library's choice (16), 1 = one launch
 *                 per step; values above 32 are clamped to 32 (one halo word of 32
 *                 cells per side). Periodic grids whose n1 is not a multiple of 32
 *                 always take one launch per step.
 *   workspace     device pointer of life_workspace_bytes() bytes (16-byte aligned,
 *                 not overlapping cells), or NULL: allocated stream-ordered and
 *                 freed after the run.
 * Returns STENCIL_OK, STENCIL_EINVAL (null pointer, extent < 1, periodic extent
 * < 3, a mask above 0x1FF, T < 0, misaligned workspace), STENCIL_ENOMEM or
 * STENCIL_ECUDA. T = 0 leaves cells untouched.
 */
int life_run(uint8_t* cells, const int64_t ext[2], int boundary, uint32_t birth_mask, uint32_t survive_mask,
             int64_t T, int tb, void* workspace, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_LIFE_H */
