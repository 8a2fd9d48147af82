/*
 * lcs.h - C ABI of the longest-common-subsequence kernels of the GB300-native
 * stencil library.
 *
 * Longest common subsequence (Section 3.4 of "Temporal Vectorization for
 * Stencils", "Longest common subsequence"): lcs[x][y] is the length of the
 * longest common subsequence of A[1..x] and B[1..y]; lcs[0][y] = lcs[x][0] = 0
 * and, for x, y >= 1,
 *     lcs[x][y] = lcs[x-1][y-1] + 1               if A[x] == B[y]
 *               = max(lcs[x-1][y], lcs[x][y-1])   otherwise.
 * The paper treats x (over A) as time and y (over B) as space: a 1D
 * Gauss-Seidel stencil whose coefficient B[y] varies with the point.
 *
 * Sequences are byte strings (any of the 256 values is a symbol) in DEVICE
 * memory. The result is the last row, row[y] = lcs[na][y] for y = 0..nb
 * (nb + 1 int32 values in DEVICE memory); row[nb] is the LCS length.
 *
 * Kernel families (both give the same row, exactly):
 *   LCS_KERNEL_DP    one cell per warp lane and step: lanes hold consecutive
 *                    rows of A (times), lane k one column behind lane k - 1,
 *                    values passed lane to lane by warp shuffle, the update
 *                    a blend of the equality mask (the paper's formulation).
 *   LCS_KERNEL_BITS  64 cells per lane and step: each row is held as the
 *                    bit vector of its differences lcs[x][y] - lcs[x][y-1]
 *                    and advanced by one 64-bit add with carry per word
 *                    (Allison and Dix 1986; Hyyro 2004); the same lane and
 *                    skew layout, several rows of A per lane.
 *   LCS_KERNEL_AUTO  the library's choice (BITS).
 * Return codes and streams as in stencil.h.
 */
#ifndef GB300_LCS_H
#define GB300_LCS_H

#include <stddef.h>
#include <stdint.h>

#include "stencil.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LCS_KERNEL_AUTO 0
#define LCS_KERNEL_DP 1
#define LCS_KERNEL_BITS 2

/* Bytes of workspace lcs_run needs for (na, nb, kernel) on the current device. */
int lcs_workspace_bytes(int64_t na, int64_t nb, int kernel, size_t* bytes);

/*
 * Compute row[y] = lcs[na][y], y = 0..nb, on stream (a cudaStream_t; NULL =
 * legacy default stream).
 *   A, na      device pointer to the na >= 0 symbols of A (may be NULL if na == 0).
 *   B, nb      device pointer to the nb >= 0 symbols of B (may be NULL if nb == 0).
 *   row        device pointer to nb + 1 int32 values (written).
 *   kernel     LCS_KERNEL_AUTO, LCS_KERNEL_DP or LCS_KERNEL_BITS.
 *   workspace  device pointer to lcs_workspace_bytes() bytes, 16-byte aligned,
 *              or NULL. With a workspace the call is asynchronous and a
 *              device-side failure (a bounded wait between the kernel's
 *              warps that gave up) is read later by lcs_status(workspace).
 *              With NULL the library allocates the workspace stream-ordered,
 *              synchronises the stream at the end, frees it and returns the
 *              device status itself.
 * Returns STENCIL_OK, STENCIL_EINVAL (a negative length, a null pointer, an
 * unknown kernel, na or nb above 2^30, misaligned workspace),
 * STENCIL_ENOMEM, STENCIL_ECUDA or (NULL workspace) STENCIL_ETIMEOUT.
 */
int lcs_run(const uint8_t* A, int64_t na, const uint8_t* B, int64_t nb, int32_t* row, int kernel, void* workspace,
            void* cuda_stream);

/*
 * Synchronise stream, then return and clear the device status kept in a
 * workspace used by lcs_run: STENCIL_OK or STENCIL_ETIMEOUT (or STENCIL_ECUDA
 * if the synchronisation failed).
 */
int lcs_status(void* workspace, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_LCS_H */
