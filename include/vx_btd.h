/*
 * vx_btd.h -- C ABI of the batched block-tridiagonal solve of the per-ray Newton systems.
 *
 * Where it sits in the method. The radial transport sweeps of Marek et al. (arXiv:1404.1719) are
 * implicit in time and run ray by ray; each ray's step is a non-linear system in the zone unknowns,
 * solved by Newton-Raphson iterations with an explicitly built Jacobian and a direct solve of the
 * linearised system (sec. 2.1). A radial difference scheme couples a zone only to its neighbours,
 * so for the zones k = 0 .. n-1 of one ray, with m unknowns per zone, that linear system reads
 *
 *     A_k x_{k-1} + B_k x_k + C_k x_{k+1} = d_k        (A_0 and C_{n-1} are not read).
 *
 * The pair-process source derivatives of vx_rates_spectral (blocks d(j0, chi0)/dJ and
 * d(j1, chi1)/dH of the partner spectrum) are part of B_k in such a system; the radial flux terms
 * make A_k and C_k. Rays are independent (sec. 2.2) and are solved in one call.
 *
 * Method (GB300: FP32 arithmetic, FP64 only where accuracy needs it). Block LU along the ray
 * without pivoting across zones: D_0 = B_0, D_k = B_k - A_k G_{k-1} with G_k = D_k^{-1} C_k,
 * each D_k factored with partial pivoting inside the block. The factorisation is done in FP32 from
 * FP32 copies of the blocks, one CTA per ray: the product A_k G_{k-1} on the tensor cores (TF32
 * with each operand split into two parts, three products: about FP32 accuracy), then Gauss-Jordan
 * elimination of [D_k | C_k] with partial pivoting, whose right-hand block ends as G_k and whose
 * multipliers are kept. Then the ray is solved by replaying those eliminations on the right-hand
 * side, and
 * n_refine sweeps of iterative refinement follow, each from the FP64 residual d - M x of the
 * caller's FP64 blocks. For a ray whose Schur complements are well conditioned (e.g. block rows
 * diagonally dominant) every sweep gains a factor of about cond x 1e-7, so two sweeps reach FP64
 * accuracy at moderate condition numbers. The reduction order is fixed: results are reproducible
 * run to run.
 *
 * Conventions (as in vx_rates.h): arrays are dense, row-major FP64 unless stated; device pointers
 * are CUDA global memory of the current device, owned by the caller; the library never retains a
 * caller pointer after a call returns. Calls are asynchronous on `stream`; argument checks happen
 * on the host before anything is launched, and a rejected call returns VX_ERR_INVALID_ARG and
 * writes nothing. A handle is not thread-safe.
 */
#ifndef VX_BTD_H
#define VX_BTD_H

#include "vx_rates.h" /* vx_status, vx_stream, vx_status_string, vx_last_error */

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vx_btd vx_btd;

#define VX_BTD_MAX_M 128      /* unknowns per zone */
#define VX_BTD_MAX_REFINE 8

/* Creates a solver for m unknowns per zone (1 .. VX_BTD_MAX_M) and batches of at most max_zones
 * zones (>= 0), with n_refine FP64 refinement sweeps (0 .. VX_BTD_MAX_REFINE; 0 leaves the FP32
 * solution). Allocates the device workspace: (12 m^2 + 16 m + 4) bytes per zone. *out is set to
 * NULL on failure. Errors: VX_ERR_INVALID_ARG, VX_ERR_OOM, VX_ERR_CUDA. */
vx_status vx_btd_create(int m, long long max_zones, int n_refine, vx_btd **out);

/* Solves every ray. n_rays >= 0; n_zones = the total zone count, 0 .. max_zones.
 *   ray_offsets: device int32 [n_rays + 1]; ray r owns zones ray_offsets[r] .. ray_offsets[r+1]-1.
 *                Must start at 0, not decrease and end at n_zones (checked on the device: if not,
 *                nothing is solved, x is left unwritten and the numeric flag is raised).
 *   A, B, C:     device FP64 [n_zones][m][m], the sub-diagonal, diagonal and super-diagonal blocks
 *                of each zone's block row (A of a ray's first zone and C of its last are not read).
 *   d:           device FP64 [n_zones][m], right-hand sides.
 *   x:           device FP64 [n_zones][m], the solution (written; must not overlap d or the blocks).
 * A ray with a zero or non-finite pivot gets NaN in x and raises the numeric flag (vx_btd_check).
 * Errors: VX_ERR_INVALID_ARG (NULL handle or pointers with n_zones > 0, a pointer that is not device
 * (or managed) memory, offsets not 4-byte or FP64 arrays not 8-byte aligned, n_rays < 0, n_zones
 * out of range, x overlapping an input), VX_ERR_CUDA. Nothing is launched then. */
vx_status vx_btd_solve(vx_btd *h, int n_rays, long long n_zones, const int *ray_offsets, const double *A,
                       const double *B, const double *C, const double *d, double *x, vx_stream stream);

/* Synchronises `stream` and returns VX_ERR_NUMERIC if a solve since the last check met a zero or
 * non-finite pivot or invalid ray offsets (then clears the flag), else VX_OK. */
vx_status vx_btd_check(vx_btd *h, vx_stream stream);

/* Frees the handle and its workspace (NULL is a no-op). */
void vx_btd_destroy(vx_btd *h);

#ifdef __cplusplus
}
#endif

#endif /* VX_BTD_H */
