/* Variable-size BSMC: a reduced camera system whose cameras carry different
 * numbers of unknowns, its product and its block-Jacobi PCG.
 *
 * Sec. 4 (Fig. 4): the RCS block (i, j) has c_i x c_j entries, c_i being the
 * number of unknowns of camera i, and BSMC stores the non-zero upper blocks
 * with their position and size; Sec. 4.1 takes c = 11 (six exterior and five
 * interior unknowns per camera) for its memory model (Eqs. 8-10).  Cameras
 * that hold their interiors fixed have c_i = 6, self-calibrating ones 11; the
 * format accepts any 1 <= c_i <= BA_VB_CMAX.  The product is the two-sided
 * upper-triangle product of Sec. 6.2 (Fig. 13); the solver is the PCG of
 * Sec. 3.2 (Eqs. 6-7) with M = the diagonal blocks of S.
 *
 * Conventions as in ba.h: every call returns a ba_status, with the reason in
 * ba_last_error(); input arrays are host arrays owned by the caller and
 * copied by ba_vbsmc_create.  After BA_ERR_CUDA or BA_ERR_TIMEOUT the object
 * only accepts ba_vbsmc_destroy (BA_ERR_STATE otherwise).  Calls on one object
 * are not thread-safe.
 */
#ifndef BA_VBSMC_H
#define BA_VBSMC_H

#include "ba.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ba_vbsmc ba_vbsmc; /* opaque; owns its device memory */

#define BA_VB_CMAX 16 /* largest number of unknowns per camera */

/* A variable-size BSMC system S x = b.
 *   opt       precision (BA_FP64, or BA_FP32: values, vectors and PCG in
 *             FP32, reductions in FP64), cuda_stream, device_mem_cap; NULL =
 *             defaults.  Other fields are ignored.
 *   n         cameras (block rows), n >= 1;
 *   cdim[n]   unknowns per camera, 1..BA_VB_CMAX; camera i's entries of x and
 *             b are the c_i consecutive entries after those of cameras < i;
 *   nnzb      stored (upper-triangle) blocks, n <= nnzb < 2^31;
 *   row_ptr[n+1], col[nnzb]: block row i holds blocks row_ptr[i] ..
 *             row_ptr[i+1]-1, the first being the diagonal (col = i), the
 *             others with strictly increasing columns i < col < n;
 *   val       the blocks in that order, block (i, j) as c_i x c_j row-major
 *             doubles, packed without gaps (sum over blocks of c_i c_j);
 *   b         sum c_i doubles.
 * The block-Jacobi preconditioner (the inverse of every diagonal block, by an
 * FP64 Cholesky factorisation on the device) is built here.
 * Errors: BA_ERR_INVALID_ARG (sizes, pattern, options), BA_ERR_NONFINITE (a
 * value or b), BA_ERR_NOT_SPD (a diagonal block), BA_ERR_OOM, BA_ERR_CUDA. */
ba_status ba_vbsmc_create(const ba_options *opt, int32_t n, const int32_t *cdim, int64_t nnzb,
                          const int32_t *row_ptr, const int32_t *col, const double *val,
                          const double *b, ba_vbsmc **out);

/* The reduced camera system of a scene whose cameras carry interior
 * parameters, formed on the device into a variable-size BSMC system.
 *   cams[n_cams x 6]  exterior [omega, t] (X_cam = R(omega) X + t);
 *   intr[n_cams x 5]  interiors [f, cx, cy, k1, k2]: with xh = x/z, yh = y/z,
 *                     r2 = xh^2 + yh^2, d = 1 + k1 r2 + k2 r2^2, the projection
 *                     is u = f d xh + cx, v = f d yh + cy;
 *   cdim[n_cams]      6 (interiors held fixed) or 11 (the five interior
 *                     unknowns follow the six exterior ones);
 *   pts, obs_*        as for ba_problem_create (every point seen at least
 *                     twice, no duplicate (camera, point) pairs);
 *   lambda >= 0       LM damping: lambda times diag(J^T J) clamped to
 *                     [1e-6, 1e32] on every unknown.
 * Forms Eq. 1's e and J (two rows per observation: 11 camera columns, 3
 * point columns), then Eq. 3-4 with c_i unknowns per camera: V_k, V_k^-1
 * and l_p per point; per stored block (i, j) the sum over the points seen by
 * both cameras of -W_ik V_k^-1 W_jk^T, plus U_i (damped) on the diagonal, and
 * b_i = l_c,i - sum_k W_ik V_k^-1 l_p,k.  Arithmetic in FP64; stored in
 * opt->precision.  No atomics: every block is summed by one warp from its
 * own list of point pairs, in track order.  The pattern is that of
 * ba_symbolic_pattern.  Then as ba_vbsmc_create (M^-1 built).  The
 * formation's temporary device buffers (a 256-byte J row per observation,
 * 96 bytes per point, 8 bytes per point pair) are freed before the call
 * returns and are not counted against device_mem_cap.
 * Errors: BA_ERR_INVALID_ARG (sizes, indices, cdim, lambda), BA_ERR_NONFINITE
 * (an input), BA_ERR_NOT_SPD (a V_k or a diagonal block), BA_ERR_OOM,
 * BA_ERR_CUDA. */
ba_status ba_vbsmc_create_interiors(const ba_options *opt, int32_t n_cams, const double *cams, const double *intr,
                                    const int32_t *cdim, int64_t n_pts, const double *pts, int64_t n_obs,
                                    const int32_t *obs_cam, const int64_t *obs_pt, const double *obs_uv,
                                    double lambda, ba_vbsmc **out);

/* The reduced camera system when the images of one physical camera share
 * its interiors: images 0 .. n_images-1 keep their six exterior unknowns
 * (blocks of size 6), and physical camera q becomes block n_images + q with
 * its five interior unknowns [f, cx, cy, k1, k2] (block size 5).  phys[i]
 * (0 .. n_phys-1) names image i's physical camera, intr_phys[n_phys x 5] the
 * physical cameras' interiors (camera model as for
 * ba_vbsmc_create_interiors); cams, pts and the observations as there.
 * Per observation of image i, the exterior columns of J_c belong to block i
 * and the interior columns to block n_images + phys[i].  Eq. 3 per block:
 * U = sum J_s^T J_t over the two column groups s, t of each observation
 * (which couples image i to its physical camera), damped with lambda times
 * its clamped diagonal on the diagonal blocks; l = -sum J_s^T e.  Eq. 4 per
 * point k: W_beta = sum of J_s^T J_p over the point's observations with
 * columns in block beta, S(beta, gamma) -= W_beta V_k^-1 W_gamma^T and
 * b_beta -= W_beta V_k^-1 l_p,k.  The pattern is every diagonal block plus
 * each (beta < gamma) that one point's observations reach.  Formed on the
 * device in FP64 (one warp per block over its list of column-group pairs; no
 * atomics), stored in opt->precision, M^-1 built as by ba_vbsmc_create.
 * Temporary device buffers as for ba_vbsmc_create_interiors.  Errors:
 * BA_ERR_INVALID_ARG (sizes, indices, phys, lambda), BA_ERR_NONFINITE,
 * BA_ERR_NOT_SPD, BA_ERR_OOM, BA_ERR_CUDA. */
ba_status ba_vbsmc_create_shared(const ba_options *opt, int32_t n_images, const double *cams, int32_t n_phys,
                                 const double *intr_phys, const int32_t *phys, int64_t n_pts, const double *pts,
                                 int64_t n_obs, const int32_t *obs_cam, const int64_t *obs_pt, const double *obs_uv,
                                 double lambda, ba_vbsmc **out);

/* ---- The LM iteration with interior parameters --------------------------
 * An LM problem whose cameras carry interiors (camera model, cdim and
 * observation rules as for ba_vbsmc_create_interiors): cameras with cdim 11
 * estimate their five interiors, those with cdim 6 hold them fixed.  One
 * ba_vbi_lm_step is the iteration of ba_lm_step with c_i unknowns per
 * camera (Fig. 2; Eq. 1 by Eqs. 3-5): linearize (FP64 rows of e and J with
 * 11 camera columns) if the state changed, form the variable-size RCS with
 * lambda (Eq. 3-4, as ba_vbsmc_create_interiors), solve it by block-Jacobi
 * PCG (Sec. 3.2; stop at pcg_rel_tol, cap pcg_max_iters or max(1000, 6n)),
 * back-substitute the points (Eq. 5: dx_p = V^-1 (l_p - sum W^T dx_c)), move
 * to the trial state (pose X_cam <- Exp(d_omega) X_cam + dt, interiors and
 * points additively), evaluate its cost and the model decrease
 * 1/2 (||e||^2 - ||e + J dx||^2) in FP64, and accept if the gain ratio
 * exceeds 1e-3 (Nielsen's damping rule, lambda starting at opt->lambda0).
 * On a rejection only lambda changes: the next step re-forms the RCS from
 * the stored linearization.  opt->precision BA_FP32 stores the RCS and runs
 * the PCG in FP32 (formation, Eq. 5 and the trial evaluation stay FP64);
 * BA_FP64 runs everything in FP64.  Other options: lambda0, pcg_rel_tol,
 * pcg_max_iters, cuda_stream, device_mem_cap.  ba_step_info: cost_before,
 * cost_after, cost_trial, predicted, rho, lambda, accepted, pcg_iters,
 * rcs_rel_resid (the PCG recurrence's ||r|| / ||r_0||), n_cheirality and
 * ms[0..5] = linearize, RCS formation with M^-1, PCG, Eq. 5 and the trial
 * cameras, trial evaluation, total.  States are in the caller's order
 * (cams n x 6, intr n x 5, pts n_pts x 3).  After BA_ERR_CUDA or
 * BA_ERR_TIMEOUT the problem only accepts ba_vbi_problem_destroy. */
typedef struct ba_vbi_problem ba_vbi_problem;

ba_status ba_vbi_problem_create(const ba_options *opt, int32_t n_cams, const double *cams, const double *intr,
                                const int32_t *cdim, int64_t n_pts, const double *pts, int64_t n_obs,
                                const int32_t *obs_cam, const int64_t *obs_pt, const double *obs_uv,
                                ba_vbi_problem **out);
ba_status ba_vbi_lm_step(ba_vbi_problem *p, ba_step_info *info);
ba_status ba_vbi_get_state(const ba_vbi_problem *p, double *cams, double *intr, double *pts);
ba_status ba_vbi_set_state(ba_vbi_problem *p, const double *cams, const double *intr, const double *pts,
                           double lambda, double nu);
/* lambda, nu and the cost F of the current state (computed if needed). */
ba_status ba_vbi_get_lm_state(const ba_vbi_problem *p, double *lambda, double *nu, double *cost);
/* The last step: dxc (sum c_i values, camera order, c_i per camera), dxp
 * (n_pts x 3); BA_ERR_STATE before the first step. */
ba_status ba_vbi_get_step(const ba_vbi_problem *p, double *dxc, double *dxp);
/* The variable-size system of the last formation (owned by the problem; for
 * ba_vbsmc_get_system / ba_vbsmc_spmv / ba_vbsmc_info). */
const ba_vbsmc *ba_vbi_system(const ba_vbi_problem *p);
ba_status ba_vbi_info(const ba_vbi_problem *p, int64_t *n_unknowns, int64_t *n_blocks, int64_t *device_bytes);
void ba_vbi_problem_destroy(ba_vbi_problem *p);

/* Copies the system to host arrays (each may be NULL): row_ptr[n+1],
 * col[nnzb], the packed block values (as ba_vbsmc_create takes them,
 * upcast to double) and b.  Synchronous.  Errors: BA_ERR_INVALID_ARG,
 * BA_ERR_STATE, BA_ERR_CUDA. */
ba_status ba_vbsmc_get_system(const ba_vbsmc *h, int32_t *row_ptr, int32_t *col, double *val, double *b);

/* y = S x on the object's stream (asynchronous): x and y are device arrays of
 * sum c_i values in the object's precision (double or float), not
 * overlapping.  Errors: BA_ERR_INVALID_ARG (null), BA_ERR_STATE, BA_ERR_CUDA. */
ba_status ba_vbsmc_spmv(ba_vbsmc *h, const void *x, void *y);

/* Block-Jacobi PCG on S y = b from y = 0 until ||r_k|| / ||r_0|| <= tol or
 * max_iters iterations (0: max(1000, 6 n)); one cooperative kernel.
 * Synchronous.  x_out (host, sum c_i doubles) receives y, and may be NULL;
 * iters, rel_resid (the recurrence's ||r_k|| / ||r_0||) and kernel_ms (the
 * device time of the solve) may be NULL.  Errors: BA_ERR_INVALID_ARG (tol <=
 * 0, max_iters < 0), BA_ERR_NOT_SPD (d^T S d <= 0), BA_ERR_NO_CONVERGENCE
 * (max_iters reached; the outputs are still written), BA_ERR_TIMEOUT (a grid
 * wait gave up), BA_ERR_STATE, BA_ERR_CUDA. */
ba_status ba_vbsmc_solve(ba_vbsmc *h, double tol, int32_t max_iters, double *x_out, int32_t *iters,
                         double *rel_resid, double *kernel_ms);

/* Sizes (each output may be NULL): unknowns (sum c_i), the bytes of the
 * stored format - the block values, a column and a value offset per block
 * (4 + 8 bytes: the three 4-byte ids per block of Eq. 9), n + 1 row starts
 * and n block sizes - and the number of stored blocks. */
ba_status ba_vbsmc_info(const ba_vbsmc *h, int64_t *n_unknowns, int64_t *storage_bytes, int64_t *n_blocks);

void ba_vbsmc_destroy(ba_vbsmc *h);

#ifdef __cplusplus
}
#endif

#endif /* BA_VBSMC_H */
