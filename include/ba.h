/*
 * ba.h - C ABI of libba, exact Levenberg-Marquardt bundle adjustment on one
 * GB300 GPU (sm_103a), after arXiv 2307.08383 ("Distributed bundle adjustment
 * with block-based sparse matrix compression for super large scale datasets").
 *
 * The library owns every device buffer of a problem.  Inputs are host arrays
 * owned by the caller and copied at creation; getters write into caller
 * buffers.  No exception crosses this boundary: every call returns a
 * ba_status, and ba_last_error() gives a message for the calling thread.
 * After BA_ERR_CUDA or BA_ERR_INTERNAL a problem is unusable and every later
 * call on it returns BA_ERR_STATE.  Calls on one problem are not thread-safe;
 * separate problems may run concurrently on different streams.
 *
 * Problem statement (Sec. 3.1): cameras c = [omega(3), t(3)] with
 * X_cam = R(omega) X + t, a pinhole u = fx x/z + cx, v = fy y/z + cy, and the
 * reprojection errors e = pi(X_cam) - u_obs.  One LM iteration solves Eq. 1,
 * (J^T J + lambda D^T D) dx = -J^T e, by the Schur complement: the reduced
 * camera system (RCS) of Eq. 4 is formed point by point (Sec. 5), stored as
 * BSMC (Sec. 4), solved by block-Jacobi PCG (Sec. 3.2, Eqs. 6-7), and the
 * points are back-substituted by Eq. 5.  Beside that path: the points can be
 * re-triangulated from the poses instead (ba_triangulate), the RCS product can
 * be run in other storage formats, or without a stored RCS, for the paper's
 * storage comparison (ba_rcs_spmv), a given BSMC system can be solved alone
 * (ba_problem_create_rcs, ba_pcg_solve_static), and a learned correction of
 * the block-Jacobi preconditioner can be attached (ba_precond_net_*).
 * Cameras that also carry interior parameters give RCS blocks of mixed sizes
 * (Sec. 4): those systems are declared in ba_vbsmc.h.
 */
#ifndef BA_H
#define BA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ba_problem ba_problem; /* opaque; owns all device memory */

typedef enum {
    BA_OK = 0,
    BA_ERR_INVALID_ARG = 1,   /* bad pointer, size, index, duplicate or option */
    BA_ERR_OOM = 2,           /* device allocation failed or device_mem_cap hit */
    BA_ERR_CUDA = 3,          /* a CUDA runtime call failed; problem unusable */
    BA_ERR_NONFINITE = 4,     /* NaN/Inf in an input or in a computed cost */
    BA_ERR_NOT_SPD = 5,       /* a V_k or an RCS diagonal block is not positive definite */
    BA_ERR_NO_CONVERGENCE = 6,/* PCG hit its iteration cap; the partial solution is kept */
    BA_ERR_TIMEOUT = 7,       /* a bounded device wait gave up; the problem is unusable after it */
    BA_ERR_STATE = 8,         /* call out of order, or problem unusable */
    BA_ERR_INTERNAL = 9       /* a device-side consistency check failed */
} ba_status;

enum { BA_FP64 = 0, BA_FP32 = 1 };            /* ba_options.precision */
enum { BA_LOSS_PLAIN = 0, BA_LOSS_HUBER = 1 }; /* ba_options.robust */
enum { BA_PC_BLOCK_JACOBI = 0, BA_PC_LEARNED = 1 };
enum { BA_PCG_AUTO = 0, BA_PCG_STANDARD = 1, BA_PCG_SPLIT = 2, BA_PCG_IMPLICIT = 3 }; /* ba_options.pcg_variant */

typedef struct {
    int32_t precision;       /* BA_FP64: everything in FP64.  BA_FP32: Jacobians,
                                RCS assembly, SpMV and PCG in FP32; cost and
                                gain-ratio sums and the outer refinement
                                residual r = b - S x in FP64. */
    double fx, fy, cx, cy;   /* pinhole intrinsics in px (1000, 1000, 500, 500) */
    int32_t robust;          /* BA_LOSS_PLAIN or BA_LOSS_HUBER */
    double huber_delta;      /* Huber threshold in px (2.0) */
    double lambda0;          /* initial LM damping (1e-4) */
    double pcg_rel_tol;      /* stop when ||b - S x|| / ||b|| <= tol (1e-10) */
    int32_t pcg_max_iters;   /* 0: max(1000, 6n) */
    double inner_rel_tol;    /* FP32 mode: tolerance of each inner FP32 PCG (1e-4); a sweep that
                                needs less (pcg_rel_tol / current rel. residual,
                                at most 0.9) asks for that instead */
    int32_t refine_max;      /* FP32 mode: outer refinement steps (20) */
    int32_t preconditioner;  /* BA_PC_BLOCK_JACOBI (only this value is accepted) */
    void *cuda_stream;       /* cudaStream_t to run on; NULL = legacy default stream */
    size_t device_mem_cap;   /* 0 = none; creation fails with BA_ERR_OOM above it */
    int32_t group_max_obs;   /* observations per point group (0 = default) */
    int32_t profile;         /* nonzero: time every kernel launch with CUDA events */
    int32_t solve_precision; /* FP64 problems only: BA_FP32 solves S x = b with FP32 inner
                                PCG on a demoted copy of S (demotion timed inside the
                                solve) and FP64 refinement with the FP64 S; 0 = as precision */
    int32_t pcg_variant;     /* FP32 solves: BA_PCG_AUTO (0) or BA_PCG_SPLIT run CG on the
                                split system G^T S G (M^-1 = G G^T per camera; the same
                                iterates as block-Jacobi PCG in exact arithmetic) with one
                                grid-wide reduction per iteration; BA_PCG_STANDARD runs the
                                Sec. 3.2 recurrence as written.  FP64 solves always run it.
                                BA_PCG_IMPLICIT (any precision) runs the Sec. 3.2 recurrence
                                with S d applied from the stored linearization as
                                U d + lambda clamp(diag U) d - W V^-1 W^T d (the implicit
                                operator of ba_rcs_spmv; S is still formed for M^-1 and
                                the FP64 residual); the solve runs in the problem's
                                precision (solve_precision is ignored); refused by
                                ba_problem_create_rcs (no linearization). */
} ba_options;

typedef struct {
    double cost_before;      /* F(x) = 1/2 sum rho(||e||^2) before the step (FP64 sum) */
    double cost_after;       /* F after the step (== cost_before when rejected) */
    double cost_trial;       /* F(x (+) dx) of the trial point */
    double predicted;        /* 1/2(||e||^2 - ||e + J dx||^2), FP64 sum */
    double rho;              /* gain ratio (cost_before - cost_trial) / predicted */
    double lambda;           /* damping used by this step */
    int32_t accepted;
    int32_t pcg_iters;       /* PCG iterations, summed over refinement steps */
    int32_t refine_steps;    /* outer FP64 refinement steps (FP32 mode) */
    int32_t used_fallback;   /* reserved for a learned preconditioner */
    double rcs_rel_resid;    /* true ||b - S dx_c|| / ||b|| in FP64 */
    int64_t n_cheirality;    /* observations with z_cam <= 1e-6 at the trial point */
    int64_t n_v_fp64;        /* FP32 mode: points whose 3x3 V was re-factored in FP64 in
                                this step's RCS formation (kappa~ > 1e4) */
    float ms[8];             /* linearize, form_rcs, solve, trial cameras, back-substitution with
                                the trial evaluation (one pass over the points), total, -, - */
} ba_step_info;

typedef struct {
    int32_t n_cams;
    int64_t n_pts, n_obs;
    int64_t nnzb;            /* BSMC blocks (upper triangle incl. n diagonal blocks) */
    int64_t n_groups;        /* point groups (one CTA each in RCS formation) */
    int64_t n_partials;      /* sub-RCS blocks written by the groups */
    int64_t n_pairs;         /* (obs, obs) products: sum_k L_k (L_k + 1) / 2 */
    int64_t device_bytes;    /* device memory held by the problem */
    int64_t kernel_launches; /* kernels launched for this problem so far */
    int32_t precision;
    double pcg_phase_us[3];  /* profile >= 2: split CG iteration phases, mean over CTAs and
                                iterations of all solves so far, in us: SpMV passes (to the
                                CTA barrier), row combine and update, grid all-reduce */
    double rcs_phase_us[3];  /* profile >= 2: RCS formation per point group, mean over the
                                groups formed so far, in us, as the CTA's last thread sees
                                them: wait at the group's barrier, products and write-out,
                                then the next group's copy wait and per-point work (V_k,
                                Cholesky, P, e^) */
    double pcg_work_imbalance; /* profile >= 2: last split CG solve, the busiest CTA's
                                passes + combine time over the mean CTA's (1 = balanced) */
    int64_t n_v_fp64;        /* FP32 problems, last RCS formation: points whose damped 3x3
                                V_k was re-factored in FP64 because its FP32 factor gave
                                kappa~ = ||V||_F ||V^-1||_F > 1e4 */
} ba_stats;

/* Fills *o with the defaults listed above. */
void ba_options_default(ba_options *o);

/* Creates a problem.  cams: n_cams x 6 doubles [omega, t]; pts: n_pts x 3;
 * obs_cam[i] in [0, n_cams), obs_pt[i] in [0, n_pts), obs_uv: n_obs x 2 px.
 * Observation order is free.  Rejected with BA_ERR_INVALID_ARG: an index out
 * of range, a duplicated (camera, point) pair, a point with fewer than two
 * observations, a camera with none.  BA_ERR_NONFINITE: a NaN/Inf input.
 * Sets up the symbolic BSMC pattern (Sec. 4), the point groups (Sec. 6.1) and
 * the local-to-global block index (Table 1, second operation). */
ba_status ba_problem_create(const ba_options *opt, int32_t n_cams, const double *cams,
                            int64_t n_pts, const double *pts, int64_t n_obs,
                            const int32_t *obs_cam, const int64_t *obs_pt,
                            const double *obs_uv, ba_problem **out);

/* Creates a problem that holds a reduced camera system only (no observations),
 * for solving and for the learned preconditioner: row_ptr[n+1], col[nnzb],
 * val[nnzb x 36] (host, BSMC upper triangle of Sec. 4 with the full diagonal
 * block first in every row, columns ascending), b[n x 6].  The block-Jacobi
 * M^-1 is formed at creation.  ba_solve_rcs, the getters of the RCS and of
 * dx_c, ba_set_precond_net and the network calls work; the LM calls return
 * BA_ERR_STATE.  Rejected with BA_ERR_INVALID_ARG: a malformed pattern;
 * BA_ERR_NONFINITE: a NaN/Inf value; BA_ERR_NOT_SPD: a diagonal block that is
 * not positive definite. */
ba_status ba_problem_create_rcs(const ba_options *opt, int32_t n, int64_t nnzb, const int32_t *row_ptr,
                                const int32_t *col, const double *val, const double *b, ba_problem **out);

/* Residuals and Jacobians at the current state (Eq. 1's e and J, weighted by
 * sqrt(rho') under the Huber loss), stored on the device.  *cost_out (may be
 * NULL) receives F(x). */
ba_status ba_linearize(ba_problem *p, double *cost_out);

/* Forms the damped RCS of Eq. 4, S = U - W V^-1 W^T and b = l_c - W V^-1 l_p,
 * with U, V, W, l_c, l_p of Eq. 3 and D^T D = clamp(diag(J^T J), 1e-6, 1e32),
 * point group by point group (Sec. 5, Sec. 6.1), into BSMC; also the
 * block-Jacobi preconditioner (inverses of the diagonal blocks, Sec. 3.2).
 * Needs ba_linearize first. */
ba_status ba_form_rcs(ba_problem *p, double lambda);

/* Solves S dx_c = b by block-Jacobi PCG (Sec. 3.2, Eqs. 6-7) with y0 = 0 and
 * the stop rule ||r_k|| / ||r_0|| <= pcg_rel_tol; in FP32 mode by FP32 inner
 * PCG with FP64 iterative refinement.  info may be NULL. */
ba_status ba_solve_rcs(ba_problem *p, ba_step_info *info);

/* Eq. 5: dx_p = V^-1 (l_p - W^T dx_c) for every point. */
ba_status ba_back_substitute(ba_problem *p);

/* One LM iteration (Fig. 2): linearize (if the state changed), form the RCS,
 * solve, back-substitute, evaluate the trial point and accept or reject by
 * the gain ratio; lambda follows Nielsen's rule.  info may be NULL. */
ba_status ba_lm_step(ba_problem *p, ba_step_info *info);

/* Current state in the caller's order: n_cams x 6 and n_pts x 3 doubles. */
ba_status ba_get_cameras(const ba_problem *p, double *out_cams);
ba_status ba_get_points(const ba_problem *p, double *out_pts);

/* The last formed RCS in BSMC form: row_ptr[n+1], col[nnzb], val[nnzb x 36]
 * (row-major 6x6 blocks, upcast to double; the first block of every row is
 * the full diagonal block), b[n x 6].  Any array may be NULL; *nnzb always
 * receives the block count. */
ba_status ba_get_rcs(const ba_problem *p, int64_t *nnzb, int32_t *row_ptr, int32_t *col,
                     double *val, double *b);

/* Triangulation of every point from the current cameras, the alternative to
 * the back-substitution of Eq. 5 that Sec. 3.1 (after Eq. 5) and Sec. 5 name
 * without giving the method.  Per point: the least-squares solution of the
 * two equations each observation gives, linear in the point X (the pinhole
 * model with the depth multiplied out:
 * ((u - cx) R_3 - fx R_1) . X = fx t_1 - (u - cx) t_3 and likewise for v),
 * through its 3x3 normal equations, then gn_iters (0..50) Gauss-Newton steps
 * on the point's plain reprojection error.  FP64 problems compute in FP64;
 * FP32 problems in FP32, for the offset from the current point (camera-point
 * vectors from the FP32 state caches), added to it in FP64.  The points of the current state
 * are replaced (cameras unchanged; the linearization and RCS are dropped, as
 * by ba_set_state).  A point whose 3x3 system is not positive definite, or
 * whose result is not finite, keeps its value; n_failed_out (may be NULL)
 * receives their number.  cost_out (may be NULL) receives the cost at the
 * new state.  Errors: BA_ERR_INVALID_ARG, BA_ERR_STATE (RCS-only problem),
 * BA_ERR_CUDA. */
ba_status ba_triangulate(ba_problem *p, int32_t gn_iters, int64_t *n_failed_out, double *cost_out);

/* The last step: dxc[n x 6], dxp[n_pts x 3] (caller's point order). */
ba_status ba_get_step(const ba_problem *p, double *dxc, double *dxp);

/* The stored linearization in the caller's observation order:
 * e[n_obs x 2], Jc[n_obs x 12] (row-major 2x6), Jp[n_obs x 6] (2x3). */
ba_status ba_get_linearization(const ba_problem *p, double *e, double *Jc, double *Jp);

/* Replaces the state (caller's order) and the LM damping state. */
ba_status ba_set_state(ba_problem *p, const double *cams, const double *pts, double lambda,
                       double nu);
ba_status ba_get_lm_state(const ba_problem *p, double *lambda, double *nu, double *cost);

ba_status ba_get_stats(const ba_problem *p, ba_stats *out);

/* Kernel timing (options.profile != 0): for kernel id k (see ba_kernel_name)
 * the number of launches and their summed device time since the last reset. */
ba_status ba_get_kernel_time(ba_problem *p, int32_t k, int64_t *launches, double *total_ms);
ba_status ba_reset_kernel_times(ba_problem *p);
/* Sets options.profile of a live problem (0 none, 1 kernel times, 2 also the
 * phase timers inside the PCG and the RCS formation), so that one problem can
 * run untimed and then replay steps with its kernels timed; the times
 * gathered so far are kept.  BA_ERR_INVALID_ARG for a level outside 0..2. */
ba_status ba_set_profile(ba_problem *p, int32_t level);

/* Test hook for the bounded device waits (not part of the method).  Every
 * grid-wide wait inside the library gives up after a limit of SM clock cycles
 * (about 2 s), sets an error word the host reads, and leaves its kernel, so
 * that a stalled wait ends as a status instead of a hung GPU.  This call arms
 * the next PCG launch of p (the split CG of FP32 solves or the Sec. 3.2
 * recurrence) to start its all-reduce arrival counters one arrival short of
 * their targets and to wait at most limit_cycles (1 .. 4e9) cycles: the first
 * all-reduce then runs out on every CTA, the kernel leaves after its copies
 * in flight have landed, and the solve returns BA_ERR_TIMEOUT.  As after any
 * BA_ERR_TIMEOUT, p is then unusable (later calls on it return BA_ERR_STATE;
 * ba_problem_destroy still frees it) while the CUDA context and other
 * problems are unaffected.  The arming is used up by that one launch. */
ba_status ba_debug_arm_wait_timeout(ba_problem *p, int64_t limit_cycles);
const char *ba_kernel_name(int32_t k); /* NULL past the last id */

void ba_problem_destroy(ba_problem *p);

/* Message of the last failed call on this thread ("" if none). */
const char *ba_last_error(void);

/* Host-only (no GPU needed): the structural BSMC pattern of an observation
 * set - every diagonal block plus each (i < j) whose cameras share a point,
 * rows in order, columns ascending (Sec. 4, Fig. 4).  row_ptr receives n+1
 * entries; col (may be NULL for a size query) nnzb entries. */
ba_status ba_symbolic_pattern(int32_t n_cams, int64_t n_pts, int64_t n_obs,
                              const int32_t *obs_cam, const int64_t *obs_pt, int32_t *row_ptr,
                              int32_t *col, int64_t *nnzb);

/* ---- Storage formats of the RCS (Sec. 4, Table 1, Eqs. 8-10) -------------
 * y = S x with the problem's current RCS held in one of three formats, each
 * with its own GPU kernel, so that the paper's storage comparison can be
 * measured (Table 1 lists the operations a format must serve; Eqs. 8-10 give
 * the bytes of scalar CSR and of BSMC):
 *   BA_FMT_BSMC      the library's storage: upper-triangle 6x6 blocks, the
 *                    full diagonal block first in every row (Fig. 4); the
 *                    product applies each off-diagonal block twice, as S_ij x_j
 *                    and as S_ij^T x_i (a warp per block row over its two-sided
 *                    entry list: no atomics, deterministic);
 *   BA_FMT_BSR_FULL  block CSR of the whole symmetric matrix: both triangles
 *                    stored as row-major 6x6 blocks, a column index per block,
 *                    n + 1 row starts;
 *   BA_FMT_CSR       scalar CSR of the whole matrix (Eq. 8): a value and a
 *                    column index per element of every non-zero block, 6n + 1
 *                    row starts.
 *   BA_FMT_IMPLICIT  no stored S (the aggregation-free next step the paper
 *                    states, Sec. 8): the product from the stored linearization,
 *                    S x = U x + lambda clamp(diag U) x - W V^-1 W^T x with the
 *                    per-point factors of V of the last ba_form_rcs (same
 *                    lambda); a thread per point forms V^-1 W^T x, a warp per
 *                    camera sums its observations; needs a linearized problem
 *                    (not an RCS-only one).  bytes_out: what one product reads
 *                    instead of S (J rows, the factors, a work vector, the
 *                    camera-major index).
 *   BA_FMT_BSMC_ONCE the library's BSMC read once: a warp per block row applies
 *                    each stored block as S_ij x_j to its row and as S_ij^T x_i
 *                    to row j, both added into y (L2-resident) with vector
 *                    reductions, so no block is read twice (the two-sided
 *                    product reads each off-diagonal block twice, and beyond L2
 *                    moves that many bytes); the order of y's terms is not
 *                    fixed, so results may differ in the last bits between
 *                    runs.  Same arrays and bytes as BA_FMT_BSMC.  y (FP32:
 *                    8-byte aligned, as any cudaMalloc'd array) is zeroed first
 *                    on the stream, as part of the product.
 * The three two-sided stored formats sum each row's blocks in the same order.  x and y are DEVICE
 * arrays of 6n values in the problem's precision (double for BA_FP64
 * problems, float for BA_FP32), owned by the caller, not overlapping; the
 * product is queued on the problem's stream (no synchronisation).  The full
 * formats are built on the device from the current S on the first call after
 * each RCS is formed (ba_form_rcs, ba_lm_step, ba_problem_create_rcs) and are
 * owned by the problem.  bytes_out (host, may be NULL) receives the format's
 * array bytes: values + column indices + row starts.  Errors:
 * BA_ERR_INVALID_ARG (bad format or NULL array), BA_ERR_STATE (no RCS
 * formed), BA_ERR_OOM, BA_ERR_CUDA. */
typedef enum { BA_FMT_BSMC = 0, BA_FMT_BSR_FULL = 1, BA_FMT_CSR = 2, BA_FMT_IMPLICIT = 3,
               BA_FMT_BSMC_ONCE = 4 } ba_rcs_format;
ba_status ba_rcs_spmv(ba_problem *p, int32_t format, const void *x, void *y, int64_t *bytes_out);

/* ---- Learned block-Jacobi correction (not in the paper) ------------------
 * The paper preconditions PCG with the block diagonal of the RCS (Sec. 3.2).
 * A small network corrects each block's inverse while keeping it SPD:
 *   S_ii = L_i L_i^T,  M_i^-1 = L_i^-T T_i T_i^T L_i^-1,
 * T_i lower triangular with T_kk = exp(0.1 o_kk), T_kl = 0.1 o_kl (k > l), o_i the
 * 21 outputs of two message-passing layers (hidden 64, BF16 weights on the
 * tensor cores, FP32 accumulation) over the camera co-visibility graph: nodes
 * are cameras, edges the off-diagonal BSMC blocks with weight
 * ||S_ij||_F / sqrt(||S_ii||_F ||S_jj||_F).  Node features: the 15 correlations
 * of S_ii, its 6 log-diagonals centred over cameras, log(1 + degree), summed
 * edge weight, 1.  Layer: h' = relu([h | mean_w(neighbours' h)] W + b).
 * Zero output weights give exactly block-Jacobi.
 * Parameters (FP32 master, packed): W1 (48 x 64), b1 (64), W2 (128 x 64),
 * b2 (64), Wo (64 x 21), bo (21), row-major. */
typedef struct ba_precond_net ba_precond_net;

int32_t ba_precond_net_num_params(void);

/* params: host array of ba_precond_net_num_params() floats, or NULL for a
 * seeded He-normal initialisation with a zero output layer. */
ba_status ba_precond_net_create(const float *params, uint64_t seed, void *cuda_stream, ba_precond_net **out);
void ba_precond_net_destroy(ba_precond_net *net);
ba_status ba_precond_net_get_params(const ba_precond_net *net, float *out);
ba_status ba_precond_net_set_params(ba_precond_net *net, const float *params);

/* Attach a network to a problem (NULL detaches): ba_solve_rcs then uses the
 * corrected M^-1, and falls back to plain block-Jacobi (info->used_fallback = 1)
 * if the learned PCG breaks down or misses its tolerance.  The network must
 * outlive the attachment. */
ba_status ba_set_precond_net(ba_problem *p, ba_precond_net *net);

/* Forward pass on the problem's last formed RCS: out_o (n x 21) and out_minv
 * (n x 36), host buffers, either may be NULL. */
ba_status ba_precond_net_forward(ba_precond_net *net, ba_problem *p, float *out_o, double *out_minv);

/* Training step on the problem's last formed RCS with kp probe vectors w_p
 * (host array kp x n x 6, or NULL for Rademacher probes from seed).  The loss
 * is the S-norm error left by one preconditioned Richardson step with the
 * optimal step length:  u_p = S w_p, z_p = M^-1 u_p, a = sum z_p^T u_p,
 * c = sum z_p^T S z_p, e = sum w_p^T u_p, loss = 1 - a^2 / (c e).
 * Gradients by the network's backward pass (tensor-core GEMMs); if lr > 0 an
 * Adam step (0.9, 0.999, 1e-8) updates the parameters.  loss and grads (host,
 * num_params floats) may be NULL. */
ba_status ba_precond_net_train_step(ba_precond_net *net, ba_problem *p, int32_t kp, const float *probes,
                                    uint64_t seed, double lr, double *loss, float *grads);

/* Small GEMM on the tensor cores (the operation of the learned preconditioner's
 * dense layers): C[M x N] = A[M x K] * B[K x N], or C += A * B when
 * accumulate != 0.  Device pointers; element (r, c) of A is A[r * a_rs + c * a_cs]
 * (likewise B, C), so transposed operands need no copy.  A and B are rounded to
 * BF16 and multiplied on the 5th-generation tensor cores (tcgen05) with FP32
 * accumulation.  N must be 32, 64, 96 or 128; M and K are free (K is split in
 * chunks of 128 whose results are added atomically).  err_dev (device int, may
 * be NULL) receives BA_ERR_TIMEOUT if a bounded device wait gave up. */
ba_status ba_tc_gemm(int32_t M, int32_t N, int32_t K, const float *A, int64_t a_rs, int64_t a_cs,
                     const float *B, int64_t b_rs, int64_t b_cs, float *C, int64_t c_rs, int64_t c_cs,
                     int32_t accumulate, int32_t *err_dev, void *cuda_stream);

/* Allocation-free PCG for callers that cannot call cudaMalloc.
 *
 * The paper has no counterpart of this entry point; it serves callers that
 * must not allocate device memory: code running while a framework owns the
 * device memory pool (a caching allocator or a fixed arena), real-time loops
 * that cannot take the allocator's lock or its implicit synchronisation, and
 * hosts under a hard device-memory budget.  It solves S x = b by block-Jacobi
 * PCG in FP32 (the iteration of ba_solve_rcs: y0 = 0, stop when
 * ||r_k|| / ||r_0|| <= rel_tol or after max_iters iterations, 0 meaning
 * max(1000, 6n)).
 *
 * All pointers are DEVICE pointers owned by the caller: row_ptr[n+1],
 * col[nnzb] and val[nnzb x 36] are an FP32 BSMC matrix in the layout that
 * ba_get_rcs returns (upper-triangle 6x6 blocks, row-major, the full diagonal
 * block first in every row, the other columns ascending above the row),
 * b[n x 6] the right-hand side, x[n x 6] receives the solution.  Only the
 * upper triangle may be stored: the product applies every off-diagonal block
 * also as its transpose, so a matrix passed with both triangles would count
 * them twice.  The pattern is checked on the device before the first
 * iteration (row_ptr[n] == nnzb, the diagonal block first, ascending columns
 * in [i, n)); a malformed one returns BA_ERR_INVALID_ARG, and a diagonal
 * block that is not positive definite BA_ERR_NOT_SPD, both after zero
 * iterations.  iters_out and rel_resid_out (host pointers, may be NULL)
 * receive the iteration count and the final ||r|| / ||r_0||.
 *
 * Scratch: one fixed array of about 2.2 MB in the library's device code,
 * present on every GPU that loads the library until the process exits; n is
 * limited to 8192 cameras (larger n returns BA_ERR_INVALID_ARG).  The first
 * call on a device looks up the array's device address with that device
 * current; make that first call before any stream capture.  All calls share
 * the one array: calls that overlap on the GPU race on it.  Each call clears
 * the parts that must start at zero.  The call allocates nothing (no
 * cudaMalloc / cudaFree) and synchronises the stream every eight iterations
 * to read the stop flag.  Errors: BA_ERR_INVALID_ARG, BA_ERR_NOT_SPD,
 * BA_ERR_NO_CONVERGENCE (x holds the last iterate), BA_ERR_CUDA. */
ba_status ba_pcg_solve_static(int32_t n, int64_t nnzb, const int32_t *row_ptr, const int32_t *col,
                              const float *val, const float *b, float *x, double rel_tol,
                              int32_t max_iters, void *cuda_stream, int32_t *iters_out,
                              double *rel_resid_out);

#ifdef __cplusplus
}
#endif
#endif /* BA_H */
