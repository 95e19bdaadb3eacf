// Internal declarations of libba: the problem object, the host-side symbolic
// setup and the kernel launchers.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ba.h"

namespace ba {

// One observation row of the stored linearization: [J_c (2x6) | J_p (2x3) | e (2)].
constexpr int JW = 20;
// One BSMC block / one sub-RCS partial block: 6x6 values.  A diagonal partial
// packs [21 upper entries of U - W V^-1 W^T | 6 diag(J_c^T J_c) | 6 b | 3 unused].
constexpr int BW = 36;
constexpr int OBS_MAX_DEFAULT = 512;  // observations staged per point group
constexpr int OBS_MAX_LIMIT = 1024;
constexpr int LB_MAX = 2048;          // local blocks (sub-RCS blocks) per group
constexpr int C_MAX = 4096;           // (obs, obs) products per group (staged in shared memory)
constexpr int ITEM_MAX = 8;           // products per work item
constexpr int FORM_THREADS = 256;
constexpr int CAMC32_W = 32;          // floats per camera of the FP32 camera cache

// A point group: a run of whole point tracks formed by one CTA (Sec. 6.1).
struct GroupDesc {
    int64_t c_begin;     // first (a, b) product in the contribution array
    int64_t part_begin;  // first partial written by the group
    int64_t item_begin;  // first work item
    int32_t obs_begin, nobs;
    int32_t pt_begin, npts;
    int32_t nitems, nc;
};

// A work item: up to ITEM_MAX products of one sub-RCS block.
//   x: cbeg (16) | cnt (4) << 16 | diag << 20 | nfollow (5) << 21 | head << 26
//   y: partial index (relative to the group) written by the head item
// Items sit 32 to a warp in order; a block's consecutive items within a warp
// form a run, summed by a segmented shuffle reduction into the run's head.
struct ItemDesc {
    uint32_t x, y;
};

// Device-resident scalars of the reductions and of the PCG recurrence.
struct DevScalars {
    double cost, cost_trial, model;
    double rz, pAp, rr, rr0, alpha, beta, tol2;
    double rr64, bb64;
    unsigned long long n_cheir, n_cheir_trial, n_v64;
    unsigned long long n_tri_fail;  // points triangulation left unchanged (last ba_triangulate)
    int iters, done, max_iters, err;
    int prof_on;   // split CG: time its phases (profile >= 2)
    double ph[4];  // split CG phase ns summed over CTAs and iterations; ph[3] = CTA iterations
    double ph_rcs[4];  // RCS formation phase ns summed over groups (profile >= 2); [3] = groups
    unsigned long long ph_work_max;  // split CG: largest per-CTA total of passes + combine ns, one solve
};
constexpr int N_COUNTERS = 16;
constexpr int RED_SLOTS = 4096 * 4;  // per-CTA partial sums

enum KernelId {
    K_PREPARE = 0, K_LINEARIZE, K_COST, K_FORM_RCS, K_RCS_REDUCE, K_RCS_DIAG,
    K_PCG_INIT, K_PCG_LOOP, K_RESID64, K_BACKSUB, K_UPDATE, K_DEMOTE, K_SPLIT_PREP, K_STEP_POINTS, K_TRIANGULATE,
    K_COUNT
};
const char *kernel_name(int k);

// Result of the host-side symbolic phase (Sec. 4 pattern, Sec. 6.1 groups,
// Table 1 second operation for the local -> global block index).
struct HostSetup {
    std::vector<int64_t> pt_perm;    // internal point -> caller's point
    std::vector<int64_t> obs_perm;   // internal observation -> caller's observation
    std::vector<int32_t> obs_cam;    // internal order: sorted by (internal point, camera)
    std::vector<int32_t> obs_pt;
    std::vector<int32_t> trk_ptr;    // P + 1
    std::vector<int32_t> row_ptr;    // n + 1
    std::vector<int32_t> col;        // nnzb
    std::vector<int32_t> ct_ptr;     // n + 1: blocks (j < i, i) of column i ...
    std::vector<int32_t> ct_blk;     // ... their BSMC ids, j ascending
    std::vector<int32_t> ct_row;     // ... and their rows j
    std::vector<int32_t> tw_ptr;     // n + 1: entries of row i for the SpMV ...
    std::vector<int2> tw_ent;        // ... {block id | transposed << 31, column j}: row blocks, then column blocks
    std::vector<GroupDesc> groups;
    std::vector<ItemDesc> items;
    std::vector<int32_t> lb_gblk;    // global block of each partial
    std::vector<uint32_t> contrib;   // a | b << 16 (observation offsets in the group)
    std::vector<int32_t> pptr;       // nnzb + 1: partials of each global block
    std::vector<int32_t> plist;
    int64_t n_pairs = 0;
    int32_t max_nobs = 0, max_nc = 0;  // largest group: observations, products
};

// Column index and two-sided SpMV entry lists from hs.row_ptr / hs.col.
void build_twosided(HostSetup &hs, int32_t n);

// Validates the observation set and builds everything above.  Returns BA_OK or
// BA_ERR_INVALID_ARG with a message.
ba_status symbolic_setup(int32_t n, int64_t P, int64_t m, const int32_t *obs_cam,
                         const int64_t *obs_pt, const double *pts, int obs_max, bool pattern_only,
                         HostSetup &hs, std::string &err);

// A parameter state with its derived per-camera / per-point caches.
struct StateBuf {
    double *cams = nullptr;   // n x 6  [omega, t]
    double *pts = nullptr;    // P x 3  (internal point order)
    void *camc = nullptr;     // FP64: n x 12 [R, t]; FP32: n x 32 [R_hi, C_hi, C_lo, 0, R_lo, 0 x 7]
    float *pts_hl = nullptr;  // FP32 mode: P x 6 [X_hi, X_lo]
    float *e = nullptr;       // FP32 mode: m x 2 residuals of the state (double-float arithmetic, rounded)
};

}  // namespace ba

struct ba_precond_net;
namespace ba {
struct GnnWork;
// The buffers a PCG solve runs on: the problem's own, or FP32 shadows of an
// FP64 problem's system (mixed-precision solve).
struct SolverView {
    bool f32 = false;
    void *S = nullptr, *Minv = nullptr;
    void *pv[8] = {};
};
}  // namespace ba

struct ba_problem {
    ba_options opt{};
    cudaStream_t st = nullptr;
    int32_t n = 0;
    int64_t P = 0, m = 0;
    bool fp32 = false;
    size_t esz = 8;
    int obs_max = ba::OBS_MAX_DEFAULT;
    ba::HostSetup hs;
    int64_t nnzb = 0, ngroups = 0, npart = 0;
    size_t dev_bytes = 0;
    std::vector<void *> allocs;

    ba::StateBuf cur, trial;
    int32_t *obs_cam = nullptr, *obs_pt = nullptr, *trk_ptr = nullptr;
    double *uv64 = nullptr;
    float *uv32 = nullptr;
    float *uv_lo = nullptr;   // FP32 mode: uv - uv32 (the observations' lo parts for the double-float cost)
    void *J = nullptr;
    int32_t *row_ptr = nullptr, *col = nullptr;
    int32_t *ct_ptr = nullptr, *ct_blk = nullptr, *ct_row = nullptr;
    int32_t *tw_ptr = nullptr;
    int2 *tw_ent = nullptr;
    void *S = nullptr, *b = nullptr, *Minv = nullptr;
    // S's generation (bumped whenever an RCS is formed or loaded) and the
    // full-block and scalar CSR copies of S for ba_rcs_spmv, with the
    // generation each was built from
    uint64_t rcs_gen = 0, fmt_gen[3] = {~0ull, ~0ull, ~0ull};
    void *fmt_bsr_val = nullptr, *fmt_csr_val = nullptr;
    int32_t *fmt_bsr_col = nullptr, *fmt_csr_ptr = nullptr, *fmt_csr_col = nullptr;
    double *tri_cam64 = nullptr;  // n x 12 FP64 [R | t] for the triangulation
    // implicit S x (ba_rcs_spmv BA_FMT_IMPLICIT): camera-major observation
    // index and the per-observation work vector
    int32_t *imp_cam_ptr = nullptr, *imp_cam_obs = nullptr;
    void *imp_w = nullptr;
    ba::GroupDesc *grp = nullptr;
    ba::ItemDesc *items = nullptr;
    uint32_t *contrib = nullptr;
    int64_t nitems = 0;
    int32_t *pptr = nullptr, *plist = nullptr;
    void *part = nullptr;
    void *Linv = nullptr, *lp = nullptr;
    void *pv[8] = {};  // y, r, z, d0, d1, q, r', q'   (n x 6, mode precision)
    double *x64 = nullptr, *r64 = nullptr, *q64 = nullptr;
    void *dxc = nullptr, *dxp = nullptr;
    ba::DevScalars *sc = nullptr;
    ba::DevScalars *sc_host = nullptr;  // pinned mirror
    double *red = nullptr;
    unsigned *counters = nullptr;

    double lambda = 1e-4, nu = 2.0, F = 0.0;
    bool have_F = false, linearized = false, rcs_formed = false, solved = false, backsub = false;
    bool step_diff = false;              // this step's trial cost is F plus its change (FP32 mode)
    double last_rel_decrease = INFINITY;  // (F - F') / F of the last accepted step
    bool dead = false;
    double rcs_lambda = 0.0;
    int last_pcg_iters = 0, last_refine = 0;
    double last_true_rel = 0.0;

    // kernel timing
    std::vector<cudaEvent_t> ev_pool;
    struct Pending { int k; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    int64_t klaunch[ba::K_COUNT] = {};
    double kms[ba::K_COUNT] = {};
    int64_t launches = 0;  // every kernel launched on behalf of this problem
    cudaEvent_t step_ev[6] = {};  // phase boundaries of ba_lm_step (ba_step_info.ms)

    // solve view and FP32 shadows (FP64 problems solved in mixed precision)
    ba::SolverView sv;
    void *S32 = nullptr, *Minv32 = nullptr, *pv32[8] = {};
    bool rcs_only = false;  // created from a BSMC system: no observations

    // learned preconditioner (optional)
    ba_precond_net *net = nullptr;
    ba::GnnWork *gw = nullptr;
    void *Minv_bj = nullptr;  // block-Jacobi copy kept for the fallback
    int last_used_fallback = 0;

    // split-preconditioned FP32 CG: per-camera factors G, H = G^-T (n x 36),
    // S^ = G^T S G in two-sided entry order (one block per entry), the vector
    // records; allocated on the first such solve
    float *Gs = nullptr, *Hs = nullptr, *Sh = nullptr, *srec = nullptr;
    float *Shd = nullptr;            // diagonal blocks of S^ when they are not the identity (n x 36)
    int32_t *tws_ptr = nullptr;      // two-sided entry lists without the diagonal block (n + 1) ...
    int2 *tws_ent = nullptr;         // ... and their entries
    int32_t *cta_rows = nullptr;   // row range of each CTA of the balanced SpMV
    uint32_t *tw_meta = nullptr;   // per entry: local row | halo index << 16 (per-CTA aligned)
    int32_t *meta_off = nullptr, *halo_ptr = nullptr, *halo_col = nullptr, *own_base = nullptr;
    int split_grid = 0;            // 0: not partitioned yet, < 0: unavailable
    int split_slot_floats = 0;
    size_t split_smem = 0;
    double ph_sum[4] = {};  // split CG phase totals over solves (profile >= 2)
    double ph_imbalance = 0.0;  // last split solve: busiest CTA's work / mean CTA's
    bool minv_learned = false;  // Minv holds the learned M^-1 (else block-Jacobi)
    float2 *xs = nullptr;  // x64 split in FP32 pairs (refinement residual of FP32 problems)
    unsigned *ar_bar = nullptr;  // arrival counters of the split CG's all-reduce (one per line)
    // > 0: the next PCG launch (split or standard recurrence) starts its
    // all-reduce counters one arrival short and waits at most this many SM
    // cycles (ba_debug_arm_wait_timeout; a test of the timeout path)
    long long test_wait_limit = 0;

    // caller-order point I/O on the device, allocated on first use: the
    // internal -> caller permutation, a P x 3 staging buffer, a flag word
    int32_t *d_perm = nullptr;
    double *stage_pts = nullptr;
    unsigned *io_flag = nullptr;
};

namespace ba {

// sets the calling thread's ba_last_error() message and returns s
ba_status set_error(ba_status s, const char *msg);

// kernel timing helpers (active when opt.profile != 0)
void ktimer_begin(ba_problem *p, int k, cudaEvent_t *a);
void ktimer_end(ba_problem *p, int k, cudaEvent_t a);
ba_status ktimer_flush(ba_problem *p);

// launchers (kernels in the .cu files); each returns cudaGetLastError()
cudaError_t launch_prepare_state(ba_problem *p, StateBuf &s);
// caller-order point I/O through a device staging buffer (d_perm, stage_pts)
cudaError_t launch_count_nonfinite(ba_problem *p, const double *a, int64_t cnt, unsigned *bad);
cudaError_t launch_gather_pts(ba_problem *p, const double *user, double *internal);
cudaError_t launch_scatter_pts(ba_problem *p, const void *internal, bool internal_fp32, double *user);
cudaError_t launch_linearize(ba_problem *p);
cudaError_t launch_cost(ba_problem *p, StateBuf &s, bool trial);
cudaError_t launch_form_rcs(ba_problem *p, double lambda);
cudaError_t launch_pcg_init(ba_problem *p, const void *rhs_T, double tol, int max_iters);
cudaError_t launch_pcg_loop(ba_problem *p);
cudaError_t launch_pcg_implicit(ba_problem *p);  // the loop on the implicit operator (k_formats.cu)
cudaError_t launch_resid64(ba_problem *p, bool from_x64);
cudaError_t launch_solution_to_step(ba_problem *p);
cudaError_t launch_refine_rhs(ba_problem *p, void *rhs_T);
cudaError_t launch_back_substitute(ba_problem *p);
// LM step tail: trial cameras, then the fused point pass (Eq. 5, trial points,
// trial cost and model decrease)
cudaError_t launch_trial_cameras(ba_problem *p);
cudaError_t launch_step_points(ba_problem *p);
cudaError_t launch_block_jacobi(ba_problem *p);               // Minv from the diagonal blocks of S
cudaError_t launch_demote(ba_problem *p);                     // S32, Minv32 from the FP64 S, Minv
// split-preconditioned FP32 CG: G, H and S^ = G^T S G from the problem's S
// (block-Jacobi) or its current M^-1 (from_minv); init, the persistent loop
// and x64 (+)= G x^
cudaError_t launch_split_prepare(ba_problem *p, bool from_minv);
bool split_available(ba_problem *p);  // partitions on first use
cudaError_t launch_split_init(ba_problem *p, const float *rhs, double tol, int max_iters);
cudaError_t launch_pcg_split(ba_problem *p);
cudaError_t launch_accumulate_split(ba_problem *p, bool first);
// y = S x for one FP32 vector (learned-preconditioner probes)
cudaError_t launch_spmv_f32(ba_problem *p, const float *x, float *y);
// every point re-triangulated from the current cameras (k_obs.cu)
cudaError_t launch_triangulate(ba_problem *p, int gn_iters);
// Resident CTAs of a kernel on the current device at a block size and dynamic
// shared-memory size: *per_sm and *n_sm (the SM count).  Computed once per
// (device, kernel, threads, smem) and cached under a lock.
cudaError_t occupancy(const void *kernel, int threads, size_t smem, int *per_sm, int *n_sm);
// RCS storage formats (k_formats.cu)
cudaError_t launch_rcs_format_build(ba_problem *p, int format);
cudaError_t launch_rcs_spmv(ba_problem *p, int format, const void *x, void *y);
int64_t rcs_format_bytes(const ba_problem *p, int format);
// learned preconditioner: M^-1 of the last formed RCS from the attached net
// (the block-Jacobi M^-1 is saved first); restore the block-Jacobi M^-1
ba_status gnn_apply(ba_problem *p);
ba_status gnn_restore_block_jacobi(ba_problem *p);
void gnn_free(ba_problem *p);

}  // namespace ba
