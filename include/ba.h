/*
 * ba.h - C ABI of the GB300 (sm_103a) linear-solve library for Levenberg-Marquardt
 * bundle adjustment, after "Multigrid for Bundle Adjustment" (Konolige & Brown).
 *
 * The library solves, once per LM step, the damped normal equations of Section 2.1,
 *     (J^T J + D) delta = -J^T f,
 * by eliminating the points (Schur complement S = A - F^T E C^-1 E^T F, Section 2.1)
 * and running preconditioned conjugate gradients on S, applied implicitly from the
 * per-observation Jacobian blocks (Section 3.6), with the unsmoothed-aggregation
 * multigrid V-cycle of Section 3 (Algorithm 1, Algorithm 2) as the preconditioner.
 *
 * Conventions (all entry points):
 *  - Array arguments are DEVICE pointers unless the comment says "host".  Callers own
 *    them; the library never keeps a pointer past the call, except as stated for
 *    ba_create.  float64, row-major, densely packed.
 *  - cams: n_cams x 9 rows [r0 r1 r2 (angle-axis), t0 t1 t2, f, k1, k2];
 *    pts: n_pts x 3; obs: n_obs x 2 pixel coordinates, in the caller's observation
 *    order (the order of cam_idx / pt_idx given to ba_create).
 *  - Camera vectors (rhs, delta_c, dL_dcams): n_cams x 9; point vectors n_pts x 3.
 *  - All GPU work is enqueued on the stream given to ba_create.  Entry points that
 *    return host scalars synchronise that stream before returning.
 *  - Errors are returned as a ba_status and never trap the GPU; ba_last_error gives
 *    a message.  A failed call leaves the problem usable (the next ba_linearize
 *    starts afresh) unless the status is BA_ERR_CUDA.
 *  - The problem object is not thread-safe; use one per host thread.
 */
#ifndef BA_H_
#define BA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ba_problem ba_problem; /* opaque, owned by the library */

typedef enum {
  BA_OK = 0,
  BA_ERR_INVALID_ARG = 1,   /* bad size, index out of range, duplicate (camera, point) pair */
  BA_ERR_CUDA = 2,          /* a CUDA call failed; the problem should be destroyed */
  BA_ERR_OOM = 3,           /* device allocation failed */
  BA_ERR_NOT_SPD = 4,       /* a 3x3 point block, a Jacobi block or the coarse matrix is not SPD */
  BA_ERR_BREAKDOWN = 5,     /* PCG breakdown: p^T S p <= 0 or a non-finite scalar */
  BA_ERR_NOT_CONVERGED = 6, /* max_iters reached; delta_c still holds the last iterate */
  BA_ERR_LIMIT = 7,         /* a documented capacity limit was exceeded (see ba_last_error) */
  BA_ERR_STATE = 8          /* entry points called out of order (e.g. solve before setup) */
} ba_status;

typedef enum { BA_FP64 = 0, BA_MIXED = 1 } ba_precision;
typedef enum { BA_PRECOND_NONE = 0, BA_PRECOND_JACOBI = 1, BA_PRECOND_MG = 2 } ba_precond;
typedef enum { BA_DAMP_MARQUARDT = 0, BA_DAMP_IDENTITY = 1 } ba_damping;
/* Level-0 operator of the V-cycle (Section 3.6 weighs applying the camera system
 * implicitly from the Jacobian blocks against assembling it): IMPLICIT streams the
 * per-observation blocks on every product; EXPLICIT uses the 9x9 block-sparse S that
 * ba_mg_setup assembles anyway for the Galerkin product; AUTO picks EXPLICIT when its
 * blocks take fewer bytes than one implicit pass over the Jacobian.  The level 0 is the
 * PCG's own operator S, so the same choice decides the outer PCG product: with the
 * assembled level 0 the PCG multiplies by its blocks (FP64 blocks in BA_FP64, float-pair
 * blocks in BA_MIXED), otherwise by the implicit product. */
typedef enum { BA_OP_IMPLICIT = 0, BA_OP_EXPLICIT = 1, BA_OP_AUTO = 2 } ba_operator;
/* Arithmetic of the outer PCG product S p in BA_MIXED (BA_FP64 always uses FP64):
 * FP64 instructions, or FP64-valued operands carried as pairs of floats (hi + lo, about
 * 48 significant bits) and combined with error-free FP32 transformations, which this
 * GPU issues at many times its FP64 rate.  The PCG vectors, dot products, residual and
 * the product's accumulation stay FP64 either way. */
typedef enum { BA_OUTER_FP64 = 0, BA_OUTER_PAIRED_FP32 = 1 } ba_outer_product;
/* PCG stopping rule: the relative recursive residual |r_i| <= rtol |b|, or the
 * Nash-Sofer forcing rule of Section 2.1, i (Q_i - Q_{i-1}) / Q_i <= tau with the
 * quadratic model Q_i = 1/2 x_i^T S x_i - x_i^T b (Q_0 = 0), evaluated from the CG
 * recurrence Q_i - Q_{i-1} = -alpha_i (r_{i-1}^T z_{i-1}) / 2. */
typedef enum { BA_STOP_RELRES = 0, BA_STOP_NASH_SOFER = 1 } ba_stop_rule;
/* Loss on the squared residual norm s_o = |f_o|^2 (Section 5's robust error metric):
 * SQUARED rho(s) = s; HUBER rho(s) = s for s <= a^2 and 2 a sqrt(s) - a^2 beyond
 * (a = loss_scale; the paper's a = 1 pixel).  The objective is 1/2 sum_o rho(s_o).  With
 * HUBER each residual and its Jacobian blocks are scaled by w_o = sqrt(rho'(s_o))
 * (1 inside, (a^2 / s_o)^(1/4) outside) before the Schur reduction, the corrected
 * Gauss-Newton model of Triggs et al. (exact here since rho'' <= 0). */
typedef enum { BA_LOSS_SQUARED = 0, BA_LOSS_HUBER = 1 } ba_loss;

typedef struct {
  double lambda;        /* LM damping used by ba_lm_step's first call (Section 5: 1/1e4) */
  double rtol;          /* PCG stop: |r_k| <= rtol |b|, r the recursive residual */
  int max_iters;        /* PCG iteration cap (1000) */
  int precision;        /* ba_precision: BA_FP64 all-double; BA_MIXED FP32 V-cycle */
  int preconditioner;   /* ba_precond (BA_PRECOND_MG) */
  int damping;          /* ba_damping: D = lambda*max(diag(J^T J),1e-6) or lambda*I */
  int recompute_jacobian; /* 1: the FP64 implicit Schur product (the PCG product and the V-cycle's
                           level 0 when implicit; BA_OUTER_FP64 in BA_MIXED) rebuilds F and E of
                           each observation from the cameras and points instead of reading stored
                           blocks, trading 192 streamed bytes per observation for about 300 FP64
                           operations, and the FP64 blocks are then never formed in BA_MIXED.
                           The paired-FP32 and FP32 products read stored blocks either way (0);
                           ba_adjoint always rebuilds its blocks */
  int max_agg;          /* Algorithm 2 aggregate size cap (20, Section 3.2) */
  int pre_smooth;       /* Chebyshev steps before the coarse correction, 1 .. 8 (2, Section 3.4) */
  int post_smooth;      /* Chebyshev steps after, 1 .. 8 (2) */
  int lanczos_steps;    /* operator applications for lambda_max (5, Section 3.4) */
  int coarse_max_nodes; /* stop coarsening at <= this many nodes (32) */
  int max_levels;       /* hierarchy depth cap (10) */
  double cheb_lo;       /* Chebyshev interval [cheb_lo, cheb_hi] * lambda_max (0.3, 1.1) */
  double cheb_hi;
  int level0_operator;  /* ba_operator of the V-cycle's finest level (BA_OP_AUTO) */
  int fused_vcycle;     /* 1: with an assembled level 0, fuse each block-sparse product of the
                           V-cycle into the smoothing or restriction step that consumes it (1) */
  int outer_product;    /* ba_outer_product used by BA_MIXED (BA_OUTER_PAIRED_FP32) */
  int stop_rule;        /* ba_stop_rule (BA_STOP_RELRES) */
  double tau;           /* Nash-Sofer tolerance (0.1; Section 5 uses 0.1 and 0.01) */
  int overlap_launches; /* 1: launch the PCG loop's kernels as programmatic dependent launches,
                           so each is scheduled while its predecessor finishes (1) */
  int loss;             /* ba_loss (BA_LOSS_SQUARED) */
  double loss_scale;    /* a of BA_LOSS_HUBER, in residual units (1.0) */
  double precond_lambda_min; /* BA_MIXED: the FP32 multigrid hierarchy is built from S at damping
                           max(lambda, precond_lambda_min); PCG still solves S at lambda.  Below
                           about 1e-6 the damping that keeps S's near-null (gauge) eigenvalues
                           apart from zero falls under the FP32 rounding of S's entries and the
                           FP32 hierarchy stops preconditioning (1e-5; 0 disables) */
  int schur_staging;    /* FP32 implicit product (BA_OP_IMPLICIT in BA_MIXED): 1 stages each warp's
                           coming observation records into a double buffer in shared memory with
                           asynchronous bulk copies; 0 loads them straight into registers, which
                           keeps twice the warps resident and is faster (0) */
} ba_options;

/* Fills *opt with the defaults listed above. */
void ba_default_options(ba_options* opt);

/* sizeof(ba_options) and sizeof(ba_info) of this build, so that a binding can check its
 * copy of the two layouts before passing them. */
size_t ba_struct_size(int which); /* 0: ba_options, 1: ba_info; 0 for anything else */

/* Creates a problem for a fixed observation graph (Section 2.1: cameras x_c, points x_p).
 * cam_idx, pt_idx: device int32 [n_obs], the camera and point of each observation; they
 * are copied (and sorted internally by point, then camera) during the call and not kept.
 * Every (camera, point) pair may appear at most once.  opt may be NULL (defaults).
 * stream: a cudaStream_t (NULL = legacy default stream).  *out receives the problem.
 * Limits: n_obs < 2^31; a camera may be covisible with at most 8192 other cameras. */
ba_status ba_create(int n_cams, int n_pts, int n_obs, const int32_t* cam_idx,
                    const int32_t* pt_idx, const ba_options* opt, void* stream,
                    ba_problem** out);

/* Frees every device and host resource of the problem (NULL is ignored). */
void ba_destroy(ba_problem* prob);

/* Message describing the last non-OK status returned for this problem ("" if none). */
const char* ba_last_error(const ba_problem* prob);

/* Linearises at (cams, pts) (Section 2.1, Eq. 1-2): residuals f_o = pi(cam, X) - obs_o,
 * F_o = df_o/dcam (2x9), E_o = df_o/dX (2x3) for the 9-parameter angle-axis camera,
 * each scaled by w_o under BA_LOSS_HUBER.  cost_out: host double, receives
 * 1/2 sum rho(|f_o|^2) (1/2 sum |f_o|^2 for the squared loss; may be NULL). */
ba_status ba_linearize(ba_problem* prob, const double* cams, const double* pts,
                       const double* obs, double* cost_out);

/* Schur reduction for damping lambda (Section 2.1, Eq. 3-4): D, C_p^-1 (FP64), the
 * gradient g = -J^T f, the reduced right-hand side b = g_c - F^T E C^-1 g_p and the
 * point-block-Jacobi blocks S_cc^-1.  Requires ba_linearize. */
ba_status ba_schur_setup(ba_problem* prob, double lambda);

/* Multigrid setup (Section 3): covisibility, Algorithm 2 aggregation, near-nullspace
 * and per-aggregate QR prolongators (3.1, 3.3), Galerkin coarse operators P^T A P
 * (Section 2.3), Jacobi blocks, Lanczos lambda_max (3.4) and the coarsest direct
 * solver.  Requires ba_schur_setup.  No-op unless preconditioner == BA_PRECOND_MG. */
ba_status ba_mg_setup(ba_problem* prob);

/* PCG on S delta_c = rhs (Section 3.6) from delta_c = 0 with the configured
 * preconditioner.  rhs: device n_cams x 9, or NULL for the reduced RHS b.
 * delta_c: device n_cams x 9 output.  iters, rel_res: host outputs (may be NULL):
 * the number of S products and |r|/|rhs| of the recursive residual. */
ba_status ba_pcg_solve(ba_problem* prob, const double* rhs, double* delta_c, int* iters,
                       double* rel_res);

/* Point step delta_p = C^-1 (g_p - E^T F delta_c) (Section 2.1), n_pts x 3 output. */
ba_status ba_back_substitute(ba_problem* prob, const double* delta_c, double* delta_p);

/* One LM step (Section 2.1; step control of Section 5 read as the gain-ratio rule):
 * linearise at (cams, pts), solve with damping *lambda_inout, evaluate the cost at
 * x + delta, accept if rho > 1e-3 (cams/pts updated in place) and update lambda.
 * accepted, cost_out: host outputs (cost at the returned cams/pts).  A solve that fails
 * (a block not positive definite, a PCG breakdown) rejects the step.  The step is queued
 * on the problem's stream and synchronised with the host once for its decision; it has
 * completed when the call returns. */
ba_status ba_lm_step(ba_problem* prob, double* cams, double* pts, const double* obs,
                     double* lambda_inout, int* accepted, double* cost_out);

/* Adjoint of the last solve: given dL/ddelta (device, 9 n_cams + 3 n_pts: camera
 * part then point part) returns dL/dobs (n_obs x 2, caller order), dL/dcams
 * (n_cams x 9) and dL/dpts (n_pts x 3) at the linearisation point, holding lambda
 * fixed and differentiating through D = lambda diag(J^T J).  Uses a second PCG solve
 * with S and the same multigrid hierarchy.  Requires a completed ba_pcg_solve with
 * rhs = NULL and the squared loss (BA_ERR_INVALID_ARG under BA_LOSS_HUBER).  Any output
 * may be NULL. */
ba_status ba_adjoint(ba_problem* prob, const double* dL_ddelta, double* dL_dobs,
                     double* dL_dcams, double* dL_dpts);

/* ---------------------------------------------------------------------------------
 * Point-partitioned solve (several ranks share one LM step).
 * --------------------------------------------------------------------------------- */

/* Sums `count` doubles of buf (HOST memory) over all ranks of a partitioned solve, in
 * place (an all-reduce), and returns 0 on success.  Called by the library on every rank at
 * the same points of each call, with the same counts. */
typedef int (*ba_allreduce_fn)(double* buf, size_t count, void* user);

/* Makes the problem one rank's part of a point-partitioned solve: the points are split
 * among the ranks, each point with all of its observations on one rank, and every rank
 * solves the same LM step.  This rank's problem was created (ba_create) on its own points
 * (ids 0 .. n_pts - 1) and their observations, with the global camera ids and count.
 * cam_idx_all, pt_idx_all (HOST int32 [n_obs_all]) describe every rank's observations
 * (global point ids, any order); the covisibility of Section 3.2, and with it the whole
 * multigrid hierarchy, is built from them, identically on every rank.  Each rank forms its
 * points' residuals, Jacobian blocks and point blocks C_p, and its share of every
 * camera-space sum: the gradient and reduced right-hand side, diag(J^T J) for the
 * damping, the diagonal blocks S_cc and the off-diagonal blocks of the assembled S, the
 * costs and the model decrease; `allreduce` adds the shares (the exchange step of the
 * point-partitioned Schur complement).  The PCG then runs on every rank on the same
 * assembled S, with no exchange inside the loop, and ba_back_substitute / ba_lm_step
 * produce this rank's points.  Call once, after ba_create and before the first
 * ba_linearize.  Requires precision BA_FP64 and level0_operator BA_OP_EXPLICIT or
 * BA_OP_AUTO (the assembled level 0 is then always used); ba_adjoint, the implicit PCG
 * product and the inspection product ba_schur_matvec are not available on a partitioned
 * problem (BA_ERR_INVALID_ARG), and the preconditioner must be BA_PRECOND_MG.  A hook that
 * returns nonzero makes the call fail with BA_ERR_STATE. */
ba_status ba_set_partition(ba_problem* prob, int n_obs_all, const int32_t* cam_idx_all,
                           const int32_t* pt_idx_all, ba_allreduce_fn allreduce, void* user);

/* ---------------------------------------------------------------------------------
 * Inspection entry points (used by the parity tests; not needed to solve).
 * --------------------------------------------------------------------------------- */

/* y = S x with the implicit operator of Section 3.6 (x, y: device n_cams x 9, FP64).
 * precision BA_MIXED runs the FP32-storage kernel used inside the V-cycle. */
ba_status ba_schur_matvec(ba_problem* prob, const double* x, double* y, int precision);

/* z = M^-1 r for the configured preconditioner (one V-cycle of Algorithm 1 for MG). */
ba_status ba_precond_apply(ba_problem* prob, const double* r, double* z);

typedef struct {
  int n_levels;           /* multigrid levels (0 if no hierarchy) */
  int level_nodes[16];    /* nodes per level */
  int level_block[16];    /* dofs per node per level (9 at level 0, 16 below) */
  int level_nnzb[16];     /* block nonzeros of the level operator (0 for coarsest) */
  double level_lambda_max[16]; /* Lanczos estimate per smoothed level */
  int pcg_iters;          /* last ba_pcg_solve */
  double pcg_rel_res;
  double cost;            /* last ba_linearize */
  double lambda;          /* last ba_schur_setup */
  long long kernel_launches; /* kernels launched by this problem so far */
  int level0_explicit;    /* 1 if the last ba_mg_setup chose the assembled level-0 operator */
} ba_info;

ba_status ba_get_info(ba_problem* prob, ba_info* info);

/* Arrays that ba_get_array can copy out.  Per-observation arrays come out in the
 * caller's observation order, per-point arrays in the caller's point order. */
typedef enum {
  BA_ARR_RESIDUAL = 0,   /* double [n_obs][2] */
  BA_ARR_JAC_F = 1,      /* double [n_obs][2][9] */
  BA_ARR_JAC_E = 2,      /* double [n_obs][2][3] */
  BA_ARR_DAMP_C = 3,     /* double [n_cams][9] */
  BA_ARR_DAMP_P = 4,     /* double [n_pts][3] */
  BA_ARR_CINV = 5,       /* double [n_pts][3][3] */
  BA_ARR_GRAD_C = 6,     /* double [n_cams][9]  g_c = -F^T f */
  BA_ARR_GRAD_P = 7,     /* double [n_pts][3]   g_p = -E^T f */
  BA_ARR_RHS = 8,        /* double [n_cams][9]  reduced RHS b */
  BA_ARR_LEVEL_ROWPTR = 9,  /* int32 [n_l + 1]  BSR row pointers of level l's operator */
  BA_ARR_LEVEL_COLS = 10,   /* int32 [nnzb]     BSR block columns (sorted per row) */
  BA_ARR_LEVEL_VALS = 11,   /* double [nnzb][b][b] operator blocks (level 0 = explicit S) */
  BA_ARR_LEVEL_W = 12,      /* int64 [nnzb]     covisibility counts W on the same pattern */
  BA_ARR_STRENGTH_PTR = 13, /* int32 [n_l + 1]  strength-ordered neighbour lists */
  BA_ARR_STRENGTH_IDX = 14, /* int32 [...] */
  BA_ARR_AGG = 15,          /* int32 [n_l]      aggregate of each node of level l */
  BA_ARR_NULLSPACE = 16,    /* double [n_l][b][16] near-nullspace rows of level l */
  BA_ARR_PROLONG = 17,      /* double [n_l][b][16] Q blocks (P restricted to each node) */
  BA_ARR_KEPT = 18,         /* uint32 [n_{l+1}] bit s set if coarse dof s is kept */
  BA_ARR_JACOBI_INV = 19,   /* double [n_l][b][b] inverse diagonal blocks of level l */
  BA_ARR_COARSE_INV = 20,   /* double [N][N] inverse of the coarsest operator */
  BA_ARR_SCC_INV = 21       /* double [n_cams][9][9] point-block-Jacobi blocks S_cc^-1 */
} ba_array;

/* Kernel classes whose launches can be timed with CUDA events on the problem's stream. */
typedef enum {
  BA_KT_SCHUR_FP64 = 0,  /* implicit Schur product, FP64 storage (outer PCG operator) */
  BA_KT_SCHUR_FP32 = 1,  /* implicit Schur product, FP32 storage (inside the V-cycle) */
  BA_KT_LINEARIZE = 2,   /* residual + Jacobian kernel */
  BA_KT_SCHUR_DF = 3,    /* implicit Schur product in paired FP32 (outer operator, mixed mode) */
  BA_KT_ASSEMBLY = 4,    /* off-diagonal blocks of the assembled level-0 S (observation pairs) */
  BA_KT_OUTER_BSR = 5,   /* PCG product with the FP64 blocks of the assembled S */
  BA_KT_VCYCLE = 6,      /* one whole preconditioner application (all of a V-cycle's kernels) */
  BA_KT_SCHUR_RECOMPUTE = 7, /* implicit Schur product, FP64, blocks rebuilt (recompute_jacobian) */
  BA_KT_COUNT = 8
} ba_kernel_class;

/* enable != 0 starts recording a CUDA event pair around every launch of the timed
 * classes (and clears earlier records); 0 stops recording. */
ba_status ba_set_kernel_timing(ba_problem* prob, int enable);

/* Sum of the recorded launch durations (ms, host) and the launch count (host) of one
 * kernel class since timing was enabled.  Synchronises the stream. */
ba_status ba_get_kernel_timing(ba_problem* prob, int kernel_class, double* total_ms,
                               long long* launches);

/* Copies internal array `which` (of multigrid level `level` where relevant) into dst
 * (device memory, capacity `bytes`).  *needed (host, may be NULL) receives the size;
 * with dst == NULL only the size is returned. */
ba_status ba_get_array(ba_problem* prob, int which, int level, void* dst, size_t bytes,
                       size_t* needed);

/* ---------------------------------------------------------------------------------
 * Allocation-free objective evaluation.
 * --------------------------------------------------------------------------------- */

/* Largest camera count ba_cost_noalloc accepts (its fixed scratch holds 12 doubles per
 * camera plus 1,024 partial sums: about 0.4 MB per GPU). */
#define BA_NOALLOC_MAX_CAMS 4096

/* Evaluates the LM objective 1/2 sum_o |pi(cam_c, X_p) - obs_o|^2 for caller-supplied
 * cameras, points and observations without allocating any device memory, and without a
 * ba_problem.  The paper has no counterpart: this entry point exists for callers that
 * must not allocate GPU memory themselves, such as code whose device memory is owned by a
 * framework or pool allocator with a fixed budget, or a step loop that must keep a fixed
 * footprint and cannot risk cudaMalloc's implicit device synchronisation or an
 * out-of-memory failure in the middle of a run.  ba_create and the solve entry points do
 * allocate; this one does not.
 *
 * cams [n_cams x 9], pts [n_pts x 3], obs [n_obs x 2]: device float64; cam_idx, pt_idx:
 * device int32 [n_obs]; cost_out: device pointer to one double, written on `stream`
 * (a cudaStream_t; the call returns without synchronising).  An observation with an
 * out-of-range index makes *cost_out NaN.
 *
 * Scratch lives in a fixed array inside the library that every GPU loading the library
 * keeps until the process exits.  The first call on a device looks up that array's
 * device address (with the device current), so make that first call before any stream
 * capture.  With CUDA's default lazy module loading, that first call is also when the
 * driver loads the array onto the device: it allocates the array's memory then, may
 * synchronise, and can fail there for lack of memory.  So make the first call at
 * start-up, before the memory budget is in force.  The looked-up address belongs to the
 * device's primary context and does not survive cudaDeviceReset: do not call this entry
 * point again in a process after resetting the device.  All calls share the array and it keeps the last call's contents; the call
 * clears the parts that must start at zero.  Calls whose GPU work overlaps (on different
 * streams without ordering) race on the array and give wrong results.
 * Returns BA_ERR_LIMIT if n_cams > BA_NOALLOC_MAX_CAMS, BA_ERR_INVALID_ARG for bad
 * sizes or null arrays, BA_ERR_CUDA if a launch fails. */
ba_status ba_cost_noalloc(int n_cams, int n_pts, int n_obs, const double* cams, const double* pts,
                          const double* obs, const int32_t* cam_idx, const int32_t* pt_idx,
                          double* cost_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BA_H_ */
