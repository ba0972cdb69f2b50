/*
 * ba.h - C ABI of the GB300 bundle-adjustment normal-equation solver.
 *
 * The library solves the reduced camera system of one Levenberg-Marquardt
 * (LM) iteration of bundle adjustment,
 *
 *     S dx_p = -b~,   S = U_lambda - W V_lambda^{-1} W^T,   b~ = b_p - W V_lambda^{-1} b_l
 *
 * (Weber, Demmel, Cremers, "Multidirectional Conjugate Gradients for Scalable
 * Bundle Adjustment", GCPR 2021: Section 3.1, Eqs. 6-14), by block-Jacobi
 * preconditioned conjugate gradients (Algorithm 1) or by multidirectional
 * conjugate gradients (Algorithm 2, Section 3.2), on one CUDA device.
 *
 * Conventions for every call:
 *  - Return value: BA_OK (0) or a negative ba_status.  No C++ exception
 *    crosses this boundary.  After a failure ba_last_error() describes it.
 *  - A ba_problem handle is not thread-safe; distinct handles are
 *    independent.  All device work of a handle is ordered on its stream
 *    (ba_set_stream); calls return after that work has finished unless
 *    stated otherwise.
 *  - Pointer arguments marked "host or device" may point to host memory
 *    (pageable or pinned) or to device memory of the handle's device: the
 *    library copies with cudaMemcpyDefault.  The caller keeps ownership of
 *    every buffer it passes; the library keeps its own copies.
 *  - Arrays are dense, row-major, float64 unless stated.
 *
 * Camera model (BAL, d_p = 9): a camera row is (omega[3], t[3], f, k1, k2),
 * omega an angle-axis rotation; a landmark X projects to
 *     P = R(omega) X + t,  p = -(P_x, P_y) / P_z,
 *     pi = f (1 + k1 |p|^2 + k2 |p|^4) p,
 * and the residual of an observation with measurement m is pi - m (Eq. 1).
 * The paper estimates these 9 parameters per pose but does not print the
 * formula; this is the model of the BAL datasets it uses.
 */
#ifndef BA_H_
#define BA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ba_status {
    BA_OK = 0,
    BA_ERR_INVALID_ARG = -1,   /* bad size, index, pointer or option */
    BA_ERR_OOM = -2,           /* device or host allocation failed */
    BA_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    BA_ERR_SINGULAR = -4,      /* a damped 3x3 V_lambda or a 9x9 block of S is not positive definite */
    BA_ERR_BREAKDOWN = -5,     /* NaN/Inf or a non-positive curvature in the Krylov solve */
    BA_ERR_NOT_CONVERGED = -6, /* max_iters reached; the iterate is still returned */
    BA_ERR_TIMEOUT = -7,       /* a bounded device-side wait gave up (see ba_options.wait_polls) */
    BA_ERR_STATE = -8          /* call out of order, e.g. a solve before ba_build_normal */
} ba_status;

typedef enum ba_damping {
    BA_DAMPING_MARQUARDT = 0,  /* D^T D = diag(J^T J), entries clamped to [1e-6, 1e32] */
    BA_DAMPING_IDENTITY = 1    /* D = I */
} ba_damping;

typedef enum ba_precision {
    BA_PRECISION_FP64 = 0,     /* every array and product in float64 */
    BA_PRECISION_MIXED = 1     /* float32 S, directions and Krylov products; float64 outer
                                  refinement on the true residual, small solves in float64;
                                  residuals, Jacobians, landmark factors, b~ and the true
                                  residual in double-float (float32 pairs, ~48 bits) */
} ba_precision;

typedef enum ba_solver {
    BA_SOLVER_PCG = 0,
    BA_SOLVER_MCG = 1
} ba_solver;

/* Options fixed at ba_problem_create. */
typedef struct ba_options {
    int32_t damping;           /* ba_damping; the paper's D_p, D_l of Eq. 5 are unspecified */
    int32_t precision;         /* ba_precision */
    int32_t chunk_iters;       /* Krylov iterations per pass of the solve graph's device-side loop
                                  between checks of the stop flags (default 8, 1..256); a solve is
                                  one graph launch and the host waits once, at its end */
    int32_t max_history;       /* MCG: maximum stored direction columns (default 0 = max_iters * n_dirs + 1);
                                  when it is full FP64 stops with OOM, while MIXED ends the float32
                                  sweep and the refinement starts another from the true residual */
    double inner_tol;          /* MIXED: relative residual reduction aimed at by one float32 sweep
                                  (default 1e-6: one sweep when float32 reaches the tolerance) */
    int32_t max_refine;        /* MIXED: maximum outer refinement sweeps (default 64) */
    int32_t item_blocks;       /* stored 9x9 blocks of S per work item of the block-sparse products
                                  (longer rows are split): 0 (default) = 512, else a multiple of 32
                                  in [32, 4096]; ba_autotune sets it */
    int32_t wait_polls;        /* bounded device waits: polls of a tile copy's barrier before the
                                  solve gives up with BA_ERR_TIMEOUT (the kernel then waits for its
                                  own copies still in flight, with the default bound, and returns).
                                  0 (default) = 2^20; 1 .. 2^30; -1 = no poll at all, so every such
                                  wait gives up at once (tests the timeout path) */
    int32_t spmv_config;       /* warps x copy stages per CTA of the tile-streaming one-column product:
                                  0 (default) = float32 16 x 1, float64 4 x 2; 1 = 8 x 2 / 8 x 1;
                                  2 = 10 x 2 / 2 x 4; ba_autotune sets it */
    int32_t host_loop;         /* 1: drive the iteration and refinement loops from the host (a plain
                                  graph of chunk_iters iterations per launch, the stop flags read back
                                  after each) instead of the solve graph's device-side loops; the same
                                  kernels run.  For profilers that cannot see kernels inside graphs
                                  with conditional nodes.  Default 0. */
    int32_t reserved[3];
} ba_options;

/* Filled by ba_solve_pcg / ba_solve_mcg. */
typedef struct ba_solve_stats {
    int32_t status;            /* same as the call's return value */
    int32_t iters;             /* Krylov steps taken (summed over refinement sweeps) */
    int32_t local_steps;       /* MCG steps whose tau-test chose the local directions */
    int32_t n_dirs_eff;        /* MCG: non-empty pose subsets actually used */
    int32_t refinements;       /* MIXED: outer sweeps; 1 for FP64 */
    int32_t history_cols;      /* MCG: direction columns stored at exit */
    int32_t pinv_steps;        /* MCG: steps whose Delta_i needed the eigen-decomposition pseudo-inverse
                                  (a rank-deficient or badly conditioned direction block) */
    int32_t host_waits;        /* times the host waited for the device during the solve (1: only for
                                  the results at its end; the iteration loop runs on the device) */
    double rel_residual;       /* recursive |r_i| / |r_0| at exit (of the last sweep for MIXED) */
    double true_rel_residual;  /* |-b~ - S x| / |b~| recomputed in float64 at exit */
    double ms;                 /* device time of the solve, CUDA events on the handle's stream
                                  (from the upload of its arguments to the copy-back of its results) */
} ba_solve_stats;

/* Filled by ba_lm_step. */
typedef struct ba_lm_stats {
    int32_t status;
    int32_t accepted;          /* 1 if F(x + dx) < F(x) and x was updated */
    int32_t converged;         /* 1 if the relative decrease of F fell below 1e-6 (Section 4.1) */
    int32_t solver_iters;
    double cost_before;        /* F(x) (Eq. 1) at entry */
    double cost_after;         /* F(x + dx) of the trial step */
    double lambda_used;
    double lambda_next;
    double ms;                 /* the whole step: cost, build, solve, back-substitution, trial cost */
    double solve_ms;           /* the solve alone (Algorithm 1 or 2), as ba_solve_stats.ms */
} ba_lm_stats;

typedef struct ba_problem ba_problem;

/* Fill *opt with the defaults listed in ba_options. */
void ba_default_options(ba_options* opt);

/*
 * Create a problem from cameras, landmarks and observations (Section 3:
 * n_p poses with d_p = 9, n_l landmarks, one 2-D residual per observation).
 *   opt        options, or NULL for the defaults
 *   cams       n_cams x 9, host or device
 *   pts        n_pts x 3, host or device
 *   obs_cam    n_obs camera indices in [0, n_cams), host or device, int32
 *   obs_pt     n_obs landmark indices in [0, n_pts), host or device, int32
 *   obs_xy     n_obs x 2 measured pixel positions m, host or device
 *   out        receives the handle
 * Observations may come in any order.  A landmark may have a single
 * observation (V_lambda stays definite through the damping).  Errors:
 * INVALID_ARG for non-positive sizes, n_obs >= 2^31, or an index out of
 * range; OOM; CUDA.  Uses the current CUDA device and the legacy default
 * stream until ba_set_stream.
 */
int ba_problem_create(const ba_options* opt, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                      const double* cams, const double* pts, const int32_t* obs_cam,
                      const int32_t* obs_pt, const double* obs_xy, ba_problem** out);

/*
 * Create one handle over n_problems independent problems (a batch).  Problem b owns the cameras
 * [cam_off[b], cam_off[b + 1]) (cam_off: n_problems + 1 int32, host or device, strictly increasing,
 * cam_off[0] = 0, cam_off[n_problems] = n_cams); every landmark must be observed only by cameras of
 * one problem, so S is block-diagonal over the problems.  The other arguments are those of
 * ba_problem_create over the concatenated arrays.  ba_build_normal builds every problem (one
 * lambda), and ba_solve_pcg / ba_solve_mcg solve every problem in the same kernel launches, each
 * problem with its own step sizes, tau-test, direction history and stop test (Algorithms 1 and 2
 * run independently per problem; the paper solves one problem at a time).  MCG's pose subsets are
 * formed per problem.  Their stats summarise the batch (the first failing problem's status, the
 * largest iteration counts and residuals); ba_get_batch_stats gives each problem's.  A problem's
 * result does not depend on the others in the batch.  ba_lm_step takes single-problem handles only.
 * Errors: those of ba_problem_create; INVALID_ARG also for n_problems outside [1, 65535], a bad
 * cam_off, or a landmark shared by two problems.
 */
int ba_batch_create(const ba_options* opt, int32_t n_problems, const int32_t* cam_off, int32_t n_cams,
                    int32_t n_pts, int64_t n_obs, const double* cams, const double* pts,
                    const int32_t* obs_cam, const int32_t* obs_pt, const double* obs_xy, ba_problem** out);

/* Free every device and host allocation of the handle.  NULL is ignored. */
void ba_problem_destroy(ba_problem* p);

/* Text of the last error of this handle ("" if none).  NULL handle: the last
 * error of a failed ba_problem_create on this thread. */
const char* ba_last_error(const ba_problem* p);

/* Order all later work of the handle on `stream` (a cudaStream_t; NULL = legacy default). */
int ba_set_stream(ba_problem* p, void* stream);

/* Replace the current parameters x = (x_p, x_l) (cams n_cams x 9, pts n_pts x 3; host or
 * device).  Either pointer may be NULL to keep that part. */
int ba_set_params(ba_problem* p, const double* cams, const double* pts);

/* Copy the current parameters out (host or device; NULL skips a part). */
int ba_get_params(const ba_problem* p, double* cams, double* pts);

/*
 * Linearise at the current parameters and build the reduced camera system for
 * damping lambda > 0 (Eqs. 2-14): residuals and Jacobians per observation, U_lambda,
 * V_lambda (Marquardt or identity damping), b_p, b_l, the block-sparse S with its
 * 9x9 blocks for every co-visible camera pair, b~, and the inverses of the diagonal
 * blocks of S for the block-Jacobi preconditioner (Section 3.2).  In MIXED precision
 * S itself is built in float32 as Lam S Lam (Lam = diag(S)^-1/2, full pattern and upper
 * triangle) from float32 Jacobians, the diagonal blocks of S in float64, and the
 * residuals, Jacobians, landmark factors and b~ in double-float arithmetic; the
 * preconditioner holds the inverses of the scaled diagonal blocks.  Errors:
 * INVALID_ARG (lambda <= 0 or not finite), SINGULAR (a V_lambda or S_jj not positive
 * definite; the system is left unusable), CUDA.
 */
int ba_build_normal(ba_problem* p, double lambda);

/*
 * Solve S dx_p = -b~ by Algorithm 1 (block-Jacobi PCG) from x_0 = 0, stopping when the
 * recursive residual satisfies |r_{i+1}| < tol |r_0| (the paper's eps, 1e-6 in Section 4.1)
 * or after max_iters steps (1000 in the paper).  MIXED precision runs float32 PCG sweeps
 * inside a float64 iterative refinement that stops on the true residual.  The result stays
 * on the device (ba_get_delta).  Returns OK, NOT_CONVERGED (result still valid), BREAKDOWN,
 * STATE (no ba_build_normal yet), INVALID_ARG, CUDA.  st may be NULL.
 */
int ba_solve_pcg(ba_problem* p, double tol, int32_t max_iters, ba_solve_stats* st);

/*
 * Solve S dx_p = -b~ by Algorithm 2 (MCG): the poses are split into n_dirs subsets of
 * ceil(n_cams / n_dirs) consecutive poses (the last holds the remainder); after each
 * step the tau-test t_i = gamma_i^T alpha_i / (r_{i+1}^T D(S)^{-1} r_{i+1}) < tau selects
 * one search direction per subset, otherwise one global direction; the small systems
 * use a float64 pseudo-inverse and every new block is reorthogonalised against all
 * previous ones (Section 3.2, Eq. 18).  n_dirs = 1 or tau = 0 reduce to PCG plus
 * reorthogonalisation.  Stop test and returns as ba_solve_pcg; also OOM when the
 * direction history exceeds max_history columns.
 */
int ba_solve_mcg(ba_problem* p, double tol, int32_t max_iters, int32_t n_dirs, double tau,
                 ba_solve_stats* st);

/*
 * Copy the last solution out: dxp (n_cams x 9) and, if dxl != NULL, the landmark
 * update dx_l = -V_lambda^{-1} (b_l + W^T dx_p) (n_pts x 3).  The paper prints
 * -V^{-1}(-b_l + W^T dx_p) in Eq. 15; the sign used here follows from the second
 * block row of Eq. 6.  Host or device pointers.  STATE if nothing was solved.
 */
int ba_get_delta(ba_problem* p, double* dxp, double* dxl);

/*
 * One LM iteration (Section 4.1): build at the current lambda (the first call uses
 * lambda0), solve with `solver` (BA_SOLVER_PCG, or BA_SOLVER_MCG with n_dirs, tau),
 * back-substitute, evaluate F(x + dx) (Eq. 1), accept when it decreases
 * (lambda <- max(lambda / 10, 1e-12)) or reject (lambda <- min(10 lambda, 1e16)).
 * The paper does not state its lambda update; this is the rule used.  st->converged
 * reports a relative decrease below ftol.  st may be NULL.
 */
int ba_lm_step(ba_problem* p, int32_t solver, double lambda0, double tol, int32_t max_iters,
               int32_t n_dirs, double tau, double ftol, ba_lm_stats* st);

/* F(x) = sum_i |r_i(x)|^2 at the current parameters (Eq. 1). */
int ba_cost(ba_problem* p, double* cost);

/* ---- standalone camera model and inspection of the built system ---------------------- */

/*
 * pi(c_j, X_l) for n_obs observations (the camera model above), device pointers only:
 * cams n_cams x 9, pts n_pts x 3, obs_cam/obs_pt int32 n_obs, out_xy n_obs x 2.
 * Indices are not checked.  Enqueued on `stream` (cudaStream_t, NULL = legacy default);
 * returns after enqueueing.
 */
int ba_project(int32_t n_cams, int32_t n_pts, int64_t n_obs, const double* cams, const double* pts,
               const int32_t* obs_cam, const int32_t* obs_pt, double* out_xy, void* stream);

/* Residuals r (n_obs x 2), J_p (n_obs x 2 x 9), J_l (n_obs x 2 x 3) of the last build,
 * in the caller's observation order (Eqs. 2-4).  Host or device; NULL skips. */
int ba_get_linearization(const ba_problem* p, double* r, double* Jp, double* Jl);

/* U_lambda (n_cams x 9 x 9), V_lambda (n_pts x 3 x 3), b_p (n_cams x 9), b_l (n_pts x 3)
 * of the last build (Eqs. 8-11).  Host or device; NULL skips. */
int ba_get_normal(const ba_problem* p, double* U, double* V, double* b_p, double* b_l);

/* Number of nonzero 9x9 blocks of S (both triangles and the diagonal). */
int ba_get_schur_nnzb(const ba_problem* p, int64_t* nnzb);

/* S in block-CSR form: row_ptr (n_cams + 1, int64), col (nnzb, int32, ascending within a
 * row), blocks (nnzb x 9 x 9, row-major), and b~ (n_cams x 9) (Eqs. 13-14).  Host or
 * device; NULL skips. */
int ba_get_schur(const ba_problem* p, int64_t* row_ptr, int32_t* col, double* blocks, double* btilde);

/* The inverse diagonal blocks D(S)^{-1} (n_cams x 9 x 9) used by the preconditioner. */
int ba_get_preconditioner(const ba_problem* p, double* Dinv);

/* Recursive relative residuals |r_{i+1}| / |r_0| of the last solve, one per step; at most
 * `cap` values are written to `hist` (host or device) and the count to *n.  MIXED: the inner
 * sweeps' values in units of |b~|.  Batches: those of problem 0 (see ba_get_batch_history). */
int ba_get_residual_history(const ba_problem* p, double* hist, int32_t cap, int32_t* n);

/* Number of problems of the handle (1 unless made by ba_batch_create). */
int ba_get_batch_size(const ba_problem* p, int32_t* n_problems);

/* Per-problem results of the last solve: stats[b] for b < n (n must equal the batch size; ms is
 * the whole batch's).  STATE if nothing was solved. */
int ba_get_batch_stats(const ba_problem* p, ba_solve_stats* stats, int32_t n);

/* ba_get_residual_history for problem `problem` of the batch. */
int ba_get_batch_history(const ba_problem* p, int32_t problem, double* hist, int32_t cap, int32_t* n);

/* ---- measurement ------------------------------------------------------------------------ */

/* Cumulative number of kernel executions this handle has issued on the device (kernels run
 * from a replayed CUDA graph count one each). */
int ba_get_launch_count(const ba_problem* p, int64_t* n);

typedef enum ba_kernel {
    BA_KERNEL_SPMV = 0,        /* q = S p of Algorithm 1, at the handle's precision */
    BA_KERNEL_SCHUR = 1,       /* the S_jk = delta U_j - sum G G^T block build (Eq. 13); mixed precision:
                                  the float32 diagonal blocks and G rows, the preconditioner and the
                                  scaled off-diagonal blocks */
    BA_KERNEL_LINEARIZE = 2,   /* residuals and Jacobians of every observation (Eqs. 2-4) */
    /* the build's kernels one by one (Eqs. 8-14), each recomputing what the last build wrote: */
    BA_KERNEL_LANDMARKS = 3,   /* per landmark: V_lambda, its Cholesky factor and b_l */
    BA_KERNEL_CAM_RHS = 4,     /* per camera: b~ (Eq. 14) and the damping; FP64 also U_lambda, b_p and
                                  the observations' G = W L^-T */
    BA_KERNEL_SCHUR_DIAG = 5,  /* the diagonal blocks S_jj; mixed precision also the float32 G rows */
    BA_KERNEL_SCHUR_OFF = 6,   /* the off-diagonal blocks S_jk, j != k, and the diagonal put in place */
    BA_KERNEL_BLOCK_JACOBI = 7 /* the preconditioner's inverse blocks (mixed precision: of the scaled S) */
} ba_kernel;

/*
 * Mean duration in milliseconds of one launch of `kernel` (ba_kernel), from CUDA events recorded
 * on the handle's stream around each of `reps` launches; a 256 MiB buffer is written between
 * launches so that no launch starts with its operands in L2.  Needs ba_build_normal; every
 * kernel here recomputes the same values, so the built system is unchanged.  STATE before a
 * build, INVALID_ARG for an unknown kernel or reps < 1.
 */
int ba_time_kernel(ba_problem* p, int32_t kernel, int32_t reps, double* ms);

/*
 * Choose the shape of the block-sparse products by measurement: the PCG product q = S p (Algorithm 1)
 * over every problem is timed for each warps x stages shape (spmv_config 0, 1, 2) and each work-item
 * size of 32, 64, 128, 256, 512 and 1024 blocks (`reps` launches each, L2 flushed before each), and
 * the fastest pair is stored in the handle's spmv_config and item_blocks options for later solves.
 * The choice is kept for the process, keyed by the precision and the size of the problem (cameras,
 * stored blocks, problems): a handle of the same key takes it without timing (*ms then holds the
 * time measured when it was chosen).  Needs ba_build_normal.  *item_blocks, *spmv_config and *ms
 * (each may be NULL) receive the choice and its mean time.  The paper has no counterpart (its products
 * run on the CPU).  STATE before a build, INVALID_ARG for reps < 1.
 */
int ba_autotune(ba_problem* p, int32_t reps, int32_t* item_blocks, int32_t* spmv_config, double* ms);

/* ---- learned pose grouping for MCG ------------------------------------------------------
 *
 * Algorithm 2 splits the poses into N subsets of consecutive poses (Section 3.2; the paper
 * notes that the best decomposition is not obvious).  A small message-passing network over the
 * camera co-visibility graph of S scores every camera; sorting the cameras by score gives a camera
 * order whose consecutive runs are the subsets (create the problem with its cameras in that order;
 * any order is valid for MCG).  The paper has no learned component: the network is this library's.
 *
 *   graph      c_jk = |Lam_j S_jk Lam_k|_F for each stored block j != k (Lam = diag(S)^-1/2),
 *              d_j = sum_k c_jk
 *   features   8 per camera: its centre -R^T t standardised per axis, its viewing axis (third row
 *              of R), log(1 + d_j) standardised, and 1
 *   layers     3 x  H' = relu(H Ws + (D^-1 C H) Wn + b), widths 8 -> 64 -> 64 -> 64
 *   read-out   s = H wo + bo
 *   loss       L = u^T (D - C) u / u^T D u with u = s - (d^T s / sum d): the Rayleigh quotient of
 *              the coupling Laplacian, small when strongly coupled cameras get close scores
 *   training   Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on dL/dtheta
 * Parameters (float32, in this order): for each layer Ws (in x 64, row-major), Wn (in x 64),
 * b (64); then wo (64), bo (1); ba_gnn_param_count gives the total.  The network is trained in
 * float32; inference may round weights and activations to bfloat16 (float32 accumulation).
 * Every call that takes a ba_problem needs ba_build_normal, a single-problem handle and at most
 * 65536 cameras (INVALID_ARG / STATE otherwise), and runs on the problem's stream.
 */
typedef struct ba_gnn ba_gnn;

/* A network with zero parameters (set them with ba_gnn_set_params).  OOM, CUDA. */
int ba_gnn_create(ba_gnn** out);
void ba_gnn_destroy(ba_gnn* g);
const char* ba_gnn_last_error(const ba_gnn* g);
int ba_gnn_param_count(int64_t* n);
/* Copy all parameters in (host or device, float32) and reset the Adam state. */
int ba_gnn_set_params(ba_gnn* g, const float* params);
int ba_gnn_get_params(const ba_gnn* g, float* params);
/* The graph of p's built system: features (n_cams x 8) and coupling weights c (nnzb, in the
 * block order of ba_get_schur, 0 on the diagonal); host or device; NULL skips. */
int ba_gnn_graph(ba_gnn* g, ba_problem* p, float* features, float* coupling);
/* Forward pass on p's built system: *loss (may be NULL), scores (n_cams, may be NULL) and, when
 * grad != NULL, the backward pass: dL/dtheta (param_count floats).  Host or device pointers. */
int ba_gnn_loss(ba_gnn* g, ba_problem* p, double* loss, float* scores, float* grad);
/* One training step on p's built system: forward, backward and an Adam update with learning rate
 * lr; *loss receives the loss before the update. */
int ba_gnn_train_step(ba_gnn* g, ba_problem* p, double lr, double* loss);
/* The grouping order: order[r] = the camera of rank r by score (ties by index), host or device,
 * n_cams int32; bf16 != 0 runs the forward pass with bfloat16 weights and activations; *loss (may
 * be NULL) receives the loss of the scores. */
int ba_gnn_order(ba_gnn* g, ba_problem* p, int32_t bf16, int32_t* order, double* loss);
/* Kernel executions issued by this network so far. */
int ba_gnn_launch_count(const ba_gnn* g, int64_t* n);

/* ---- allocation-free residual check ---------------------------------------------------- */

/* Largest n_cams accepted by ba_schur_residual_static. */
#define BA_STATIC_MAX_CAMS 65536

/*
 * |-b~ - S x| and |b~| for a block-sparse S that the caller holds in device memory, computed
 * without allocating anything.  The paper has no counterpart; this exists for callers that
 * cannot call cudaMalloc where they check a solution: loops whose device memory is fixed up
 * front, or hosts whose allocator owns all device memory.
 *   n_cams   block rows of S, 1 .. BA_STATIC_MAX_CAMS (larger: INVALID_ARG, nothing launched)
 *   row_ptr  n_cams + 1 int64 block offsets, device
 *   col      block column indices (int32), device
 *   blocks   9x9 row-major blocks, device (the layout ba_get_schur returns)
 *   btilde   9 n_cams, device;  x   9 n_cams, device
 *   out      2 doubles, device: out[0] = |-b~ - S x|_2, out[1] = |b~|_2
 *   stream   cudaStream_t (NULL = legacy default); the call returns after enqueueing
 * Working memory is one file-scope device array of 2 * BA_STATIC_MAX_CAMS doubles (1 MiB) that
 * every GPU loading the library holds until the process exits; each call overwrites every
 * entry it reads, so nothing has to be cleared between calls.  All calls share that array:
 * calls that overlap on the GPU (different streams, or different host threads) race and give
 * wrong results, so order them.  A call made outside a stream capture looks up the array's
 * device address on the current device (cudaGetSymbolAddress, not a stream operation), so the
 * address stays right after cudaDeviceReset; a call whose stream is capturing uses the address
 * found by the last call outside capture on that device.  Make the first call on a device before
 * any stream capture (otherwise STATE).  No cudaMalloc, cudaFree or other allocating call is
 * made.  The library cannot check the lengths or the device of the arrays (it gets pointers
 * only): the caller keeps them as stated above.  Errors: INVALID_ARG, STATE, CUDA; the text is
 * available from ba_last_error(NULL) on the calling thread.
 */
int ba_schur_residual_static(int32_t n_cams, const int64_t* row_ptr, const int32_t* col,
                             const double* blocks, const double* btilde, const double* x,
                             double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BA_H_ */
