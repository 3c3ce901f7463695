/*
 * rpt.h -- C ABI of librpt: robust proton treatment planning by ADMM with a
 * Barzilai-Borwein dual step (ADMM-BB), on one GPU (sm_103a).
 *
 * Problem (Sec. 2.1, Eqs. 1-2; scenario probabilities as in Sec. 2.1):
 *     minimise  f(x) = sum_s c_s sum_i w_i (a_{s,i}^T x - p_i)^2
 *     subject to lb <= x <= ub
 * A_s (m x n, one per uncertainty scenario s = 1..N) are dose-influence
 * matrices with rows = voxels and columns = proton spots; w = voxel weights,
 * p = prescription, c_s = scenario weights.  The paper's case is lb = 0,
 * ub = +inf.
 *
 * Conventions for every entry point:
 *  - The return value is a status code (RPT_OK = 0, > 0 warning, < 0 error).
 *    On an error no output array is written.  No call aborts the process.
 *    rpt_last_error() gives a thread-local message for the last failure.
 *  - Array arguments are HOST pointers unless the name ends in "_dev".
 *    Host input arrays are only read during the call; the library copies what
 *    it keeps.  Output arrays are caller-allocated and written on success.
 *  - Dense vectors are float64.  "[N*n]" means scenario-major: element j of
 *    scenario s is at s*n + j.
 *  - A plan owns its device memory and one CUDA stream (the caller's stream if
 *    given in rpt_device_opts).  Calls on one plan must not overlap; different
 *    plans may be used from different threads.
 *  - All device-side loops are bounded (max_iter, cg_max, max_trials);
 *    the library has no unbounded device wait.
 */
#ifndef RPT_H
#define RPT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define RPT_OK              0
#define RPT_NOT_CONVERGED   1   /* iteration cap reached; the last iterate is returned */
#define RPT_EINVAL        (-1)  /* bad argument: sizes, CSR structure, NaN/Inf, lb > ub */
#define RPT_ENOMEM        (-2)  /* device or host allocation failed */
#define RPT_ECUDA         (-3)  /* a CUDA runtime call failed (message in rpt_last_error) */
#define RPT_TIMEOUT       (-4)  /* a bounded device-side wait ran out */
#define RPT_DIVERGED      (-5)  /* a residual or objective became non-finite */
#define RPT_EUNSUPPORTED  (-6)  /* valid request outside this build's limits (e.g. n too large) */

/* ---- value formats of the stored dose-influence matrix ------------------- */
#define RPT_F32      0   /* float32 as given */
#define RPT_BF16     1   /* bfloat16 with one float32 scale per spot column */
#define RPT_FP8E4M3  2   /* float8 e4m3 with one float32 scale per spot column */

/* ---- ADMM variants (readings of Sec. 2.2, see rpt_admm_params) ----------- */
#define RPT_BB_PAPER    0   /* Eq. 8: BB value if > 0 (and finite), else rho */
#define RPT_BB_GUARDED  1   /* Eq. 8 clamped to [rho/bb_kappa, bb_kappa*rho] */
#define RPT_BB_OFF      2   /* always rho: textbook consensus ADMM */
#define RPT_Z_STD       0   /* z = P(mean_s(x_s + y_s/rho)): exact z-minimiser */
#define RPT_Z_LIT       1   /* z = P(mean_s x_s): the update as printed in Sec. 2.2 */

/* Largest spot count this build supports (the spot vector and its accumulator
 * are staged in shared memory of one CTA). */
#define RPT_MAX_SPOTS 24576

typedef struct rpt_plan rpt_plan;   /* opaque; created and owned by the library */

/* The problem, as host arrays (Sec. 2.1).  All pointers are read-only and only
 * read during rpt_plan_create. */
typedef struct {
  int32_t m;                        /* voxels (rows), >= 1 */
  int32_t n;                        /* spots (columns), 1..RPT_MAX_SPOTS */
  int32_t N;                        /* scenarios, >= 1 */
  const int32_t* const* row_ptr;    /* N arrays of m+1: row_ptr[s][0] = 0, non-decreasing */
  const int32_t* const* col_idx;    /* N arrays of nnz_s = row_ptr[s][m]: in [0,n), strictly increasing within a row */
  const float*   const* val;        /* N arrays of nnz_s: finite and >= 0 (dose influence) */
  const double* voxel_w;            /* [m] voxel weights w_i, finite and >= 0 (Eq. 1) */
  const double* presc;              /* [m] prescription p_i, finite and >= 0 (Eq. 1) */
  const double* scen_weight;        /* [N] scenario weights c_s in [0,1], or NULL for all 1 */
  const double* lb;                 /* [n] lower bounds, or NULL for 0 (Eq. 2: x >= 0) */
  const double* ub;                 /* [n] upper bounds, or NULL for +inf; lb <= ub */
  int32_t value_format;             /* RPT_F32 | RPT_BF16 | RPT_FP8E4M3 */
  int32_t index_width;              /* 32, or 16 (column indices stored as uint16; needs n <= 65535) */
} rpt_problem;

typedef struct {
  int32_t device;                   /* CUDA device ordinal */
  void*   stream;                   /* cudaStream_t to run on, or NULL for a stream owned by the plan */
  int32_t ctas_per_sm;              /* row-pass CTAs per SM (0 = library choice) */
  int32_t row_path;                 /* row-pass layout and kernel:
                                       1 register-direct loads of CSR rows;
                                       2 bulk-copy (TMA) ring over CSR rows;
                                       3 streaming (warps claim chunks, entries go straight to registers);
                                       4 bundled ring: rows grouped 4 at a time in the given row order, one
                                         spot index per column of a group (rows that are neighbours in the
                                         input order should share spots, as voxels in grid order do); see
                                         accumulate for its exact (bitwise reproducible) sums;
                                       0: 4 when its shared-memory stage fits the plan, else 2, else 1 */
  int32_t autotune;                 /* 1: time every ring configuration that fits this plan (entries and
                                       rows per stage, stages) on its own row pass and keep the fastest;
                                       0: the first that fits */
  int32_t chunk_entries;            /* ring geometry (paths 2-4): entries (path 4: block columns) per stage;
                                       0 = library choice.  With chunk_rows and stages it replaces the
                                       candidate list (and the autotuner) */
  int32_t chunk_rows;               /* rows (path 4: bundles) per stage; 0 = library choice */
  int32_t stages;                   /* ring stages (2..8, paths 2 and 4); 0 = library choice */
  int32_t min_lanes;                /* smallest lanes-per-row group of paths 1 and 2 (1..32, rounded down to a
                                       power of two); 0 = 8 */
  int32_t inject_timeout;           /* testing hook: 1 makes the ring's producer (paths 2 and 4) issue no
                                       copy, so every consumer wait runs out after its one-second bound and
                                       the call returns RPT_TIMEOUT (no GPU fault is involved); 0 normally */
  int64_t device_mem_cap;           /* testing hook: bytes the plan may allocate on the device (a request past
                                       it fails as an out-of-memory would, RPT_ENOMEM); 0 = no cap */
  int32_t accumulate;               /* row path 4's scatter: 0 = library choice (2); 1 = exact 64-bit fixed-point
                                       sums: every pass, and so every solve, is bitwise reproducible whatever
                                       the scheduling, and tight tolerances (1e-7) converge where float
                                       rounding noise can stall them; about 40 % slower per pass;
                                       2 = float32 shared-memory atomics, whose results vary in the last bits
                                       from run to run */
  int32_t ring_threads;             /* row path 4: threads of a row-pass CTA, 1024 (31 consumer warps, 6 block
                                       columns per lane held in registers), 768 (23 warps, 8) or 640 (19 warps,
                                       10); fewer warps hide less latency, more registers re-read fewer block
                                       columns of wide bundles.  0 = library choice (1024, or the autotuner's
                                       pick among the three) */
} rpt_device_opts;

/* ADMM-BB parameters (Sec. 2.2).  Fill with rpt_admm_params_default(). */
typedef struct {
  double  rho;            /* penalty rho > 0; <= 0 selects rho_scale * 2 mean_s(trace(A~_s^T A~_s))/n */
  double  rho_scale;      /* multiplier for the default rule (default 1.0) */
  double  eps_abs;        /* stopping tolerances of Eq. 9 (default 1e-4) */
  double  eps_rel;
  double  tol_obj;        /* relative change of f(z) AND-ed with Eq. 9 (Sec. 2.3); +inf = off (default) */
  int32_t max_iter;       /* ADMM iteration cap (default 5000) */
  int32_t bb_mode;        /* RPT_BB_PAPER (default) | RPT_BB_GUARDED | RPT_BB_OFF */
  double  bb_kappa;       /* guard factor for RPT_BB_GUARDED (default 10) */
  int32_t z_mode;         /* RPT_Z_STD (default) | RPT_Z_LIT */
  int32_t cg_max;         /* CG iterations per subproblem solve (default 50) */
  double  cg_theta;       /* CG stops at ||c_s - B_s x|| <= theta (rho/2) max(r_prim, eps_prim)/sqrt(N) (default 0.15) */
  double  cg_eta0;        /* first ADMM iteration: CG stops at ||r|| <= eta0 ||r_0|| (default 1e-2) */
  double  cg_floor_rel;   /* do not ask CG for ||r|| below floor_rel * ||r_0|| of the first solve
                             (default 1e-6), unless Eq. 9 needs it: the floor is capped at
                             (rho/2) eps_prim / sqrt(N), so that tight eps_abs / eps_rel are reached */
  int32_t use_graph;      /* 1 (default): one CUDA graph with device-side loops; 0: host-driven loop */
  int32_t check_every;    /* host-driven loop: read the convergence flag every k iterations (default 1);
                             the up to k - 1 iterations launched after the stop do nothing, so the
                             result and the iteration count are those of the stopping iteration */
  int32_t resume;         /* 1: start from the plan's stored state (rpt_state_set / previous solve) */
  int32_t cg_precond;     /* 0: plain CG; 1: Jacobi-preconditioned CG, M = diag(B_s) (default 1) */
  int32_t subproblem;     /* x-update (App. A): RPT_SUB_CG (default) conjugate gradients on the sparse
                             operator; RPT_SUB_CHOL the cached factor: B_s = A~_s^T A~_s + (rho/2) I
                             formed, factored and inverted once per (plan, rho) in FP32 on the device,
                             then x_s = B_s^{-1} c_s each iteration (4 n^2 N bytes of device memory,
                             plus as much again while it is formed) */
  int32_t trace;          /* 1: record one entry per iteration (see rpt_trace_get); default 0 */
  int32_t bb_per_scenario;/* 0 (default): one dual step over the concatenated vectors (Eq. 8 as
                             written); 1: Eq. 8 applied to each scenario's own blocks dd_s, dy_s,
                             one step beta_s per scenario (same bb_mode rules per scenario);
                             rpt_solve_info.step then reports the mean of the beta_s */
  double  f_target;       /* > 0: stop as soon as f(z) <= f_target instead of by Eq. 9 (one objective
                             pass per iteration checks it; tol_obj is then ignored), e.g.
                             (1 + 1e-4) f* for a time to a given objective; 0 = off (default) */
} rpt_admm_params;

#define RPT_SUB_CG   0
#define RPT_SUB_CHOL 1

/* PGD parameters (Sec. 2.1, Eq. 3 read as sufficient decrease). */
typedef struct {
  double  alpha;          /* initial step; <= 0 selects 4 / L with L = 2 lambda_max(sum_s A~_s^T A~_s) */
  double  beta;           /* sufficient-decrease constant in (0,1) (default 1e-4) */
  double  gamma;          /* step shrink factor in (0,1) (default 0.5) */
  double  tol_rel_df;     /* stop when |f_k - f_{k+1}| / f_k <= tol (default 1e-5) */
  double  f_target;       /* > 0: also stop once f <= f_target (default 0 = off) */
  int32_t max_iter;       /* default 20000 */
  int32_t max_trials;     /* Armijo trials per iteration (default 30) */
  int32_t use_graph;      /* 1 (default): device-side loops in a CUDA graph */
  int32_t reserved;
} rpt_pgd_params;

typedef struct {
  int32_t status;         /* same code as the return value */
  int32_t iterations;     /* ADMM or PGD iterations done */
  int64_t inner;          /* CG iterations (summed over scenarios) or Armijo trials */
  int64_t row_passes;     /* full passes over the stored matrices */
  int64_t kernels;        /* kernel launches of the solve (row passes + vector kernels) */
  double  seconds;        /* device time of the solve (CUDA events) */
  double  f;              /* f(x_out) (float64 accumulation) */
  double  r_prim, r_dual, eps_prim, eps_dual;   /* Eq. 9 at the last iteration (ADMM) */
  double  step;           /* last dual step (ADMM) or accepted step (PGD) */
  double  rho;            /* penalty used (ADMM) or Lipschitz estimate L (PGD) */
  double  setup_seconds;  /* RPT_SUB_CHOL: forming and inverting B_s in this call (0 if cached) */
} rpt_solve_info;

typedef struct {
  int32_t m, n, N;
  int32_t m_active;       /* rows kept on the device (rows empty in every scenario are dropped) */
  int64_t nnz;            /* total stored entries over all scenarios */
  int64_t matrix_bytes;   /* device bytes of values + indices + row pointers */
  int32_t value_format, index_width;
  int32_t row_blocks;     /* CTAs of one row pass */
  int32_t sm_count;
  double  default_rho;    /* 2 mean_s(trace(A~_s^T A~_s))/n (without rho_scale) */
  double  const_term;     /* sum over rows not stored for a scenario of c_s w_i p_i^2 (part of every f) */
  int32_t row_path;       /* row-pass implementation in use: 1 register-direct, 2 bulk-copy ring, 3 streaming,
                             4 bundled ring */
  int32_t min_lanes;      /* smallest lanes-per-row group */
  int32_t chunk_entries;  /* ring / streaming: entries per chunk (0 for the register path) */
  int32_t chunk_rows;     /* ring / streaming: rows per chunk */
  int32_t stages;         /* ring: stages */
  int32_t autotuned;      /* ring configurations timed at plan creation (0: none) */
  double  autotune_ms;    /* the chosen configuration's pass time in that timing */
  int64_t bundles;        /* path 4: row bundles over all scenarios (0 otherwise) */
  int64_t block_cols;     /* path 4: stored block columns (4 values and one index each) */
  double  bundle_fill;    /* path 4: stored entries / (4 block_cols): the share of stored values that
                             are entries of the matrix */
  int32_t exact_sums;     /* 1: the row passes sum in exact fixed point (path 4 with accumulate 1), so
                             their results do not depend on scheduling; 0: float atomics */
  int32_t ring_threads;   /* path 4: threads of a row-pass CTA (1024, 768 or 640); 0 otherwise */
  /* wall time of rpt_plan_create by phase (seconds): */
  double  layout_seconds;   /* host: validation, row compaction and the stored layout */
  double  device_seconds;   /* device set-up, allocation, upload and device-side preparation */
  double  autotune_seconds; /* ring autotuning (0 when no configuration was timed) */
} rpt_plan_stats;

/* ---- defaults ----------------------------------------------------------- */
void rpt_admm_params_default(rpt_admm_params* p);
void rpt_pgd_params_default(rpt_pgd_params* p);

/* ---- plans -------------------------------------------------------------- */

/* Validate and upload a problem; computes the weighted layout of App. A
 * (w folded per row at run time, not into the values), the row-block
 * partition and the default penalty.  Fails with RPT_EINVAL on malformed CSR
 * (row_ptr not starting at 0 or decreasing, column out of range or not
 * strictly increasing within a row), non-finite or negative val/w/p, lb > ub,
 * non-finite lb (ub may be +inf); RPT_EUNSUPPORTED for n > RPT_MAX_SPOTS, an
 * unsupported format, or a scenario with more than 2^31 - 65 entries once
 * every row is padded to a multiple of 4; RPT_ENOMEM/RPT_ECUDA on device
 * failures.  *out is set only on success. */
int rpt_plan_create(const rpt_problem* prob, const rpt_device_opts* opts, rpt_plan** out);

/* New objective weights for an existing plan (weight sweeps: the same
 * dose-influence matrices under other structure weights or prescriptions, as
 * the learned warm start is trained on).  voxel_w, presc: host [m], finite and
 * >= 0, indexed like rpt_problem.  Rewrites the stored row weights and
 * prescriptions, the Jacobi preconditioner (summed exactly in fixed point),
 * the default rho, the constant of Eq. 2 and, for row path 4, its fixed-point
 * bounds; forgets the cached factor and the Lipschitz estimate.  The stored
 * state (rpt_state_get) is kept.  The row passes then compute what a plan
 * created with these weights computes (the Jacobi diagonal and the default rho
 * may differ from a fresh plan's in the last bits, as they are summed in
 * another order).  Allocates and frees temporary device memory.  RPT_EINVAL
 * for null or invalid arrays. */
int rpt_plan_set_weights(rpt_plan* plan, const double* voxel_w, const double* presc);

/* Release a plan and its device memory.  NULL is accepted. */
void rpt_plan_destroy(rpt_plan* plan);

int rpt_plan_query(const rpt_plan* plan, rpt_plan_stats* out);

/* ---- batched plans: several problems in one plan and one launch per pass ----
 *
 * rpt_plans_create_batched puts n_plans problems with the same scenario count
 * N into one plan.  Scenario s of problem k becomes the plan's unit k * N + s,
 * with its own row lists (problem k's rows of scenario s) and its own copy of
 * the spot vectors; the problems' voxels are numbered one after another, and
 * every unit has the spot count of the widest problem (a narrower problem's
 * extra spots are held at 0 and touched by no row).  One persistent row pass
 * covers the units of every problem that is still iterating.  A batched
 * solve runs the problems side by side, each with its own consensus variable
 * z_k, its own penalty (the default rule of rpt_plan_stats.default_rho on its
 * own scenarios and spots, unless params->rho > 0 sets one for all), its own
 * BB step (Eq. 8 over its own blocks), its own residuals and tolerances of
 * Eq. 9 (eps_abs and eps_rel from params) and its own stop; a problem that
 * has converged drops out of the row passes while the others go on.  The
 * problems must share N, value_format and index_width; scenario weights and
 * bounds are each problem's own (NULL lb/ub: 0 / +inf).
 *   probs: n_plans <= 64 host pointers, each valid as for rpt_plan_create
 *          (checked per problem, so a column index is checked against its own
 *          problem's spot count).
 *   *out:  one plan holding all problems; destroy it with rpt_plan_destroy.
 *          Creation builds, on the host, one row-pointer array over all the
 *          problems' voxels per unit (4 bytes x total voxels x n_plans x N,
 *          released when the call returns).
 *          rpt_plan_query reports the problems together: m and n summed, N
 *          the scenario count of one problem, default_rho the rule on all of
 *          them stacked, const_term summed.
 * A batched plan serves rpt_admm_bb_solve_batched, rpt_plan_query,
 * rpt_plan_batch_query, rpt_profile_row_pass and rpt_trace_get (entries of
 * problem 0); the calls that take one problem's vectors (rpt_admm_bb_solve,
 * rpt_pgd_solve, rpt_objective, rpt_gradient, rpt_apply_normal,
 * rpt_state_get/set, rpt_plan_set_weights, rpt_admm_bb_solve_constrained,
 * rpt_admm_bb_solve_learned) return RPT_EUNSUPPORTED on it.
 * Errors: RPT_EINVAL for n_plans < 1, NULL arguments, an invalid problem or
 * problems that differ in N, format or index width; RPT_EUNSUPPORTED for more
 * than 64 problems or a plan beyond a limit of rpt_plan_create (e.g. the
 * widest problem's spot count above RPT_MAX_SPOTS); RPT_ENOMEM, RPT_ECUDA. */
int rpt_plans_create_batched(int32_t n_plans, const rpt_problem* const* probs, const rpt_device_opts* opts,
                             rpt_plan** out);

/* Problems in a plan and their spots numbered one after another: *n_plans (1
 * for a plan made by rpt_plan_create); col_offsets [n_plans + 1] or NULL:
 * problem k has col_offsets[k+1] - col_offsets[k] spots. */
int rpt_plan_batch_query(const rpt_plan* plan, int32_t* n_plans, int32_t* col_offsets);

/* ADMM-BB on every problem of a batched plan, side by side from a cold start
 * (z0 = 0), each problem with its own penalty, BB step and stopping test (see
 * rpt_plans_create_batched); a plan of one problem is solved as by
 * rpt_admm_bb_solve.  params->tol_obj must be +inf and f_target 0 (the
 * objective tests are not available here: RPT_EUNSUPPORTED).
 *   x_out:     one non-NULL host array per problem (rpt_plan_batch_query),
 *              x_out[k] of problem k's own spot count; for a batched plan
 *              written for every problem whatever its status (see plan_info);
 *              for a plan of one problem on RPT_OK and RPT_NOT_CONVERGED.
 *   info:      (may be NULL) the whole solve: status (RPT_OK when every problem
 *              converged, RPT_DIVERGED when one diverged, else
 *              RPT_NOT_CONVERGED), iterations (of the longest problem), CG steps,
 *              row passes, kernels and time of the one solve, f the summed
 *              objective, the residual norms over all problems' stacked
 *              vectors; step and rho 0 (they are per problem).
 *   plan_info: (may be NULL) n_plans entries, one per problem: its own status,
 *              iterations, CG steps, objective, residuals of Eq. 9, last BB
 *              step and penalty (row_passes, kernels and times: the solve's).
 * Returns info's status (also when info is NULL). */
int rpt_admm_bb_solve_batched(rpt_plan* plan, const rpt_admm_params* params, double* const* x_out,
                              rpt_solve_info* info, rpt_solve_info* plan_info);

/* ---- solvers ------------------------------------------------------------ */

/* ADMM-BB (Sec. 2.2, Eqs. 5-9; App. A).  Each iteration: x_s-updates
 * (Eq. 6) on B_s x = c_s (App. A) for all scenarios at once, by warm-started
 * conjugate gradients (RPT_SUB_CG) or by the cached inverse of B_s
 * (RPT_SUB_CHOL); z-update (box projection of the scenario mean); BB dual step
 * (Eq. 8; global, or per scenario with bb_per_scenario) and dual update
 * (Eq. 7); stopping rule (Eq. 9).
 * z0: [n] initial consensus point (projected onto the box) or NULL for 0.
 * y0: [N*n] initial duals or NULL for 0.  x_out: [n] the final z.
 * info may be NULL.  Returns RPT_OK when Eq. 9 (and the optional tol_obj
 * test) holds, RPT_NOT_CONVERGED at max_iter (x_out written), RPT_DIVERGED
 * if a residual became non-finite (x_out not written). */
int rpt_admm_bb_solve(rpt_plan* plan, const rpt_admm_params* params,
                      const double* z0, const double* y0,
                      double* x_out, rpt_solve_info* info);

/* ---- linear dose constraints (Sec. 4) --------------------------------------
 * Sec. 4 notes that ADMM, unlike PGD, accepts linear constraints on the plan
 * such as maximum or mean dose limits.  Each limit below applies to the
 * physical dose A_s x (unweighted) in every scenario s: */
#define RPT_DOSE_MAX   0   /* a_{s,i}^T x <= limit for every voxel i of the set (one row per voxel) */
#define RPT_DOSE_MIN   1   /* a_{s,i}^T x >= limit for every voxel i of the set (one row per voxel) */
#define RPT_DOSE_MEAN  2   /* (1/|S|) sum_{i in S} a_{s,i}^T x <= limit (one row) */

typedef struct {
  int32_t kind;             /* RPT_DOSE_MAX | RPT_DOSE_MIN | RPT_DOSE_MEAN */
  int32_t n_voxels;         /* >= 1 */
  const int32_t* voxels;    /* [n_voxels] host, voxel (row) indices in [0, m) */
  double  limit;            /* dose limit D (finite) */
} rpt_dose_constraint;

/* ADMM-BB with linear dose constraints as extra ADMM blocks: besides the
 * consensus x_s = z, v_s = G_s x_s with v_s <= h_s, a second dual mu_s and a
 * fixed penalty sigma (G_s, h_s: the constraint rows of scenario s, in the order
 * of `cons`, voxels in the given order, a mean constraint one row).  Each
 * iteration: x_s from the cached factor of B_s + (sigma/2) G_s^T G_s (App. A;
 * formed and inverted for this call), the z-update, v_s = min(G_s x_s +
 * mu_s/sigma, h_s), the dual step of Eq. 8 on the consensus blocks, mu_s +=
 * sigma (G_s x_s - v_s), and Eq. 9 extended to both blocks.  sigma: > 0, or 0
 * for rho.  params as for rpt_admm_bb_solve (subproblem, use_graph, resume and
 * bb_per_scenario are ignored; tol_obj and f_target are not supported:
 * RPT_EUNSUPPORTED).  x_out: [n] the final z; mu_out: [N*K] or NULL, the dose
 * duals (the multipliers of the limits at the optimum), K rows per scenario in
 * constraint order.  A voxel whose row is empty in a scenario contributes a
 * zero row there.  Returns as rpt_admm_bb_solve; RPT_EINVAL for invalid
 * constraints. */
int rpt_admm_bb_solve_constrained(rpt_plan* plan, const rpt_admm_params* params, int32_t n_cons,
                                  const rpt_dose_constraint* cons, double sigma, double* x_out, double* mu_out,
                                  rpt_solve_info* info);

/* Projected gradient descent with Armijo backtracking (Sec. 2.1, Eq. 3 read
 * as f(x+) <= f(x) + beta grad'(x+ - x)).  x0: [n] or NULL for 0; x_out [n]. */
int rpt_pgd_solve(rpt_plan* plan, const rpt_pgd_params* params,
                  const double* x0, double* x_out, rpt_solve_info* info);

/* ---- operators (for checking and for users who verify plans) ------------- */

/* f(x) (Eq. 2) and optionally the physical doses A_s x.  x: [n];
 * f_out: scalar; dose_out: [N*m] scenario-major or NULL. */
int rpt_objective(rpt_plan* plan, const double* x, double* f_out, double* dose_out);

/* Gradient of Eq. 2: g = sum_s 2 A~_s^T (A~_s x - p~_s) (Eq. 4 summed), and f(x).
 * x, g_out: [n]; f_out may be NULL. */
int rpt_gradient(rpt_plan* plan, const double* x, double* g_out, double* f_out);

/* Subproblem operator of App. A: u_s = (A~_s^T A~_s + (rho/2) I) v_s for every
 * scenario.  v, u_out: [N*n]; rho >= 0. */
int rpt_apply_normal(rpt_plan* plan, const double* v, double rho, double* u_out);

/* Time the row pass alone: `reps` back-to-back launches on the plan's stream
 * bracketed by CUDA events, over every scenario, with the spot vectors last
 * staged on the plan (e.g. by rpt_apply_normal).  mode 0: the CG operator
 * pass (A~_s^T A~_s v_s); mode 1: the residual pass (A~_s^T (A~_s v_s - p~),
 * with the objective).  *ms_per_pass: average milliseconds per launch;
 * *bytes_per_pass: the algorithmic bytes of one launch (stored values and
 * indices, row pointers, one voxel weight per row and scenario (+ one
 * prescription in mode 1), the spot vectors in and out). */
int rpt_profile_row_pass(rpt_plan* plan, int mode, int reps, double* ms_per_pass,
                         double* bytes_per_pass);

/* ---- allocation-free operator -------------------------------------------- */

/* The scenario operator u = A^T diag(w) A v + (rho/2) v (the B_s of the
 * x-subproblem, with w the scenario's row weights c_s w_i) computed from a CSR
 * matrix the caller already holds in device memory, without allocating any
 * memory.  The paper has no counterpart: it is for callers that cannot call
 * cudaMalloc -- code whose device memory is owned by a pool or framework, or a
 * loop that must not block on the allocator -- and so cannot create a plan.
 *
 * Arguments (all pointers are DEVICE pointers owned by the caller):
 *   m, n        rows (voxels) and columns (spots); 1 <= n <= 8192
 *   row_ptr_dev int32[m+1] valid CSR offsets (row_ptr[0] = 0, non-decreasing)
 *   col_idx_dev int32[row_ptr[m]] column of each entry; entries outside [0, n)
 *               are ignored
 *   val_dev     float32[row_ptr[m]] values;  row_w_dev float32[m] row weights
 *   v_dev       float32[n] input;  u_dev float32[n] output (written)
 *   rho         >= 0;  stream  cudaStream_t to run on (NULL = default stream)
 * Working memory: a file-scope device array of 4 MiB (128 x 8192 floats of
 * per-CTA partial sums), held by every device that loads the library until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  The call enqueues two kernels and returns without synchronising.
 * Every call overwrites the scratch slots it reads, so nothing needs clearing,
 * but calls that overlap on the GPU (on different streams, or on different
 * threads) share the array and race.  Results are within the float32 bound of
 * the sums but not bitwise reproducible (shared-memory float atomics).  The
 * looked-up address is kept for the process: do not call this entry point on a
 * device after a cudaDeviceReset of it.  Allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  Errors: RPT_EINVAL for bad sizes,
 * null pointers or rho < 0; RPT_EUNSUPPORTED for n > 8192; RPT_ECUDA if a
 * launch fails. */
int rpt_normal_apply_noalloc(int32_t m, int32_t n, const int32_t* row_ptr_dev, const int32_t* col_idx_dev,
                             const float* val_dev, const float* row_w_dev, const float* v_dev, double rho,
                             float* u_dev, void* stream);

/* ---- ADMM state (checkpoint / resume) ----------------------------------- */

/* The plan keeps the state (z, x_s, y_s) of its last ADMM solve.  get copies
 * it out (any pointer may be NULL to skip); set replaces it (all three
 * required), for rpt_admm_params.resume.  z: [n]; x, y: [N*n]. */
int rpt_state_get(rpt_plan* plan, double* z, double* x, double* y);
int rpt_state_set(rpt_plan* plan, const double* z, const double* x, const double* y);

/* ---- learned warm start ---------------------------------------------------
 * The paper has no learned part.  This optional form fits a small multilayer
 * perceptron that maps a plan's objective weights (features the caller chooses,
 * e.g. log structure weights and the prescription) to a spot vector, and uses it
 * as z0 of ADMM-BB; cold-start ADMM-BB is the fallback.  Network: n_in ->
 * n_hidden (x n_hidden_layers, ReLU) -> n_out (linear); loss: mean squared error
 * over the batch and the outputs; training: Adam on minibatches (every
 * minibatch full; the remainder of an epoch's permutation is skipped), on
 * the device.  Parameters as one float array: for each layer W ([out][in],
 * row-major) then b ([out]).  Host arrays X [n][n_in] and Y [n][n_out] are
 * row-major.  Compute form: see rpt_mlp_set_compute.  Errors: RPT_EINVAL for bad
 * sizes or null pointers, RPT_ECUDA. */
typedef struct rpt_mlp rpt_mlp;

typedef struct {
  int32_t epochs;         /* default 300 */
  int32_t batch;          /* minibatch rows (default 128; capped at the sample count) */
  double  lr;             /* Adam step size (default 1e-3) */
  double  beta1, beta2;   /* Adam moment decays (defaults 0.9, 0.999) */
  double  eps;            /* Adam denominator floor (default 1e-8) */
  double  weight_decay;   /* added to the gradient as wd * p (default 0) */
  uint64_t seed;          /* minibatch permutation seed (default 1) */
} rpt_mlp_train_params;

int rpt_mlp_train_params_default(rpt_mlp_train_params* tp);
/* Glorot-uniform weights from `seed`, zero biases.  n_hidden_layers may be 0. */
int rpt_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_hidden_layers, int32_t n_out, uint64_t seed,
                   int32_t device, rpt_mlp** out);
int rpt_mlp_destroy(rpt_mlp* mlp);
/* Compute form of the network's GEMMs: RPT_BF16 (default) bfloat16 weights,
 * activations and activation gradients on the tensor cores with FP32
 * accumulation (FP32 master weights take the Adam step); RPT_F32 FP32 on the
 * CUDA cores.  RPT_EINVAL for any other value. */
int rpt_mlp_set_compute(rpt_mlp* mlp, int32_t value_format);
int rpt_mlp_param_count(const rpt_mlp* mlp, int64_t* count);
int rpt_mlp_get_params(rpt_mlp* mlp, float* params);          /* params: [count] host */
int rpt_mlp_set_params(rpt_mlp* mlp, const float* params);    /* also resets the Adam moments */
/* Loss of the batch (X, Y; n rows) and its gradient with respect to the parameters
 * (grad: [count] host, or NULL), at the current parameters. */
int rpt_mlp_loss_grad(rpt_mlp* mlp, const float* X, const float* Y, int32_t n, double* loss, float* grad);
/* Train on n samples; final_loss (may be NULL) = loss of the last minibatch. */
int rpt_mlp_train(rpt_mlp* mlp, const float* X, const float* Y, int32_t n, const rpt_mlp_train_params* tp,
                  double* final_loss);
/* Network outputs for n inputs: X [n][n_in] host, Y [n][n_out] host (written). */
int rpt_mlp_predict(rpt_mlp* mlp, const float* X, int32_t n, float* Y);
/* One input: features [n_in] host -> z0_out [n_out] host, the network's warm
 * start in its training scale (multiply by the scale used for training, e.g.
 * ub, and project onto the box to use it as z0).  RPT_EINVAL for NULL
 * arguments. */
int rpt_mlp_infer(rpt_mlp* mlp, const float* features, float* z0_out);
/* ADMM-BB started from z0 = P_[lb,ub](prediction(features) * zscale) (features:
 * [n_in] host, zscale: [n] host, the scale the network was trained in, e.g. ub).
 * If that solve ends RPT_NOT_CONVERGED or RPT_DIVERGED, the cold-start solve is
 * run and returned; info then sums both.  used_warm_start (may be NULL): 1 if
 * the returned result is the warm-started one. */
int rpt_admm_bb_solve_learned(rpt_plan* plan, rpt_mlp* mlp, const float* features, const double* zscale,
                              const rpt_admm_params* params, double* x_out, rpt_solve_info* info,
                              int32_t* used_warm_start);

/* ---- tracing --------------------------------------------------------------
 * The per-iteration record of the plan's last solve run with params.trace = 1:
 * count (<= 65536) entries of 8 doubles {iteration, seconds since the first
 * iteration ended (device clock), r_prim, r_dual, eps_prim, eps_dual (Eq. 9),
 * dual step (Eq. 8), CG steps so far summed over scenarios}.  out: [cap][8] host
 * or NULL (count only).  Solves also appear as NVTX ranges ("rpt: ...") for tools. */
int rpt_trace_get(rpt_plan* plan, double* out, int32_t cap, int32_t* count);

/* ---- diagnostics --------------------------------------------------------- */
const char* rpt_status_string(int status);   /* static string */
const char* rpt_last_error(void);            /* thread-local, valid until the next call on this thread */
const char* rpt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RPT_H */
