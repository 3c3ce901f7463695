// Host-side plan object (what an rpt_plan* points to) and the solver entry
// points implemented in solver.cu.
#pragma once
#include <string>
#include <vector>

#include "../../include/rpt.h"
#include "common.cuh"

namespace rpt {

// Groups of a batched plan.  A batched plan holds G independent problems with
// the same scenario count Ns; its scenario index u = g * Ns + s runs over
// (problem g, scenario s) units, each with its own row lists and its own copy
// of the spot vectors (n spots each, the widest problem's count; a narrower
// problem's extra spots are fixed at 0 by the box lb = ub = 0 and touched by
// no row).  Every problem keeps its own consensus z_g, penalty, BB step,
// residuals and stopping test, and a problem that has converged drops out of
// the row passes.  A plan from rpt_plan_create is one group (G = 1, Ns = N).
constexpr int kMaxGroups = 64;
struct Grp {
  double rho, inv_rho;                 // penalty of the group's B_s, z-update and r_dual
  double r_prim, r_dual, eps_prim, eps_dual, step, step_prev, sz2, dz2;
  double nn;                           // Ns x (the problem's own spot count): the length in eps_abs sqrt(N n)
  double cst;                          // constant objective term of the group's rows
  double f;                            // objective of the group's z after the solve
  long long cg;                        // CG steps of the group's scenarios
  int k, have_prev, first, status, done, diverged;
};

// Device-resident solver control block: parameters of the current solve and
// the scalars of the iteration (written and read by the kernels).
struct Ctl {
  // ADMM parameters
  double eps_abs, eps_rel, bb_kappa, cg_theta, cg_eta0, cg_floor, tol_obj, f_goal;
  double const_term;
  int max_iter, cg_max, bb_mode, z_mode, use_obj, precond;
  // ADMM scalars over all groups: loop count, loop condition, every group
  // converged, some group diverged
  int k, kcg, cg_any, stop, status, diverged;
  long long cg_total, passes, cg_steps;
  double f_prev, f_cur;
  // PGD parameters and scalars
  double alpha, beta_a, gamma, tol_df, f_target, t, fx, ft, gd, pstep;
  int pgd_max_iter, max_trials, trial, accepted, failed, pk, pouter, pad2;
  long long trials_total;
  // last-block-done counters (every finisher resets its own counter)
  unsigned int cnt_init, cnt_upd, cnt_d, cnt_y, cnt_z, cnt_red, cnt_pg, cnt_pt;
  unsigned int pad3;
  // optional per-iteration trace (rpt_admm_params.trace): kTraceFields doubles per
  // iteration, at most trace_cap iterations, written by the dual update's last block
  double* trace;
  int trace_cap, trace_on;
  unsigned long long t_start;      // %globaltimer at the first iteration (trace time base)
  // per-scenario dual steps (rpt_admm_params.bb_per_scenario): [N], each holding the
  // step of the scenario's last dual update until the next BB computation replaces it
  double* step_s;
  int bb_scen, pad4;
  // dose-constraint blocks (rpt_admm_bb_solve_constrained): the residual pieces of
  // the iteration, written by the constraint kernels before k_admm_d / k_admm_y
  const double* con_q;    // [N][n] sigma G_s^T (v_s - v_s_prev)
  const double* con_t;    // [N][n] G_s^T mu_s
  const double* con_sums; // [4] ||G x - v||^2, ||G x||^2, ||v||^2 over all scenarios
  double con_K;           // constraint rows over all scenarios
  int con_on, pad5;
  // per-unit activity of the residual pass of a batched plan (0: the unit's
  // problem has converged), written with the groups' stopping tests
  int* uact;
  Grp g[kMaxGroups];      // per group (one per problem of a batched plan)
};

// trace entry: iteration, seconds since the solve started, r_prim, r_dual,
// eps_prim, eps_dual, dual step, CG steps so far (summed over scenarios)
constexpr int kTraceFields = 8;
constexpr int kTraceCap = 1 << 16;

struct Plan {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int sm_count = 0;
  rpt_plan_stats stats{};
  DevPlan dp{};
  int nchunk = 0;                 // column chunks of kVecThreads

  // device allocations (owned)
  std::vector<void*> allocs;

  // matrix-side arrays are in dp; solver buffers:
  double *x = nullptr, *r = nullptr, *p = nullptr, *u = nullptr, *y = nullptr;
  double *d = nullptr, *dprev = nullptr, *z = nullptr, *znew = nullptr;
  double *lb = nullptr, *ub = nullptr;
  float *v32 = nullptr;           // [N][n_pad] staged per-scenario vectors
  float *vz32 = nullptr;          // [n_pad] staged shared vector
  float *partial = nullptr;       // [nblocks][n_pad]
  double *objp = nullptr;         // [nblocks]
  double *q = nullptr, *dinv = nullptr;   // CG: B p, M^{-1}
  float *diag = nullptr;          // [N][n] diag(A~_s^T A~_s)
  double *gam = nullptr, *tol = nullptr, *r0n = nullptr, *alpha = nullptr, *beta = nullptr;
  double *bb_step = nullptr;      // [N] per-scenario ADMM dual steps
  double *gprev = nullptr, *aprev = nullptr;
  int *act = nullptr, *act_next = nullptr, *cgcnt = nullptr, *cgi = nullptr;
  int *err = nullptr;             // device error word of the row passes
  unsigned int *cnt_s = nullptr;  // [N] per-scenario counters
  double *dots = nullptr;         // [N][nchunk][4]
  double *vpart = nullptr;        // [nchunk*N][8]
  double *g = nullptr, *xt = nullptr, *xp = nullptr;   // PGD [n]
  float *dose = nullptr;          // [N][m_act] (allocated on demand)
  Ctl *ctl = nullptr;             // device control block
  Ctl *ctl_host = nullptr;        // pinned mirror

  // cached-factor subproblem (chol.cu): B_s^{-1} [N][n][n] FP32, A~_s^T p~ [N][n],
  // record index of kept row k in scenario s's list [N][m_act] (-1: empty there)
  float *binv = nullptr;
  double *bchol = nullptr;
  int *rec_of = nullptr;
  double *trace = nullptr;         // [kTraceCap][kTraceFields] (allocated on first traced solve)
  int trace_count = 0;             // entries of the last traced solve
  bool chol_ready = false;
  bool chol_con = false;          // the cached factor includes dose-constraint terms
  std::vector<double> chol_rho;   // per group: the penalties the cached factor was formed with
  cudaGraphExec_t admm_chol_exec = nullptr;
  int admm_chol_exec_obj = -1;

  std::vector<int32_t> kept_rows; // original row index of each device row
  // what rpt_plan_set_weights needs: scenario weights c_s, rows dropped at
  // creation (empty in every scenario), per scenario the kept rows that are empty
  // there, and per scenario max_j sum_i a_ij^2 (the scale of the diagonal sums)
  std::vector<double> scen_c;
  std::vector<int32_t> dropped_rows;
  std::vector<std::vector<int32_t>> empty_kept;
  std::vector<double> colsq_max;
  // where each kept row of each scenario sits in the stored layout (dose
  // constraints read constrained rows from it): rec_of_host = the device rec_of
  // ([N][m_act]: CSR paths: position of kept row k in scenario s's row list;
  // bundled path: sorted position of the q-th bundle in creation order), and
  // nz_index[s][k] = position of kept row k among scenario s's non-empty rows in
  // kept order (-1: the row is empty in s), which gives a row's bundle (index / 4)
  // and slot (index % 4)
  std::vector<int32_t> rec_of_host;
  std::vector<int32_t> nz_index;
  std::vector<int32_t> batch_col_off;  // batched plan: problem k owns spots [off[k], off[k+1]) of the
                                       // stacked numbering; else empty
  // per group (one for a plan from rpt_plan_create): default penalty (the rule of
  // stats.default_rho on the group's own scenarios and spots), constant objective
  // term, own spot count
  std::vector<double> grp_rho, grp_const;
  std::vector<int32_t> grp_n;
  int *uact = nullptr;            // [N] residual-pass activity per unit (batched plans)
  double lipschitz = 0.0;         // cached 2 lambda_max, 0 = not computed
  bool state_valid = false;

  // CUDA graphs (built on first use)
  cudaGraphExec_t admm_exec = nullptr;
  int admm_exec_obj = -1;         // use_obj flag the graph was built with
  cudaGraphExec_t pgd_exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// chol.cu: form, factor and invert B_s for this rho; `extra` (may be null) adds
// further terms to the lower triangle of every B_s before the factorisation
// (B_s row-major [N][n][n] float, launched on the plan's stream) and marks the
// factor as not reusable by plain solves
struct CholExtra {
  virtual cudaError_t add(Plan* P, float* B) = 0;
  virtual ~CholExtra() = default;
};
// Dose-constraint blocks of a cached-factor ADMM-BB solve (dosecon.cu): the
// solver calls init after its own initialisation, rhs in place of the plain
// right-hand side c_s (into v32, float), and after_z between the z-update and
// the BB / dual kernels; q, t, sums and K feed the extended residuals of Eq. 9.
struct ConHook : CholExtra {
  const double* q = nullptr;      // [N][n]
  const double* t = nullptr;      // [N][n]
  const double* sums = nullptr;   // [4]
  double K = 0.0;
  virtual cudaError_t init(Plan* P) = 0;
  virtual cudaError_t rhs(Plan* P) = 0;
  virtual cudaError_t after_z(Plan* P) = 0;
};

// x_out: n spots (G x n for a batched plan, group-major); group_info: G entries or null
int admm_solve(Plan* P, const rpt_admm_params* prm, const double* z0, const double* y0,
               double* x_out, rpt_solve_info* info, ConHook* con = nullptr,
               rpt_solve_info* group_info = nullptr);
int pgd_solve(Plan* P, const rpt_pgd_params* prm, const double* x0, double* x_out,
              rpt_solve_info* info);
int op_apply_normal(Plan* P, const double* v, double rho, double* u_out);
int op_gradient(Plan* P, const double* x, double* g_out, double* f_out);
int op_objective(Plan* P, const double* x, double* f_out, double* dose_out);
int compute_lipschitz(Plan* P, double* L);
int profile_row_pass(Plan* P, int mode, int reps, double* ms, double* bytes);
void destroy_graphs(Plan* P);
// chol.cu (see CholExtra)
// rho: one penalty per group
int chol_prepare(Plan* P, const std::vector<double>& rho, CholExtra* extra = nullptr);


int compute_bconst(Plan* P);             // solver.cu: P->bchol = A~_s^T p~

// error reporting (api.cu)
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// Calls that take one problem's vectors refuse a batched plan (several groups):
// RPT_EUNSUPPORTED with the message set, else RPT_OK.
inline int refuse_batched(const Plan* P, const char* call) {
  if (P->dp.G <= 1) return RPT_OK;
  set_error(std::string(call) + ": not available on a batched plan (use rpt_admm_bb_solve_batched)");
  return RPT_EUNSUPPORTED;
}

}  // namespace rpt
