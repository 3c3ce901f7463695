// batch.h -- several planning problems as the groups of one plan (host only, no device code).
//
// Problems with the same scenario count Ns become the groups of one plan.  The
// plan's scenario u = g * Ns + s is the unit (problem g, scenario s).  The
// voxels (rows) of all problems are concatenated: unit u's matrix holds
// problem g's rows of scenario s at problem g's row offset and no entry in any
// other problem's rows.  Spot indices stay the problem's own (0 .. n_g - 1);
// every unit has n = max_g n_g spots, and the spots a narrower problem does not
// have are fixed at 0 by the box lb = ub = 0 (no row touches them).  The
// plan's objective (Eq. 2) is the sum of the problems' objectives and the
// problems share no variable, so the solver runs them side by side, each with
// its own consensus variable, penalty, BB step and stopping rule, while one
// row pass per operator application covers the units of every problem that is
// still iterating.  Compiled into the library and, on its own, by the CPU
// tests that check the stacking.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/rpt.h"

namespace rpt {
namespace batch {

constexpr int kMaxProblems = 64;   // problems in one batched plan

// The units' arrays and an rpt_problem view of them (G * Ns scenarios of n
// spots).  Row pointers are owned; column indices and values point into the
// problems' own arrays.  Bounds are per problem: lb, ub [G][n].
struct Units {
  int G = 0, Ns = 0, n = 0;
  std::vector<std::vector<int32_t>> rp;    // [G * Ns][M + 1]
  std::vector<const int32_t*> rp_p, ci_p;  // [G * Ns]
  std::vector<const float*> va_p;          // [G * Ns]
  std::vector<double> w, p, sw;            // [M], [M], [G * Ns] (a problem's NULL weights: 1)
  std::vector<double> lb, ub;              // [G][n]; spots j >= n_g: lb = ub = 0
  std::vector<int32_t> row_off;            // [G + 1]: problem g owns rows row_off[g] .. row_off[g+1]
  std::vector<int32_t> n_g;                // [G]
  std::vector<int32_t> col_off;            // [G + 1]: the problems' spots numbered one after another
  rpt_problem view{};                      // view.lb / view.ub: problem 0's; the plan reads lb, ub
};

// Build the units of n_plans problems whose CSR arrays are already valid (each
// problem as rpt_plan_create requires).  Checks what stacking itself needs: at
// most kMaxProblems problems, the same scenario count, value format and index
// width in every problem, and sizes that fit the int32 fields of the result.
// Returns RPT_OK or an error code with *err set; *out is complete only on RPT_OK.
inline int stack_units(int n_plans, const rpt_problem* const* probs, Units* out, std::string* err) {
  if (n_plans < 1 || !probs || !out) {
    *err = "n_plans >= 1 and non-null arguments needed";
    return RPT_EINVAL;
  }
  if (n_plans > kMaxProblems) {
    *err = "at most " + std::to_string(kMaxProblems) + " problems in one batched plan";
    return RPT_EUNSUPPORTED;
  }
  for (int k = 0; k < n_plans; ++k)
    if (!probs[k]) {
      *err = "problem " + std::to_string(k) + " is NULL";
      return RPT_EINVAL;
    }
  const rpt_problem& p0 = *probs[0];
  const int Ns = p0.N;
  int64_t M = 0, nmax = 0, ntot = 0;
  for (int k = 0; k < n_plans; ++k) {
    const rpt_problem& q = *probs[k];
    if (q.N != Ns || q.value_format != p0.value_format || q.index_width != p0.index_width) {
      *err = "problem " + std::to_string(k) + " differs from problem 0 in scenario count, value format or index width";
      return RPT_EINVAL;
    }
    M += q.m;
    nmax = std::max<int64_t>(nmax, q.n);
    ntot += q.n;
  }
  if (M > INT32_MAX - 1 || ntot > INT32_MAX - 1) {
    *err = "stacked voxel or spot count exceeds int32";
    return RPT_EUNSUPPORTED;
  }
  const int G = n_plans, U = G * Ns;
  out->G = G;
  out->Ns = Ns;
  out->n = (int)nmax;
  out->row_off.assign(1, 0);
  out->col_off.assign(1, 0);
  out->n_g.clear();
  out->w.clear();
  out->p.clear();
  out->lb.assign((size_t)G * nmax, 0.0);
  out->ub.assign((size_t)G * nmax, 0.0);
  out->sw.assign(U, 1.0);
  for (int k = 0; k < G; ++k) {
    const rpt_problem& q = *probs[k];
    out->w.insert(out->w.end(), q.voxel_w, q.voxel_w + q.m);
    out->p.insert(out->p.end(), q.presc, q.presc + q.m);
    for (int j = 0; j < q.n; ++j) {
      out->lb[(size_t)k * nmax + j] = q.lb ? q.lb[j] : 0.0;
      out->ub[(size_t)k * nmax + j] = q.ub ? q.ub[j] : HUGE_VAL;
    }
    if (q.scen_weight)
      for (int s = 0; s < Ns; ++s) out->sw[(size_t)k * Ns + s] = q.scen_weight[s];
    out->row_off.push_back(out->row_off.back() + q.m);
    out->col_off.push_back(out->col_off.back() + q.n);
    out->n_g.push_back(q.n);
  }
  out->rp.assign(U, {});
  out->rp_p.assign(U, nullptr);
  out->ci_p.assign(U, nullptr);
  out->va_p.assign(U, nullptr);
  for (int k = 0; k < G; ++k) {
    const rpt_problem& q = *probs[k];
    const int r0 = out->row_off[k];
    for (int s = 0; s < Ns; ++s) {
      const int u = k * Ns + s;
      const int32_t* qrp = q.row_ptr[s];
      const int32_t nnz = qrp[q.m];
      std::vector<int32_t>& rp = out->rp[u];
      rp.assign((size_t)M + 1, 0);   // rows before problem k: empty
      for (int i = 0; i <= q.m; ++i) rp[(size_t)r0 + i] = qrp[i];
      for (int64_t i = (int64_t)r0 + q.m + 1; i <= M; ++i) rp[(size_t)i] = nnz;   // rows after: empty
      out->rp_p[u] = rp.data();
      out->ci_p[u] = q.col_idx[s];
      out->va_p[u] = q.val[s];
    }
  }
  rpt_problem& v = out->view;
  v.m = (int32_t)M;
  v.n = (int32_t)nmax;
  v.N = U;
  v.row_ptr = out->rp_p.data();
  v.col_idx = out->ci_p.data();
  v.val = out->va_p.data();
  v.voxel_w = out->w.data();
  v.presc = out->p.data();
  v.scen_weight = out->sw.data();
  v.lb = out->lb.data();
  v.ub = out->ub.data();
  v.value_format = p0.value_format;
  v.index_width = p0.index_width;
  return RPT_OK;
}

}  // namespace batch
}  // namespace rpt
