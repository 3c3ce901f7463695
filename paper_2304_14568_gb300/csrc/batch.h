// batch.h -- several planning problems stacked into one (host only, no device code).
//
// Problems with the same scenario count N are placed side by side: voxels
// (rows) and spots (columns) are concatenated, so scenario s of the result is
// blockdiag(A_s of each problem).  The objective of the result is the sum of
// the problems' objectives (Eq. 2) and its box is the product of their boxes,
// so its optimum is the problems' optima side by side and one plan, one row
// pass per operator application and one solve cover them all.  Compiled into
// the library and, on its own, by the CPU tests that check the stacking.
#pragma once

#include <stdint.h>

#include <climits>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/rpt.h"

namespace rpt {
namespace batch {

// The stacked problem's arrays (owned) and an rpt_problem view of them.
struct Stacked {
  std::vector<std::vector<int32_t>> rp, ci;
  std::vector<std::vector<float>> va;
  std::vector<const int32_t*> rp_p, ci_p;
  std::vector<const float*> va_p;
  std::vector<double> w, p, sw, lb, ub;
  std::vector<int32_t> col_off;   // [n_plans + 1]: problem k owns spots col_off[k] .. col_off[k+1]
  rpt_problem view{};
};

// Stack n_plans problems whose CSR arrays are already valid (each problem as
// rpt_plan_create requires).  Checks what stacking itself needs: the same N,
// value format and index width in every problem, equal scenario weights (all
// NULL, or the same N values: the stacked problem has one c_s per scenario),
// and sizes that fit the int32 fields of the result.  Returns RPT_OK or an
// error code with *err set; *out is complete only on RPT_OK.
inline int stack_problems(int n_plans, const rpt_problem* const* probs, Stacked* out, std::string* err) {
  if (n_plans < 1 || !probs || !out) {
    *err = "n_plans >= 1 and non-null arguments needed";
    return RPT_EINVAL;
  }
  for (int k = 0; k < n_plans; ++k)
    if (!probs[k]) {
      *err = "problem " + std::to_string(k) + " is NULL";
      return RPT_EINVAL;
    }
  const rpt_problem& p0 = *probs[0];
  const int N = p0.N;
  int64_t M = 0, Ncol = 0;
  for (int k = 0; k < n_plans; ++k) {
    const rpt_problem& q = *probs[k];
    if (q.N != N || q.value_format != p0.value_format || q.index_width != p0.index_width) {
      *err = "problem " + std::to_string(k) + " differs from problem 0 in scenario count, value format or index width";
      return RPT_EINVAL;
    }
    if ((q.scen_weight == nullptr) != (p0.scen_weight == nullptr)) {
      *err = "problem " + std::to_string(k) + ": scenario weights given for some problems only";
      return RPT_EINVAL;
    }
    if (q.scen_weight)
      for (int s = 0; s < N; ++s)
        if (!(q.scen_weight[s] == p0.scen_weight[s])) {
          *err = "problem " + std::to_string(k) + ": scenario weights differ from problem 0";
          return RPT_EINVAL;
        }
    M += q.m;
    Ncol += q.n;
  }
  if (M > INT32_MAX - 1 || Ncol > INT32_MAX - 1) {
    *err = "stacked voxel or spot count exceeds int32";
    return RPT_EUNSUPPORTED;
  }
  out->rp.assign(N, {});
  out->ci.assign(N, {});
  out->va.assign(N, {});
  for (int s = 0; s < N; ++s) {
    int64_t nnz = 0;
    for (int k = 0; k < n_plans; ++k) nnz += probs[k]->row_ptr[s][probs[k]->m];
    if (nnz > INT32_MAX) {
      *err = "scenario " + std::to_string(s) + ": stacked entry count exceeds int32";
      return RPT_EUNSUPPORTED;
    }
    std::vector<int32_t>& rp = out->rp[s];
    std::vector<int32_t>& ci = out->ci[s];
    std::vector<float>& va = out->va[s];
    rp.resize((size_t)M + 1);
    ci.resize((size_t)nnz);
    va.resize((size_t)nnz);
    int64_t r0 = 0, e0 = 0, c0 = 0;
    for (int k = 0; k < n_plans; ++k) {
      const rpt_problem& q = *probs[k];
      const int32_t* qrp = q.row_ptr[s];
      for (int i = 0; i < q.m; ++i) rp[(size_t)(r0 + i)] = (int32_t)(e0 + qrp[i]);
      const int32_t qn = qrp[q.m];
      for (int32_t e = 0; e < qn; ++e) {
        ci[(size_t)(e0 + e)] = (int32_t)(c0 + q.col_idx[s][e]);
        va[(size_t)(e0 + e)] = q.val[s][e];
      }
      r0 += q.m;
      e0 += qn;
      c0 += q.n;
    }
    rp[(size_t)M] = (int32_t)e0;
  }
  out->w.clear();
  out->p.clear();
  out->lb.clear();
  out->ub.clear();
  out->col_off.assign(1, 0);
  for (int k = 0; k < n_plans; ++k) {
    const rpt_problem& q = *probs[k];
    out->w.insert(out->w.end(), q.voxel_w, q.voxel_w + q.m);
    out->p.insert(out->p.end(), q.presc, q.presc + q.m);
    for (int j = 0; j < q.n; ++j) {
      out->lb.push_back(q.lb ? q.lb[j] : 0.0);
      out->ub.push_back(q.ub ? q.ub[j] : HUGE_VAL);
    }
    out->col_off.push_back(out->col_off.back() + q.n);
  }
  out->sw.assign(p0.scen_weight ? p0.scen_weight : nullptr, p0.scen_weight ? p0.scen_weight + N : nullptr);
  out->rp_p.resize(N);
  out->ci_p.resize(N);
  out->va_p.resize(N);
  for (int s = 0; s < N; ++s) {
    out->rp_p[s] = out->rp[s].data();
    out->ci_p[s] = out->ci[s].data();
    out->va_p[s] = out->va[s].data();
  }
  rpt_problem& v = out->view;
  v.m = (int32_t)M;
  v.n = (int32_t)Ncol;
  v.N = N;
  v.row_ptr = out->rp_p.data();
  v.col_idx = out->ci_p.data();
  v.val = out->va_p.data();
  v.voxel_w = out->w.data();
  v.presc = out->p.data();
  v.scen_weight = out->sw.empty() ? nullptr : out->sw.data();
  v.lb = out->lb.data();
  v.ub = out->ub.data();
  v.value_format = p0.value_format;
  v.index_width = p0.index_width;
  return RPT_OK;
}

}  // namespace batch
}  // namespace rpt
