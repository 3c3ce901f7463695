// C entry points over the stacking header, built by tests/test_batch_host.py
// with the host compiler alone (no CUDA runtime, no device).
#include <cstdint>
#include <cstring>
#include <string>

#include "batch.h"

namespace {
rpt::batch::Stacked g_st;
std::string g_err;
}  // namespace

extern "C" {

int shim_stack(int n_plans, const rpt_problem* const* probs) {
  g_st = rpt::batch::Stacked();
  return rpt::batch::stack_problems(n_plans, probs, &g_st, &g_err);
}

const char* shim_error() { return g_err.c_str(); }

void shim_sizes(int32_t* m, int32_t* n, int32_t* N, int32_t* n_off, int32_t* has_sw) {
  *m = g_st.view.m;
  *n = g_st.view.n;
  *N = g_st.view.N;
  *n_off = (int32_t)g_st.col_off.size();
  *has_sw = g_st.view.scen_weight != nullptr;
}

int32_t shim_nnz(int s) { return g_st.view.row_ptr[s][g_st.view.m]; }

void shim_scenario(int s, int32_t* rp, int32_t* ci, float* va) {
  const int32_t nnz = shim_nnz(s);
  std::memcpy(rp, g_st.view.row_ptr[s], sizeof(int32_t) * (size_t)(g_st.view.m + 1));
  std::memcpy(ci, g_st.view.col_idx[s], sizeof(int32_t) * (size_t)nnz);
  std::memcpy(va, g_st.view.val[s], sizeof(float) * (size_t)nnz);
}

// which: 0 voxel_w, 1 presc, 2 lb, 3 ub, 4 scen_weight
void shim_vector(int which, double* out) {
  const rpt_problem& v = g_st.view;
  const double* src = which == 0 ? v.voxel_w : which == 1 ? v.presc : which == 2 ? v.lb : which == 3 ? v.ub
                                                                                                      : v.scen_weight;
  const int len = which <= 1 ? v.m : which <= 3 ? v.n : v.N;
  std::memcpy(out, src, sizeof(double) * (size_t)len);
}

void shim_offsets(int32_t* out) {
  for (size_t k = 0; k < g_st.col_off.size(); ++k) out[k] = g_st.col_off[k];
}

}  // extern "C"
