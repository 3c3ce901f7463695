// C entry points over the batched-plan stacking header, built by
// tests/test_batch_host.py with the host compiler alone (no CUDA runtime, no
// device).
#include <cstdint>
#include <cstring>
#include <string>

#include "batch.h"

namespace {
rpt::batch::Units g_un;
std::string g_err;
}  // namespace

extern "C" {

int shim_stack(int n_plans, const rpt_problem* const* probs) {
  g_un = rpt::batch::Units();
  return rpt::batch::stack_units(n_plans, probs, &g_un, &g_err);
}

const char* shim_error() { return g_err.c_str(); }

// sizes of the result: voxels, spots per unit, units, problems, scenarios per problem
void shim_sizes(int32_t* m, int32_t* n, int32_t* U, int32_t* G, int32_t* Ns) {
  *m = g_un.view.m;
  *n = g_un.view.n;
  *U = g_un.view.N;
  *G = g_un.G;
  *Ns = g_un.Ns;
}

int32_t shim_nnz(int u) { return g_un.view.row_ptr[u][g_un.view.m]; }

void shim_unit(int u, int32_t* rp, int32_t* ci, float* va) {
  const int32_t nnz = shim_nnz(u);
  std::memcpy(rp, g_un.view.row_ptr[u], sizeof(int32_t) * (size_t)(g_un.view.m + 1));
  if (nnz > 0) {
    std::memcpy(ci, g_un.view.col_idx[u], sizeof(int32_t) * (size_t)nnz);
    std::memcpy(va, g_un.view.val[u], sizeof(float) * (size_t)nnz);
  }
}

// which: 0 voxel_w [m], 1 presc [m], 2 lb [G n], 3 ub [G n], 4 scen_weight [U]
void shim_vector(int which, double* out) {
  const rpt_problem& v = g_un.view;
  const double* src = which == 0 ? v.voxel_w : which == 1 ? v.presc : which == 2 ? g_un.lb.data()
                      : which == 3 ? g_un.ub.data() : v.scen_weight;
  const size_t len = which <= 1 ? (size_t)v.m : which <= 3 ? (size_t)g_un.G * v.n : (size_t)v.N;
  std::memcpy(out, src, sizeof(double) * len);
}

// which: 0 row offsets [G + 1], 1 spot offsets [G + 1], 2 spot counts [G]
void shim_offsets(int which, int32_t* out) {
  const std::vector<int32_t>& v = which == 0 ? g_un.row_off : which == 1 ? g_un.col_off : g_un.n_g;
  for (size_t k = 0; k < v.size(); ++k) out[k] = v[k];
}

}  // extern "C"
