// Linear dose constraints as extra ADMM blocks (Sec. 4 names maximum and mean
// dose limits as constraints that ADMM accepts and PGD does not; the splitting
// is a reading of that sentence, the same one the CPU oracle implements).
//
// Every limit applies in every scenario.  Rows of G_s, built from the physical
// dose A_s (unweighted):
//   max   a_{s,i}^T x <= D for each voxel i of a set      (one row per voxel)
//   min  -a_{s,i}^T x <= -D for each voxel i of a set     (one row per voxel)
//   mean (1/|S|) sum_{i in S} a_{s,i}^T x <= D             (one dense row)
// With v_s = G_s x_s, v_s <= h_s, a dual mu_s and a fixed penalty sigma, one
// iteration (the cached-factor x-update of App. A, B_s including the term
// (sigma/2) G_s^T G_s):
//   x_s = B_s^{-1} (A~_s^T p~ + (rho/2)(z - y_s/rho) + (sigma/2) G_s^T (v_s - mu_s/sigma))
//   z   = P_box(mean_s(x_s + y_s/rho));   v_s = min(G_s x_s + mu_s/sigma, h_s)
//   y_s += step (x_s - z) (Eq. 8 step on the consensus blocks);   mu_s += sigma (G_s x_s - v_s)
//   Eq. 9 over both blocks.
// The max and min rows are read in place from the plan's stored rows (CSR rows
// or bundle slots); mean rows are formed once per solve as dense n-vectors.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "plan.h"
#include "rowcommon.cuh"

namespace rpt {
namespace {

// One sparse constraint row of scenario s: where its entries are stored.
//   x: record (CSR row list) or bundle (bundled layout) position, -1 for a row
//      with no entries in this scenario;  y: bundle slot (-1 on CSR layouts);
//   z: +1 (max row) or -1 (min row);  w: unused
struct ConDev {
  int N, n, n_pad, Ks, Km, K;      // sparse rows, mean rows and K = Ks + Km per scenario
  const int4* rows;                // [N][Ks]
  const double* gmean;             // [N][Km][n]
  const double* h;                 // [K] limits in device order (sparse rows, then mean rows)
  double* v;                       // [N][K]
  double* mu;                      // [N][K]
  double* dv;                      // [N][K] v - v_prev of the last update
  double* cx;                      // [N][n] (sigma/2) G_s^T (v_s - mu_s/sigma)
  double* q;                       // [N][n] sigma G_s^T dv_s
  double* t;                       // [N][n] G_s^T mu_s
  double* sums;                    // [4]
  double sigma;
};

// Entry range of a stored row: CSR record q, or bundle q.
__device__ __forceinline__ void row_range(const DevPlan& P, int s, int q, bool bun, int& lo, int& hi) {
  const int4* rec = P.rowrec + P.rec_base[s];
  lo = hi = 0;
  if (q < 0) return;
  if (bun) {
    lo = rec[4 * q].x;
    hi = rec[4 * q + 4].x;
  } else {
    lo = rec[q].x;
    hi = rec[q + 1].x;
  }
}

// Column and dequantised value of stored entry e of scenario s (bundle slot r).
template <typename VT, typename IT, bool BUN>
__device__ __forceinline__ void row_entry(const DevPlan& P, int s, int e, int r, int& c, double& a) {
  const long long base = P.nnz_base[s];
  c = (int)cols<IT>(P)[base + e];
  float v;
  if (BUN) {
    float q4[4];
    quad_v<true, VT>(vals<VT>(P) + 4 * (size_t)(base + e), q4);
    v = q4[r];
  } else {
    v = to_f<VT>(vals<VT>(P)[base + e]);
  }
  a = (double)v * (P.colscale ? (double)P.colscale[(size_t)s * P.n_pad + c] : 1.0);
}

// Mean rows: gmean[s][c] += a_{s,i} / |S_c| for every member row (one warp per
// member of scenario s); members [N][M] {row position, slot, mean row c, -}, inv [Km].
template <typename VT, typename IT, bool BUN>
__global__ void k_con_mean_build(DevPlan P, ConDev D, const int4* __restrict__ members, int M,
                                 const double* __restrict__ inv) {
  const int s = blockIdx.y, lane = threadIdx.x & 31;
  const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (wid >= M) return;
  const int4 mb = members[(size_t)s * M + wid];
  int lo, hi;
  row_range(P, s, mb.x, BUN, lo, hi);
  double* g = const_cast<double*>(D.gmean) + ((size_t)s * D.Km + mb.z) * D.n;
  for (int e = lo + lane; e < hi; e += 32) {
    int c;
    double a;
    row_entry<VT, IT, BUN>(P, s, e, mb.y, c, a);
    if (a != 0.0) atomicAdd(&g[c], a * inv[mb.z]);
  }
}

// (sigma/2) G_s^T G_s into the lower triangle of B_s: sparse rows (one block per
// row and scenario, all pairs of its entries) ...
template <typename VT, typename IT, bool BUN>
__global__ void k_con_gtg(DevPlan P, ConDev D, float* __restrict__ B) {
  const int g = blockIdx.x, s = blockIdx.y;
  const int4 rw = D.rows[(size_t)s * D.Ks + g];
  int lo, hi;
  row_range(P, s, rw.x, BUN, lo, hi);
  const int len = hi - lo;
  const long long pairs = (long long)len * len;
  float* Bs = B + (size_t)s * D.n * D.n;
  for (long long p = threadIdx.x; p < pairs; p += blockDim.x) {
    const int e1 = lo + (int)(p / len), e2 = lo + (int)(p % len);
    int c1, c2;
    double a1, a2;
    row_entry<VT, IT, BUN>(P, s, e1, rw.y, c1, a1);
    row_entry<VT, IT, BUN>(P, s, e2, rw.y, c2, a2);
    if (c1 < c2 || a1 == 0.0 || a2 == 0.0) continue;
    atomicAdd(&Bs[(size_t)c1 * D.n + c2], (float)(0.5 * D.sigma * a1 * a2));
  }
}

// ... and the dense mean rows (thread per B row j, grid (ceil(n/256), N)).
__global__ void k_con_gtg_mean(ConDev D, float* __restrict__ B) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, s = blockIdx.y;
  if (j >= D.n || D.Km == 0) return;
  const double* G = D.gmean + (size_t)s * D.Km * D.n;
  float* row = B + (size_t)s * D.n * D.n + (size_t)j * D.n;
  for (int k = 0; k <= j; ++k) {
    double acc = 0.0;
    for (int c = 0; c < D.Km; ++c) acc += G[(size_t)c * D.n + j] * G[(size_t)c * D.n + k];
    if (acc != 0.0) row[k] += (float)(0.5 * D.sigma * acc);
  }
}

// After x (or at the start, with init): G_s x_s for every row, then
//   init:  v = min(Gx, h), mu = 0, dv = 0
//   else:  v' = min(Gx + mu/sigma, h), dv = v' - v, mu += sigma (Gx - v'), v = v'
// and the iteration's sums ||Gx - v'||^2, ||Gx||^2, ||v'||^2.
__device__ __forceinline__ void con_row_update(const ConDev& D, int s, int r, double gx, int init) {
  const size_t o = (size_t)s * D.K + r;
  const double h = D.h[r];
  if (init) {
    D.v[o] = fmin(gx, h);
    D.mu[o] = 0.0;
    D.dv[o] = 0.0;
    return;
  }
  const double vn = fmin(gx + D.mu[o] / D.sigma, h);
  const double rr = gx - vn;
  D.dv[o] = vn - D.v[o];
  D.mu[o] += D.sigma * rr;
  D.v[o] = vn;
  atomicAdd(&D.sums[0], rr * rr);
  atomicAdd(&D.sums[1], gx * gx);
  atomicAdd(&D.sums[2], vn * vn);
}

// one warp per (row, scenario): rows [0, Ks) sparse, [Ks, K) mean
template <typename VT, typename IT, bool BUN>
__global__ void k_con_update(DevPlan P, ConDev D, const double* __restrict__ x, int init) {
  const int s = blockIdx.y, lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= D.K) return;
  const double* xs = x + (size_t)s * D.n;
  double acc = 0.0;
  if (r < D.Ks) {
    const int4 rw = D.rows[(size_t)s * D.Ks + r];
    int lo, hi;
    row_range(P, s, rw.x, BUN, lo, hi);
    for (int e = lo + lane; e < hi; e += 32) {
      int c;
      double a;
      row_entry<VT, IT, BUN>(P, s, e, rw.y, c, a);
      acc += a * xs[c];
    }
    acc *= (double)rw.z;
  } else {
    const double* g = D.gmean + ((size_t)s * D.Km + (r - D.Ks)) * D.n;
    for (int j = lane; j < D.n; j += 32) acc += g[j] * xs[j];
  }
  acc = warp_sum_d(acc);
  if (lane == 0) con_row_update(D, s, r, acc, init);
}

// G_s^T of three row coefficients at once: cx += (sigma/2)(v - mu/sigma),
// q += sigma dv, t += mu (the buffers are zeroed by the caller).  Sparse rows:
// one warp per (row, scenario), double atomics; mean rows: see below.
template <typename VT, typename IT, bool BUN>
__global__ void k_con_scatter(DevPlan P, ConDev D) {
  const int s = blockIdx.y, lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= D.Ks) return;
  const int4 rw = D.rows[(size_t)s * D.Ks + r];
  const size_t o = (size_t)s * D.K + r;
  const double sg = (double)rw.z;
  const double wc = sg * 0.5 * D.sigma * (D.v[o] - D.mu[o] / D.sigma);
  const double wq = sg * D.sigma * D.dv[o];
  const double wt = sg * D.mu[o];
  int lo, hi;
  row_range(P, s, rw.x, BUN, lo, hi);
  double* cx = D.cx + (size_t)s * D.n;
  double* q = D.q + (size_t)s * D.n;
  double* t = D.t + (size_t)s * D.n;
  for (int e = lo + lane; e < hi; e += 32) {
    int c;
    double a;
    row_entry<VT, IT, BUN>(P, s, e, rw.y, c, a);
    if (a == 0.0) continue;
    if (wc != 0.0) atomicAdd(&cx[c], wc * a);
    if (wq != 0.0) atomicAdd(&q[c], wq * a);
    if (wt != 0.0) atomicAdd(&t[c], wt * a);
  }
}

// mean rows of the same scatter (thread per (spot, scenario), after k_con_scatter)
__global__ void k_con_scatter_mean(ConDev D) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, s = blockIdx.y;
  if (j >= D.n || D.Km == 0) return;
  double ac = 0.0, aq = 0.0, at = 0.0;
  for (int c = 0; c < D.Km; ++c) {
    const size_t o = (size_t)s * D.K + D.Ks + c;
    const double g = D.gmean[((size_t)s * D.Km + c) * D.n + j];
    ac += g * 0.5 * D.sigma * (D.v[o] - D.mu[o] / D.sigma);
    aq += g * D.sigma * D.dv[o];
    at += g * D.mu[o];
  }
  const size_t o = (size_t)s * D.n + j;
  D.cx[o] += ac;
  D.q[o] += aq;
  D.t[o] += at;
}

// c_s = A~_s^T p~ + (rho/2) z - y_s/2 + (sigma/2) G_s^T (v_s - mu_s/sigma), as float
// for the cached-factor product (grid (nchunk, N)).
__global__ void k_con_rhs(DevPlan P, const Ctl* __restrict__ C, const double* __restrict__ bchol,
                          const double* __restrict__ z, const double* __restrict__ y,
                          const double* __restrict__ cx, float* c) {
  const int s = blockIdx.y, j = blockIdx.x * kVecThreads + threadIdx.x;
  if (j >= P.n) return;
  const size_t o = (size_t)s * P.n + j;
  c[(size_t)s * P.n_pad + j] = (float)(bchol[o] + 0.5 * C->g[0].rho * z[j] - 0.5 * y[o] + cx[o]);
}

// ---- host side ----------------------------------------------------------------

template <typename VT, typename IT, bool BUN>
struct Launch {
  static void mean_build(const DevPlan& P, const ConDev& D, const int4* mem, int M, const double* inv,
                         cudaStream_t st) {
    if (M > 0) k_con_mean_build<VT, IT, BUN><<<dim3((M + 7) / 8, P.N), 256, 0, st>>>(P, D, mem, M, inv);
  }
  static void gtg(const DevPlan& P, const ConDev& D, float* B, cudaStream_t st) {
    if (D.Ks > 0) k_con_gtg<VT, IT, BUN><<<dim3(D.Ks, P.N), 256, 0, st>>>(P, D, B);
  }
  static void update(const DevPlan& P, const ConDev& D, const double* x, int init, cudaStream_t st) {
    if (D.K > 0) k_con_update<VT, IT, BUN><<<dim3((D.K + 7) / 8, P.N), 256, 0, st>>>(P, D, x, init);
  }
  static void scatter(const DevPlan& P, const ConDev& D, cudaStream_t st) {
    if (D.Ks > 0) k_con_scatter<VT, IT, BUN><<<dim3((D.Ks + 7) / 8, P.N), 256, 0, st>>>(P, D);
  }
};

// the layout- and format-specific launcher of a plan
template <template <typename, typename, bool> class F, typename... A>
void dispatch(const DevPlan& P, A&&... args) {
  const bool bun = P.path == 3;
  if (P.index_width == 16) {
    if (P.value_format == RPT_BF16) { if (bun) F<__nv_bfloat16, uint16_t, true>::run(P, args...); else F<__nv_bfloat16, uint16_t, false>::run(P, args...); }
    else if (P.value_format == RPT_FP8E4M3) { if (bun) F<__nv_fp8_e4m3, uint16_t, true>::run(P, args...); else F<__nv_fp8_e4m3, uint16_t, false>::run(P, args...); }
    else { if (bun) F<float, uint16_t, true>::run(P, args...); else F<float, uint16_t, false>::run(P, args...); }
  } else {
    if (P.value_format == RPT_BF16) { if (bun) F<__nv_bfloat16, int32_t, true>::run(P, args...); else F<__nv_bfloat16, int32_t, false>::run(P, args...); }
    else if (P.value_format == RPT_FP8E4M3) { if (bun) F<__nv_fp8_e4m3, int32_t, true>::run(P, args...); else F<__nv_fp8_e4m3, int32_t, false>::run(P, args...); }
    else { if (bun) F<float, int32_t, true>::run(P, args...); else F<float, int32_t, false>::run(P, args...); }
  }
}

template <typename VT, typename IT, bool BUN>
struct DoMean { static void run(const DevPlan& P, const ConDev& D, const int4* m, int M, const double* inv, cudaStream_t st) { Launch<VT, IT, BUN>::mean_build(P, D, m, M, inv, st); } };
template <typename VT, typename IT, bool BUN>
struct DoGtg { static void run(const DevPlan& P, const ConDev& D, float* B, cudaStream_t st) { Launch<VT, IT, BUN>::gtg(P, D, B, st); } };
template <typename VT, typename IT, bool BUN>
struct DoUpdate { static void run(const DevPlan& P, const ConDev& D, const double* x, int init, cudaStream_t st) { Launch<VT, IT, BUN>::update(P, D, x, init, st); } };
template <typename VT, typename IT, bool BUN>
struct DoScatter { static void run(const DevPlan& P, const ConDev& D, cudaStream_t st) { Launch<VT, IT, BUN>::scatter(P, D, st); } };

struct ConSolve : ConHook {
  ConDev D{};
  std::vector<void*> mem;
  double* d_sums = nullptr;

  ~ConSolve() override {
    for (void* p : mem) cudaFree(p);
  }
  template <typename T>
  cudaError_t get(T** p, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) mem.push_back(v);
    *p = static_cast<T*>(v);
    return e;
  }
  cudaError_t zero_scatter_targets(cudaStream_t st) {
    const size_t bytes = sizeof(double) * (size_t)D.N * D.n;
    cudaError_t e = cudaMemsetAsync(D.cx, 0, bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.q, 0, bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.t, 0, bytes, st);
    return e;
  }
  cudaError_t scatter(Plan* P) {
    cudaError_t e = zero_scatter_targets(P->stream);
    if (e != cudaSuccess) return e;
    dispatch<DoScatter>(P->dp, D, P->stream);
    if (D.Km > 0) k_con_scatter_mean<<<dim3((D.n + 255) / 256, D.N), 256, 0, P->stream>>>(D);
    return cudaGetLastError();
  }
  cudaError_t add(Plan* P, float* B) override {
    dispatch<DoGtg>(P->dp, D, B, P->stream);
    if (D.Km > 0) k_con_gtg_mean<<<dim3((D.n + 255) / 256, D.N), 256, 0, P->stream>>>(D, B);
    return cudaGetLastError();
  }
  cudaError_t init(Plan* P) override {
    dispatch<DoUpdate>(P->dp, D, (const double*)P->x, 1, P->stream);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? scatter(P) : e;
  }
  cudaError_t rhs(Plan* P) override {
    k_con_rhs<<<dim3(P->nchunk, D.N), kVecThreads, 0, P->stream>>>(P->dp, P->ctl, P->bchol, P->z, P->y, D.cx,
                                                                   P->v32);
    return cudaGetLastError();
  }
  cudaError_t after_z(Plan* P) override {
    cudaError_t e = cudaMemsetAsync(d_sums, 0, sizeof(double) * 4, P->stream);
    if (e != cudaSuccess) return e;
    dispatch<DoUpdate>(P->dp, D, (const double*)P->x, 0, P->stream);
    if ((e = cudaGetLastError())) return e;
    return scatter(P);
  }
};

}  // namespace
}  // namespace rpt

using namespace rpt;

extern "C" int rpt_admm_bb_solve_constrained(rpt_plan* plan, const rpt_admm_params* params, int32_t n_cons,
                                             const rpt_dose_constraint* cons, double sigma, double* x_out,
                                             double* mu_out, rpt_solve_info* info) {
  if (!plan || !params || n_cons < 0 || (n_cons > 0 && !cons)) {
    set_error("rpt_admm_bb_solve_constrained: null argument or negative count");
    return RPT_EINVAL;
  }
  Plan* P = reinterpret_cast<Plan*>(plan);
  if (int rc = refuse_batched(P, "rpt_admm_bb_solve_constrained")) return rc;
  const DevPlan& dp = P->dp;
  const int m = dp.m, n = dp.n, N = dp.N, m_act = dp.m_act;
  if (!(sigma >= 0.0) || !std::isfinite(sigma)) {
    set_error("rpt_admm_bb_solve_constrained: sigma must be finite and >= 0 (0: rho)");
    return RPT_EINVAL;
  }
  // rows in the order of the constraints (voxels in the given order, a mean row
  // where its constraint stands); on the device the sparse rows come first
  struct RowRef { int kind; int con; int voxel; double limit; };
  std::vector<RowRef> rows;
  int Km = 0;
  for (int c = 0; c < n_cons; ++c) {
    const rpt_dose_constraint& dc = cons[c];
    if (dc.kind < RPT_DOSE_MAX || dc.kind > RPT_DOSE_MEAN || dc.n_voxels < 1 || !dc.voxels ||
        !std::isfinite(dc.limit)) {
      set_error("constraint " + std::to_string(c) + ": kind, voxel list or limit invalid");
      return RPT_EINVAL;
    }
    for (int k = 0; k < dc.n_voxels; ++k)
      if (dc.voxels[k] < 0 || dc.voxels[k] >= m) {
        set_error("constraint " + std::to_string(c) + ": voxel index out of range");
        return RPT_EINVAL;
      }
    if (dc.kind == RPT_DOSE_MEAN) {
      rows.push_back({RPT_DOSE_MEAN, c, -1, dc.limit});
      ++Km;
    } else {
      for (int k = 0; k < dc.n_voxels; ++k)
        rows.push_back({dc.kind, c, dc.voxels[k], dc.kind == RPT_DOSE_MIN ? -dc.limit : dc.limit});
    }
  }
  const int K = (int)rows.size(), Ks = K - Km;
  std::vector<int> dev_of(K);   // device order: sparse rows, then mean rows
  {
    int a = 0, b = Ks;
    for (int r = 0; r < K; ++r) dev_of[r] = rows[r].kind == RPT_DOSE_MEAN ? b++ : a++;
  }
  return [&]() -> int {
    try {
      int prev = -1;
      cudaGetDevice(&prev);
      cudaSetDevice(P->device);
      struct Restore {
        int d;
        ~Restore() {
          if (d >= 0) cudaSetDevice(d);
        }
      } restore{prev};
      std::vector<int> kept_of(m, -1);
      for (int k = 0; k < m_act; ++k) kept_of[P->kept_rows[k]] = k;
      const bool bun = dp.path == 3;
      // where a voxel's row of scenario s is stored: {position, slot}
      auto locate = [&](int s, int voxel) {
        const int k = kept_of[voxel];
        if (k < 0) return std::make_pair(-1, -1);
        const int idx = P->nz_index[(size_t)s * m_act + k];
        if (idx < 0) return std::make_pair(-1, -1);
        if (bun) return std::make_pair(P->rec_of_host[(size_t)s * m_act + idx / kBundleRows], idx % kBundleRows);
        return std::make_pair(P->rec_of_host[(size_t)s * m_act + k], -1);
      };
      std::vector<int4> h_rows((size_t)N * Ks);
      std::vector<double> h_lim(K);
      for (int r = 0; r < K; ++r) h_lim[dev_of[r]] = rows[r].limit;
      for (int s = 0; s < N; ++s)
        for (int r = 0; r < K; ++r) {
          if (rows[r].kind == RPT_DOSE_MEAN) continue;
          const auto loc = locate(s, rows[r].voxel);
          h_rows[(size_t)s * Ks + dev_of[r]] =
              make_int4(loc.first, loc.second, rows[r].kind == RPT_DOSE_MIN ? -1 : 1, 0);
        }
      // mean-row members
      std::vector<double> inv(std::max(Km, 1), 0.0);
      std::vector<std::vector<int4>> mem_s(N);
      for (int r = 0; r < K; ++r) {
        if (rows[r].kind != RPT_DOSE_MEAN) continue;
        const rpt_dose_constraint& dc = cons[rows[r].con];
        const int c = dev_of[r] - Ks;
        inv[c] = 1.0 / dc.n_voxels;
        for (int s = 0; s < N; ++s)
          for (int k = 0; k < dc.n_voxels; ++k) {
            const auto loc = locate(s, dc.voxels[k]);
            if (loc.first >= 0) mem_s[s].push_back(make_int4(loc.first, loc.second, c, 0));
          }
      }
      int M = 0;
      for (int s = 0; s < N; ++s) M = std::max(M, (int)mem_s[s].size());
      std::vector<int4> h_mem((size_t)N * M, make_int4(-1, -1, 0, 0));
      for (int s = 0; s < N; ++s) std::copy(mem_s[s].begin(), mem_s[s].end(), h_mem.begin() + (size_t)s * M);

      ConSolve S;
      ConDev& D = S.D;
      D.N = N;
      D.n = n;
      D.n_pad = dp.n_pad;
      D.Ks = Ks;
      D.Km = Km;
      D.K = K;
      int4 *d_rows = nullptr, *d_mem = nullptr;
      double *d_gmean = nullptr, *d_h = nullptr, *d_inv = nullptr;
      const size_t Nn = (size_t)N * n;
      cudaError_t e = S.get(&d_rows, h_rows.size());
      if (!e) e = S.get(&d_mem, h_mem.size());
      if (!e) e = S.get(&d_gmean, (size_t)N * Km * n);
      if (!e) e = S.get(&d_h, K);
      if (!e) e = S.get(&d_inv, inv.size());
      if (!e) e = S.get(&D.v, (size_t)N * K);
      if (!e) e = S.get(&D.mu, (size_t)N * K);
      if (!e) e = S.get(&D.dv, (size_t)N * K);
      if (!e) e = S.get(&D.cx, Nn);
      if (!e) e = S.get(&D.q, Nn);
      if (!e) e = S.get(&D.t, Nn);
      if (!e) e = S.get(&S.d_sums, 4);
      if (e) return cuda_fail(e, "dose-constraint buffers");
      cudaStream_t st = P->stream;
      if (!h_rows.empty()) e = cudaMemcpyAsync(d_rows, h_rows.data(), sizeof(int4) * h_rows.size(), cudaMemcpyHostToDevice, st);
      if (!e && !h_mem.empty()) e = cudaMemcpyAsync(d_mem, h_mem.data(), sizeof(int4) * h_mem.size(), cudaMemcpyHostToDevice, st);
      if (!e && K) e = cudaMemcpyAsync(d_h, h_lim.data(), sizeof(double) * K, cudaMemcpyHostToDevice, st);
      if (!e) e = cudaMemcpyAsync(d_inv, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice, st);
      if (!e && Km) e = cudaMemsetAsync(d_gmean, 0, sizeof(double) * (size_t)N * Km * n, st);
      if (!e) e = cudaMemsetAsync(S.d_sums, 0, sizeof(double) * 4, st);
      if (e) return cuda_fail(e, "dose-constraint upload");
      D.rows = d_rows;
      D.gmean = d_gmean;
      D.h = d_h;
      D.sums = S.d_sums;
      // the penalty: sigma, or rho when 0 (the oracle's default)
      const double rho = params->rho > 0 ? params->rho : params->rho_scale * P->stats.default_rho;
      D.sigma = sigma > 0.0 ? sigma : rho;
      if (M > 0 && Km > 0) dispatch<DoMean>(dp, D, (const int4*)d_mem, M, (const double*)d_inv, st);
      if ((e = cudaGetLastError())) return cuda_fail(e, "mean rows");
      S.q = D.q;
      S.t = D.t;
      S.sums = S.d_sums;
      S.K = (double)N * K;
      rpt_admm_params prm = *params;
      prm.subproblem = RPT_SUB_CHOL;
      prm.use_graph = 0;
      prm.resume = 0;
      prm.bb_per_scenario = 0;
      if (std::isfinite(prm.tol_obj) || prm.f_target > 0.0) {
        set_error("rpt_admm_bb_solve_constrained: tol_obj and f_target are not supported with constraints");
        return RPT_EUNSUPPORTED;
      }
      const int rc = admm_solve(P, &prm, nullptr, nullptr, x_out, info, &S);
      if ((rc == RPT_OK || rc == RPT_NOT_CONVERGED) && mu_out && K > 0) {
        std::vector<double> mu((size_t)N * K);
        e = cudaMemcpyAsync(mu.data(), D.mu, sizeof(double) * mu.size(), cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaStreamSynchronize(st);
        if (e) return cuda_fail(e, "copy mu");
        for (int s = 0; s < N; ++s)
          for (int r = 0; r < K; ++r) mu_out[(size_t)s * K + r] = mu[(size_t)s * K + dev_of[r]];
      }
      cudaStreamSynchronize(st);
      return rc;
    } catch (const std::bad_alloc&) {
      set_error("out of host memory");
      return RPT_ENOMEM;
    }
  }();
}
