// ADMM-BB and PGD on the device.
//
// ADMM-BB (Sec. 2.2).  One iteration k:
//   a. residual pass   g_s = A~_s^T (A~_s x_s - p~)              (row pass, kResid)
//      r_s = c_s - B_s x_s = -g_s - (rho/2)(x_s - z) - y_s/2     (App. A: B_s, c_s)
//   b. CG on B_s x_s = c_s for all scenarios at once, warm-started from x_s
//      (each CG step: one row pass kNormal + one vector kernel)
//   c. z = P_box(mean_s(x_s + y_s/rho))                          (z-update)
//   d. d = x - 1(x)z; BB step from dd = d - d_prev and dy = step_prev d_prev (Eq. 8)
//   e. y_s += step d_s (Eq. 7); residuals and tolerances of Eq. 9; stop test.
// All loops are device-side: a CUDA graph with a WHILE node for the ADMM
// iteration whose body holds a nested WHILE node for CG; the conditions are
// set by the finishing kernels.  Every loop is capped (max_iter, cg_max,
// max_trials), so the graph always terminates.
//
// Vectors are float64; the row passes see them rounded to float32 (staged in
// shared memory).  Dot products and norms are float64; the per-CTA partials of
// a row pass are summed in a fixed order with compensated float32 sums.
#include <chrono>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>
#include <nvtx3/nvToolsExt.h>

#include "plan.h"

namespace rpt {
namespace {

namespace cg = cooperative_groups;
constexpr int VT = kVecThreads;

__device__ __forceinline__ double clampd(double v, double lo, double hi) {
  return fmin(fmax(v, lo), hi);
}

// Compensated sum, in the slot list's fixed order, of scenario s's row-pass
// partials at column j; list holds the cnt slots of scenario s (in global or
// shared memory, written before this kernel started).  Sixteen slots at a
// time: all loads of a batch are issued before the (order-preserving) sums
// consume them.
__device__ __forceinline__ double sum_partials_of(const DevPlan& P, const float* __restrict__ part, int s, int j,
                                                  const int* list, int cnt) {
  constexpr int kB = 16;
  if (P.acc64) {
    // bundled path: 64-bit fixed-point partials, summed exactly (every partial
    // and every sum stays below 2^62 in magnitude), then scaled by 2^-fexp[s]
    // and by the column scale of quantised values
    const long long* pl = reinterpret_cast<const long long*>(part);
    long long sum = 0;
    int k = 0;
    for (; k + kB <= cnt; k += kB) {
      long long v[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) v[u] = __ldcg(pl + (size_t)list[k + u] * P.n_pad + j);
#pragma unroll
      for (int u = 0; u < kB; ++u) sum += v[u];
    }
    for (; k < cnt; ++k) sum += __ldcg(pl + (size_t)list[k] * P.n_pad + j);
    const int fe = __ldcg(&P.fexp[s]);
    if (fe == kFexpNaN) return __longlong_as_double(0x7ff8000000000000ll);
    double r = ldexp((double)sum, -fe);
    if (P.colscale) r *= (double)P.colscale[(size_t)s * P.n_pad + j];
    return r;
  }
  float sum = 0.f, c = 0.f;
  int k = 0;
  for (; k + kB <= cnt; k += kB) {
    float v[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) v[u] = __ldcg(part + (size_t)list[k + u] * P.n_pad + j);
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      float t, e;
      two_sum(sum, v[u], t, e);
      sum = t;
      c += e;
    }
  }
  for (; k < cnt; ++k) {
    const float v = __ldcg(part + (size_t)list[k] * P.n_pad + j);
    float t, e;
    two_sum(sum, v, t, e);
    sum = t;
    c += e;
  }
  return (double)sum + (double)c;
}

__device__ __forceinline__ double sum_partials(const DevPlan& P, const float* __restrict__ part, int s, int j) {
  return sum_partials_of(P, part, s, j, P.slot_list + (size_t)s * P.slot_cap, __ldcg(&P.slot_count[s]));
}

// Objective of the last objective pass: sum over scenarios (fixed order).
__device__ __forceinline__ double objective_sum(const DevPlan& P) {
  double f = 0.0;
  for (int s = 0; s < P.N; ++s) f += __ldcg(&P.objs[s]);
  return f;
}

// Last-block-done: every block calls it once (all threads); returns true in the
// block that arrives last; that block also resets the counter.
__device__ __forceinline__ bool last_block(unsigned int* counter, unsigned int total) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(counter, 1u);
    am_last = (prev + 1u == total);
    if (am_last) *counter = 0u;
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// In the last block: S[k] = sum over b < count of buf[b * stride + off + k], the
// whole block taking entries b = tid, tid + blockDim, ... then a block reduction
// (a fixed order for a given launch shape).  Result valid in thread 0.
template <int K>
__device__ __forceinline__ void last_block_sums(const double* buf, int count, int stride, int off, double (&S)[K],
                                                double* sh /* [K*32] */) {
#pragma unroll
  for (int k = 0; k < K; ++k) S[k] = 0.0;
  for (int b = threadIdx.x; b < count; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) S[k] += __ldcg(&buf[(size_t)b * stride + off + k]);
  block_sum_d<K>(S, sh);
}

// In warp 0 of a block: the sums over c < count of buf[c * stride + off] and
// buf[c * stride + off + 1], lane l taking c = l, l + 32, ... (independent loads
// in flight instead of a serial chain) and a butterfly across the warp: a fixed
// order for a given count.  Results valid in every lane of warp 0.
__device__ __forceinline__ void warp_sums2(const double* buf, int count, int stride, int off, double& a, double& b) {
  a = 0.0;
  b = 0.0;
  for (int c = threadIdx.x; c < count; c += 32) {
    a += __ldcg(&buf[(size_t)c * stride + off]);
    b += __ldcg(&buf[(size_t)c * stride + off + 1]);
  }
  a = warp_sum_d(a);
  b = warp_sum_d(b);
}

__device__ __forceinline__ void set_cond(unsigned long long h, int use, int value) {
  if (use) cudaGraphSetConditional((cudaGraphConditionalHandle)h, value ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// ADMM-BB kernels
// ---------------------------------------------------------------------------

// grid (nchunk, N).  Initial state: z = P(z0), y = y0, x_s = z, d_prev = 0;
// with resume: keep (z, x, y), d_prev = x - z.  Stages float32 x for the first
// residual pass; sets the CG preconditioner for this rho.  z0, z, lb, ub hold
// one n-vector per group (scenario s belongs to group s / Ns).
__global__ void k_admm_init(DevPlan P, const Ctl* __restrict__ C, const double* __restrict__ z0,
                            const double* __restrict__ y0, int has_z0, int has_y0, int resume,
                            const double* __restrict__ lb, const double* __restrict__ ub,
                            const float* __restrict__ diag, double* dinv, double* x, double* y, double* z,
                            double* dprev, float* v32) {
  const int s = blockIdx.y, gi = s / P.Ns, j = blockIdx.x * VT + threadIdx.x;
  if (j < P.n) {
    const size_t o = (size_t)s * P.n + j, zo = (size_t)gi * P.n + j;
    // Jacobi preconditioner of B_s = A~_s^T A~_s + (rho/2) I, or the identity
    dinv[o] = C->precond ? 1.0 / ((double)diag[o] + 0.5 * C->g[gi].rho) : 1.0;
    if (!resume) {
      const double zj = clampd(has_z0 ? z0[zo] : 0.0, lb[zo], ub[zo]);
      x[o] = zj;
      y[o] = has_y0 ? y0[o] : 0.0;
      dprev[o] = 0.0;
      if (s % P.Ns == 0) z[zo] = zj;
      v32[(size_t)s * P.n_pad + j] = (float)zj;
    } else {
      dprev[o] = x[o] - z[zo];
      v32[(size_t)s * P.n_pad + j] = (float)x[o];
    }
  } else if (j < P.n_pad) {
    v32[(size_t)s * P.n_pad + j] = 0.f;
  }
}

// Subproblem solves (App. A: B_s x_s = c_s) by preconditioned conjugate
// gradients in the Chronopoulos-Gear arrangement: each step applies B_s once,
// to u = M^{-1} r (M = I, or the Jacobi diagonal of B_s), so the vector a row
// pass needs is known before the step's reductions; both inner products of a
// step are reduced explicitly (no algebraic norm updates).
//   w = B u;  delta = (w, u);  beta = gamma / gamma_prev;
//   alpha = gamma / (delta - beta gamma / alpha_prev)          (first step: gamma / delta)
//   p = u + beta p;  q = w + beta q;  x += alpha p;  r -= alpha q;  u = M^{-1} r
//   gamma = (r, u);  stop scenario s when ||r|| <= tol_s.

// grid (nchunk, N).  r = -g - (rho/2)(x - z) - y/2 with g from the residual pass
// (this is c_s - B_s x_s); u = M^{-1} r; per-scenario gamma, ||r||, tolerance, activity.
// Scenarios of a group that has stopped are left as they are and inactive.
__global__ void k_cg_init(DevPlan P, Ctl* C, const float* __restrict__ partial,
                          const double* __restrict__ x, const double* __restrict__ y,
                          const double* __restrict__ z, const double* __restrict__ dinv, double* r,
                          double* u, float* v32, double* dots, int nchunk, double* gam, double* tol,
                          double* r0n, int* act, int* cgi, unsigned int* cnt_s, unsigned long long hcg,
                          int use_cond) {
  __shared__ double sh[2 * 32];
  const int s = blockIdx.y, gi = s / P.Ns, j = blockIdx.x * VT + threadIdx.x;
  const Grp& G = C->g[gi];
  const bool live = !G.done;
  const double rho = G.rho;
  double v[2] = {0.0, 0.0};
  if (live && j < P.n) {
    const size_t o = (size_t)s * P.n + j;
    const double gj = sum_partials(P, partial, s, j);
    const double ri = -gj - 0.5 * rho * (x[o] - z[(size_t)gi * P.n + j]) - 0.5 * y[o];
    const double ui = dinv[o] * ri;
    r[o] = ri;
    u[o] = ui;
    v32[(size_t)s * P.n_pad + j] = (float)ui;
    v[0] = ri * ui;
    v[1] = ri * ri;
  } else if (live && j < P.n_pad) {
    v32[(size_t)s * P.n_pad + j] = 0.f;
  }
  block_sum_d<2>(v, sh);
  if (threadIdx.x == 0) {
    double* d = &dots[((size_t)s * nchunk + blockIdx.x) * 4];
    d[0] = v[0];
    d[1] = v[1];
  }
  if (!last_block(&cnt_s[s], gridDim.x)) return;
  double g = 0.0, rr = 0.0;
  if (threadIdx.x < 32) warp_sums2(dots + (size_t)s * nchunk * 4, nchunk, 4, 0, g, rr);
  if (threadIdx.x == 0 && !live) {
    cgi[s] = 0;
    act[s] = 0;
  } else if (threadIdx.x == 0) {
    const double rn = sqrt(rr);
    double t;
    if (G.first) {
      r0n[s] = rn;
      t = C->cg_eta0 * rn;
    } else {
      // theta-rule, with the floor capped at the accuracy Eq. 9 needs (a summed
      // subproblem error of eps_prim): a floor above it stalls the iteration
      const double sN = sqrt((double)P.Ns);
      t = fmax(C->cg_theta * 0.5 * rho * fmax(G.r_prim, G.eps_prim) / sN,
               fmin(C->cg_floor * __ldcg(&r0n[s]), 0.5 * rho * G.eps_prim / sN));
    }
    gam[s] = g;
    tol[s] = t;
    cgi[s] = 0;
    act[s] = (rn > t && g > 0.0 && C->cg_max > 0) ? 1 : 0;
  }
  if (!last_block(&C->cnt_init, P.N)) return;
  if (threadIdx.x < 32) {
    int any = 0;
    for (int k = threadIdx.x; k < P.N; k += 32) any += __ldcg(&act[k]);
    any = __reduce_add_sync(0xffffffffu, any);
    if (threadIdx.x != 0) return;
    C->cg_any = any;
    C->kcg = 0;
    C->passes += 1;
    set_cond(hcg, use_cond, any > 0);
  }
}

// grid (kCgCluster, N) in clusters of kCgCluster CTAs along x; the cluster of
// scenario s makes one whole CG step after the operator pass:
//   w = B u = (row-pass partials) + (rho/2) u;  delta = (w, u);  beta and alpha;
//   p = u + beta p;  q = w + beta q;  x += alpha p;  r -= alpha q;  u = M^{-1} r (staged);
//   gamma = (r, u), ||r||; activity; loop condition.
// A CTA has kCgSub rows of kVecThreads threads; column chunk c (kVecThreads
// columns) belongs to the cluster's CTA c mod kCgCluster, to its thread row
// (c / kCgCluster) mod kCgSub and to its round c / (kCgCluster kCgSub), column
// j to thread j mod kVecThreads of that row, and a thread takes its rounds in
// increasing order; each CTA's sums are block reductions and the cluster's the
// CTAs' sums added in rank order through distributed shared memory.  The order
// depends on the column index only, not on n: the wider spot range of a
// batched plan adds exact zeros.  w and u stay in registers between the two
// halves; the cluster barriers are hardware barriers.
constexpr int kCgCluster = 8;
constexpr int kCgSub = 4;
constexpr int kCgThreads = kCgSub * kVecThreads;
constexpr int kCgChunks = (RPT_MAX_SPOTS + kCgThreads * kCgCluster - 1) / (kCgThreads * kCgCluster);
constexpr int kErrCgCluster = 16;   // error word: the CG step ran without its cluster
constexpr int kCgListCap = 2048;    // slot lists up to this length are read from shared memory

__global__ void __cluster_dims__(kCgCluster, 1, 1) __launch_bounds__(kCgThreads, 1)
k_cg_step(DevPlan P, Ctl* C, double* x, double* r, double* u, double* p, double* q,
          const float* __restrict__ partial, const double* __restrict__ dinv, float* v32, double* gam,
          double* gprev, double* aprev, const double* __restrict__ tol, int* act, int* act_next, int* cgi,
          int* cgcnt, unsigned long long hcg, int use_cond) {
  __shared__ double sh[2 * 32];
  __shared__ double cl_part[3];   // this CTA's parts of delta, gamma and ||r||^2 (read by the cluster)
  __shared__ double ab[2];
  __shared__ int s_list[kCgListCap];
  cg::cluster_group cl = cg::this_cluster();
  if (cl.num_blocks() != kCgCluster) {   // never expected: report it and touch nothing
    if (threadIdx.x == 0) atomicExch(P.err, kErrCgCluster);
    return;
  }
  const int s = blockIdx.y, rank = (int)cl.block_rank();
  const int sub = threadIdx.x / VT, col = threadIdx.x % VT;
  if (__ldcg(&act[s]) == 0) return;      // the same answer in every CTA of the cluster
  const int any = __ldcg(&C->cg_any);
  const bool first = __ldcg(&cgi[s]) == 0;
  const double hr = 0.5 * C->g[s / P.Ns].rho;
  // the scenario's slot list into shared memory, and the step's scalars, all
  // loads in flight together (this kernel's rank 0 rewrites the scalars only
  // after every CTA of the cluster has passed its second barrier)
  const int cnt = __ldcg(&P.slot_count[s]);
  const int* glist = P.slot_list + (size_t)s * P.slot_cap;
  const int* list = cnt <= kCgListCap ? s_list : glist;
  if (cnt <= kCgListCap)
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) s_list[k] = __ldcg(&glist[k]);
  double g_s = 0.0, gp_s = 0.0, ap_s = 0.0, tol_s = 0.0;
  if (threadIdx.x == 0) {
    g_s = __ldcg(&gam[s]);
    gp_s = __ldcg(&gprev[s]);
    ap_s = __ldcg(&aprev[s]);
    tol_s = __ldcg(&tol[s]);
  }
  __syncthreads();
  double uv[kCgChunks], wv[kCgChunks];
  // the second half's operands of the first round are loaded now, so that
  // their latency overlaps the first half's sums and barriers
  const int j0 = (sub * kCgCluster + rank) * VT + col;
  const size_t o0 = (size_t)s * P.n + j0;
  double p0 = 0.0, q0 = 0.0, r0 = 0.0, d0 = 0.0;
  if (j0 < P.n) {
    p0 = p[o0];
    q0 = q[o0];
    r0 = r[o0];
    d0 = dinv[o0];
  }
  double dl[1] = {0.0};
#pragma unroll
  for (int t = 0; t < kCgChunks; ++t) {
    const int j = ((t * kCgSub + sub) * kCgCluster + rank) * VT + col;
    uv[t] = 0.0;
    wv[t] = 0.0;
    if (j < P.n) {
      const size_t o = (size_t)s * P.n + j;
      uv[t] = u[o];
      wv[t] = sum_partials_of(P, partial, s, j, list, cnt) + hr * uv[t];
      dl[0] += wv[t] * uv[t];
    }
  }
  block_sum_d<1>(dl, sh);
  if (threadIdx.x == 0) cl_part[0] = dl[0];
  cl.sync();
  if (threadIdx.x == 0) {
    double parts[kCgCluster];
#pragma unroll
    for (int k = 0; k < kCgCluster; ++k) parts[k] = *cl.map_shared_rank(&cl_part[0], k);
    double delta = 0.0;
#pragma unroll
    for (int k = 0; k < kCgCluster; ++k) delta += parts[k];
    const double b = first ? 0.0 : g_s / gp_s;
    const double den = first ? delta : delta - b * g_s / ap_s;
    ab[0] = (den > 0.0 && isfinite(den) && isfinite(b)) ? g_s / den : 0.0;
    ab[1] = b;
  }
  __syncthreads();
  const double a = ab[0], b = ab[1];
  double v[2] = {0.0, 0.0};
#pragma unroll
  for (int t = 0; t < kCgChunks; ++t) {
    const int j = ((t * kCgSub + sub) * kCgCluster + rank) * VT + col;
    if (j < P.n) {
      const size_t o = (size_t)s * P.n + j;
      const double pj = first ? uv[t] : fma(b, t == 0 ? p0 : p[o], uv[t]);
      const double qj = first ? wv[t] : fma(b, t == 0 ? q0 : q[o], wv[t]);
      p[o] = pj;
      q[o] = qj;
      x[o] = fma(a, pj, x[o]);
      const double rj = fma(-a, qj, t == 0 ? r0 : r[o]);
      const double uj = (t == 0 ? d0 : dinv[o]) * rj;
      r[o] = rj;
      u[o] = uj;
      v32[(size_t)s * P.n_pad + j] = (float)uj;
      v[0] += rj * uj;
      v[1] += rj * rj;
    }
  }
  block_sum_d<2>(v, sh);
  if (threadIdx.x == 0) {
    cl_part[1] = v[0];
    cl_part[2] = v[1];
  }
  cl.sync();
  if (rank == 0 && threadIdx.x == 0) {
    double pg[kCgCluster], pr[kCgCluster];
#pragma unroll
    for (int k = 0; k < kCgCluster; ++k) {
      pg[k] = *cl.map_shared_rank(&cl_part[1], k);
      pr[k] = *cl.map_shared_rank(&cl_part[2], k);
    }
    double g = 0.0, rr = 0.0;
#pragma unroll
    for (int k = 0; k < kCgCluster; ++k) {
      g += pg[k];
      rr += pr[k];
    }
    gprev[s] = g_s;
    aprev[s] = a;
    gam[s] = g;
    cgi[s] += 1;
    cgcnt[s] += 1;
    act_next[s] = (a > 0.0 && g > 0.0 && sqrt(rr) > tol_s) ? 1 : 0;
  }
  cl.sync();   // every CTA's shared memory stays until rank 0 has read it
  if (rank != 0) return;
  // rank 0 of every stepping scenario; the last to arrive ends the step
  if (!last_block(&C->cnt_upd, (unsigned int)any) || threadIdx.x >= 32) return;
  // warp 0: the scenarios of this step (lane l takes l, l + 32, ...) count one CG
  // step each and take their next activity
  int was = 0, na = 0;
  for (int k = threadIdx.x; k < P.N; k += 32) {
    const int ak = __ldcg(&act[k]), nx = __ldcg(&act_next[k]);   // both loads in flight
    if (ak) {
      ++was;
      atomicAdd(reinterpret_cast<unsigned long long*>(&C->g[k / P.Ns].cg), 1ull);
      act[k] = nx;
      na += nx;
    }
  }
  was = __reduce_add_sync(0xffffffffu, was);
  na = __reduce_add_sync(0xffffffffu, na);
  if (threadIdx.x == 0) {
    C->cg_total += was;
    C->cg_any = na;
    C->kcg += 1;
    C->cg_steps += 1;
    C->passes += 1;
    set_cond(hcg, use_cond, na > 0 && C->kcg < C->cg_max);
  }
}

// grid (nchunk, G).  Per group: z_new = P_box(mean_s(x_s + y_s/rho)) [std] or
// P_box(mean_s x_s) [lit] over the group's scenarios; ||z_new||^2, ||z_new - z||^2.
__global__ void k_admm_z(DevPlan P, Ctl* C, const double* __restrict__ x, const double* __restrict__ y,
                         const double* __restrict__ z, double* znew, const double* __restrict__ lb,
                         const double* __restrict__ ub, double* vpart, int nchunk) {
  __shared__ double sh[2 * 32];
  const int gi = blockIdx.y, j = blockIdx.x * VT + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (!C->g[gi].done && j < P.n) {
    const double ir = C->g[gi].inv_rho;
    const bool std_form = (C->z_mode == 0);
    const size_t zo = (size_t)gi * P.n + j;
    double acc = 0.0;
    for (int s = gi * P.Ns; s < (gi + 1) * P.Ns; ++s) {
      const size_t o = (size_t)s * P.n + j;
      acc += std_form ? fma(y[o], ir, x[o]) : x[o];
    }
    const double zn = clampd(acc / (double)P.Ns, lb[zo], ub[zo]);
    znew[zo] = zn;
    const double dz = zn - z[zo];
    v[0] = zn * zn;
    v[1] = dz * dz;
  }
  block_sum_d<2>(v, sh);
  if (threadIdx.x == 0) {
    vpart[((size_t)gi * nchunk + blockIdx.x) * 8 + 0] = v[0];
    vpart[((size_t)gi * nchunk + blockIdx.x) * 8 + 1] = v[1];
  }
  if (!last_block(&C->cnt_z, gridDim.x * gridDim.y)) return;
  for (int g = 0; g < P.G; ++g) {
    double S2[2];
    last_block_sums<2>(vpart + (size_t)g * nchunk * 8, nchunk, 8, 0, S2, sh);
    if (threadIdx.x == 0 && !C->g[g].done) {
      C->g[g].sz2 = S2[0];
      C->g[g].dz2 = S2[1];
    }
  }
}

// grid (nchunk, N).  d = x - z_new; BB sums dd'd_prev and ||dd||^2; ||d||^2, ||x||^2.
// Last block, per group: BB step (Eq. 8), r_prim, r_dual, eps_prim (Eq. 9).
// vpart: the first G * nchunk entries belong to k_admm_z, then one per block.
__global__ void k_admm_d(DevPlan P, Ctl* C, const double* __restrict__ x, const double* __restrict__ z,
                         const double* __restrict__ znew, const double* __restrict__ dprev, double* d,
                         double* vpart, int nchunk) {
  __shared__ double sh[5 * 32];
  const int s = blockIdx.y, gi = s / P.Ns, j = blockIdx.x * VT + threadIdx.x;
  const int con = C->con_on;
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (!C->g[gi].done && j < P.n) {
    const size_t o = (size_t)s * P.n + j, zo = (size_t)gi * P.n + j;
    const double xj = x[o];
    const double dj = xj - znew[zo];
    const double dp = dprev[o];
    const double dd = dj - dp;
    d[o] = dj;
    v[0] = dd * dp;
    v[1] = dd * dd;
    v[2] = dj * dj;
    v[3] = xj * xj;
    if (con) {   // dual residual with the dose blocks: rho (z - z_prev) + sigma G_s'(v_s - v_s_prev)
      const double rd = C->g[gi].rho * (znew[zo] - z[zo]) + C->con_q[o];
      v[4] = rd * rd;
    }
  }
  block_sum_d<5>(v, sh);
  const size_t base = (size_t)P.G * nchunk;
  const int blk = s * nchunk + blockIdx.x;
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) vpart[(base + blk) * 8 + k] = v[k];
    vpart[(base + blk) * 8 + 5] = v[4];
  }
  if (!last_block(&C->cnt_d, gridDim.x * gridDim.y)) return;
  const int per_group = P.Ns * nchunk;   // blocks of one group, consecutive
  for (int g = 0; g < P.G; ++g) {
    Grp& G = C->g[g];
    if (G.done) continue;   // the same for every thread of the block
    double S[4], SC[1];
    last_block_sums<4>(vpart + (base + (size_t)g * per_group) * 8, per_group, 8, 0, S, sh);
    last_block_sums<1>(vpart + (base + (size_t)g * per_group) * 8, per_group, 8, 5, SC, sh);
    const double rho = G.rho;
    const bool use_bb = C->bb_mode != 2 && G.have_prev;
    if (C->bb_scen) {
      // Eq. 8 on scenario s's own blocks: its partial sums in chunk order, and
      // dy_s = step_s d_prev_s with step_s the scenario's last dual step
      for (int s = g * P.Ns + threadIdx.x; s < (g + 1) * P.Ns; s += blockDim.x) {
        const double* vp = vpart + (base + (size_t)s * nchunk) * 8;
        double a = 0.0, b = 0.0;
        for (int c = 0; c < nchunk; ++c) {
          a += __ldcg(&vp[(size_t)c * 8 + 0]);
          b += __ldcg(&vp[(size_t)c * 8 + 1]);
        }
        double st = rho;
        if (use_bb && b > 0.0) {
          const double bb = -C->step_s[s] * a / b;
          if (isfinite(bb) && bb > 0.0) {
            st = bb;
            if (C->bb_mode == 1) st = fmin(fmax(st, rho / C->bb_kappa), C->bb_kappa * rho);
          }
        }
        C->step_s[s] = st;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double step = rho;
      if (C->bb_scen) {
        double acc = 0.0;
        for (int s = g * P.Ns; s < (g + 1) * P.Ns; ++s) acc += C->step_s[s];
        step = acc / (double)P.Ns;
      } else if (use_bb && S[1] > 0.0) {
        const double bb = -G.step_prev * S[0] / S[1];
        if (isfinite(bb) && bb > 0.0) {
          step = bb;
          if (C->bb_mode == 1) step = fmin(fmax(step, rho / C->bb_kappa), C->bb_kappa * rho);
        }
      }
      const double sN = sqrt((double)P.Ns);
      G.step = step;
      if (con) {
        // Eq. 9 extended to both blocks: r_prim over [x_s - z; G_s x_s - v_s],
        // eps_prim over [x_s; G_s x_s] and [z (N times); v_s]
        const double* cs = C->con_sums;
        G.r_prim = sqrt(S[2] + cs[0]);
        G.r_dual = sqrt(SC[0]);
        G.eps_prim = C->eps_abs * sqrt(G.nn + C->con_K) +
                     C->eps_rel * fmax(sqrt(S[3] + cs[1]), sqrt((double)P.Ns * G.sz2 + cs[2]));
      } else {
        G.r_prim = sqrt(S[2]);
        G.r_dual = sN * rho * sqrt(G.dz2);
        G.eps_prim = C->eps_abs * sqrt(G.nn) + C->eps_rel * fmax(sqrt(S[3]), sN * sqrt(G.sz2));
      }
    }
    __syncthreads();
  }
}

// grid (nchunk, N).  y += step d (Eq. 7); z <- z_new; d_prev <- d; stage x and z.
// Last block, per group: eps_dual and the stop test of Eq. 9; then the activity
// of every scenario and the next iteration's condition (all groups stopped, or
// the iteration cap).
__global__ void k_admm_y(DevPlan P, Ctl* C, const double* __restrict__ x, double* y, double* z,
                         const double* __restrict__ znew, const double* __restrict__ d, double* dprev,
                         float* v32, float* vz32, double* vpart, int nchunk, unsigned long long hadmm,
                         int use_cond) {
  __shared__ double sh[32];
  const int s = blockIdx.y, gi = s / P.Ns, j = blockIdx.x * VT + threadIdx.x;
  const bool live = !C->g[gi].done;
  const double step = C->bb_scen ? __ldcg(&C->step_s[s]) : __ldcg(&C->g[gi].step);
  double v[1] = {0.0};
  if (live && j < P.n) {
    const size_t o = (size_t)s * P.n + j, zo = (size_t)gi * P.n + j;
    const double dj = d[o];
    const double yn = fma(step, dj, y[o]);
    y[o] = yn;
    dprev[o] = dj;
    v32[(size_t)s * P.n_pad + j] = (float)x[o];
    const double ye = C->con_on ? yn + C->con_t[o] : yn;   // with dose blocks: y_s + G_s' mu_s
    v[0] = ye * ye;
    if (s % P.Ns == 0) {
      const double zn = znew[zo];
      z[zo] = zn;
      if (P.G == 1) vz32[j] = (float)zn;
    }
  } else if (P.G == 1 && s == 0 && j < P.n_pad) {
    vz32[j] = 0.f;
  }
  block_sum_d<1>(v, sh);
  const size_t base = (size_t)P.G * nchunk;
  const int blk = s * nchunk + blockIdx.x;
  if (threadIdx.x == 0) vpart[(base + blk) * 8 + 4] = v[0];
  if (!last_block(&C->cnt_y, gridDim.x * gridDim.y)) return;
  const int per_group = P.Ns * nchunk;
  for (int g = 0; g < P.G; ++g) {
    Grp& G = C->g[g];
    if (G.done) continue;   // the same for every thread of the block
    double SY[1];
    last_block_sums<1>(vpart + (base + (size_t)g * per_group) * 8, per_group, 8, 4, SY, sh);
    if (threadIdx.x == 0) {
      const double Y = SY[0];
      G.eps_dual = C->eps_abs * sqrt(G.nn) + C->eps_rel * sqrt(Y);
      const int conv = (G.r_prim <= G.eps_prim) && (G.r_dual <= G.eps_dual);
      G.k += 1;
      G.have_prev = 1;
      G.step_prev = G.step;
      G.first = 0;
      if (!(isfinite(G.r_prim) && isfinite(G.r_dual) && isfinite(Y))) G.diverged = 1;
      G.status = conv;
      // with the objective test (one group only) k_admm_obj decides the stop
      if (!C->use_obj) G.done = conv || G.diverged || G.k >= C->max_iter;
    }
    __syncthreads();
  }
  if (P.G > 1 && C->uact)
    for (int u = threadIdx.x; u < P.N; u += blockDim.x) C->uact[u] = C->g[u / P.Ns].done ? 0 : 1;
  if (threadIdx.x == 0) {
    const Grp& G0 = C->g[0];
    if (C->trace_on && C->k < C->trace_cap) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (C->k == 0) C->t_start = t;
      double* e = C->trace + (size_t)C->k * kTraceFields;
      e[0] = (double)(C->k + 1);
      e[1] = 1e-9 * (double)(t - C->t_start);
      e[2] = G0.r_prim;
      e[3] = G0.r_dual;
      e[4] = G0.eps_prim;
      e[5] = G0.eps_dual;
      e[6] = G0.step;
      e[7] = (double)C->cg_total;
    }
    C->k += 1;
    int all_done = 1, all_conv = 1, any_div = 0;
    for (int g = 0; g < P.G; ++g) {
      all_done &= C->g[g].done;
      all_conv &= C->g[g].status;
      any_div |= C->g[g].diverged;
    }
    C->status = all_conv;
    C->diverged = any_div;
    if (!C->use_obj) {
      C->stop = all_done || C->k >= C->max_iter;
      set_cond(hadmm, use_cond, !C->stop);
    }
  }
}

// <<<1, 32>>>.  Objective of z (after a kObj row pass; plans of one group only):
// optional relative-change test AND-ed with Eq. 9 (Sec. 2.3), or, with an
// objective target, f(z) <= target alone.
__global__ void k_admm_obj(DevPlan P, Ctl* C, unsigned long long hadmm, int use_cond) {
  if (threadIdx.x == 0) {
    Grp& G = C->g[0];
    const double f = objective_sum(P) + C->const_term;
    const int conv_obj = fabs(C->f_prev - f) <= C->tol_obj * fmax(fabs(f), 1e-300);
    C->f_prev = f;
    C->f_cur = f;
    C->passes += 1;
    G.status = C->f_goal > 0.0 ? (f <= C->f_goal) : (G.status && conv_obj);
    G.done = G.status || G.diverged || G.k >= C->max_iter;
    C->status = G.status;
    C->stop = G.done || C->k >= C->max_iter;
    set_cond(hadmm, use_cond, !C->stop);
  }
}

// <<<1, 32>>>.  f = sum of block objectives + constant; per group the same over
// the group's scenarios.
__global__ void k_final_obj(DevPlan P, Ctl* C) {
  if (threadIdx.x == 0) {
    C->f_cur = objective_sum(P) + C->const_term;
    for (int g = 0; g < P.G; ++g) {
      double f = C->g[g].cst;
      for (int s = g * P.Ns; s < (g + 1) * P.Ns; ++s) f += __ldcg(&P.objs[s]);
      C->g[g].f = f;
    }
    C->passes += 1;
  }
}

// grid (nchunk, N).  Stage every scenario's copy of its group's z (the final
// objective pass of a batched plan, where the groups' z differ).
__global__ void k_stage_z(DevPlan P, const double* __restrict__ z, float* v32) {
  const int s = blockIdx.y, j = blockIdx.x * VT + threadIdx.x;
  if (j < P.n) v32[(size_t)s * P.n_pad + j] = (float)z[(size_t)(s / P.Ns) * P.n + j];
  else if (j < P.n_pad) v32[(size_t)s * P.n_pad + j] = 0.f;
}

// ---------------------------------------------------------------------------
// PGD kernels (Sec. 2.1)
// ---------------------------------------------------------------------------

// grid (nchunk).  x = P(x0); stage float32 x (shared by all scenarios).
__global__ void k_pgd_init(DevPlan P, const double* __restrict__ x0, int has_x0,
                           const double* __restrict__ lb, const double* __restrict__ ub, double* x,
                           float* vz32) {
  const int j = blockIdx.x * VT + threadIdx.x;
  if (j < P.n) {
    const double xj = clampd(has_x0 ? x0[j] : 0.0, lb[j], ub[j]);
    x[j] = xj;
    vz32[j] = (float)xj;
  } else if (j < P.n_pad) {
    vz32[j] = 0.f;
  }
}

// grid (nchunk).  g = 2 sum_s A~_s^T (A~_s x - p~) (Eq. 4 summed over s) from a kResid
// pass over all scenarios; f(x); start the Armijo trials at t = alpha.
__global__ void k_pgd_grad(DevPlan P, Ctl* C, const float* __restrict__ partial,
                           double* g, unsigned long long htrial, int use_cond) {
  const int j = blockIdx.x * VT + threadIdx.x;
  if (j < P.n) {
    double gj = 0.0;
    for (int s = 0; s < P.N; ++s) gj += sum_partials(P, partial, s, j);
    g[j] = 2.0 * gj;
  }
  if (!last_block(&C->cnt_pg, gridDim.x)) return;
  if (threadIdx.x == 0) {
    C->fx = objective_sum(P) + C->const_term;
    C->t = C->alpha;
    C->trial = 0;
    C->accepted = 0;
    C->passes += 1;
    set_cond(htrial, use_cond, 1);
  }
}

// grid (nchunk).  Trial point x_t = P(x - t g), staged; g'(x_t - x).
__global__ void k_pgd_trial(DevPlan P, Ctl* C, const double* __restrict__ x,
                            const double* __restrict__ g, const double* __restrict__ lb,
                            const double* __restrict__ ub, double* xt, float* vt32, double* vpart) {
  __shared__ double sh[32];
  const int j = blockIdx.x * VT + threadIdx.x;
  const double t = __ldcg(&C->t);
  double v[1] = {0.0};
  if (j < P.n) {
    const double xj = x[j], gj = g[j];
    const double xn = clampd(xj - t * gj, lb[j], ub[j]);
    xt[j] = xn;
    vt32[j] = (float)xn;
    v[0] = gj * (xn - xj);
  } else if (j < P.n_pad) {
    vt32[j] = 0.f;
  }
  block_sum_d<1>(v, sh);
  if (threadIdx.x == 0) vpart[blockIdx.x * 8] = v[0];
  if (!last_block(&C->cnt_pt, gridDim.x)) return;
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) a += __ldcg(&vpart[c * 8]);
    C->gd = a;
  }
}

// <<<1, 256>>>.  Sufficient-decrease test (Eq. 3 read as f(x_t) <= f(x) + beta g'(x_t - x)).
__global__ void k_pgd_accept(DevPlan P, Ctl* C, unsigned long long htrial, int use_cond) {
  if (threadIdx.x == 0) {
    const double ft = objective_sum(P) + C->const_term;
    C->ft = ft;
    C->trials_total += 1;
    C->passes += 1;
    int more = 0;
    if (ft <= C->fx + C->beta_a * C->gd) {
      C->accepted = 1;
    } else {
      C->t *= C->gamma;
      C->trial += 1;
      if (C->trial >= C->max_trials) C->failed = 1;
      else more = 1;
    }
    set_cond(htrial, use_cond, more);
  }
}

// grid (nchunk).  Accept x_t, stage it; stopping rule on the relative change of f.
__global__ void k_pgd_finish(DevPlan P, Ctl* C, double* x, const double* __restrict__ xt,
                             float* vz32, unsigned long long houter, int use_cond) {
  const int j = blockIdx.x * VT + threadIdx.x;
  const int acc = __ldcg(&C->accepted);
  if (acc && j < P.n) {
    const double xn = xt[j];
    x[j] = xn;
    vz32[j] = (float)xn;
  }
  if (!last_block(&C->cnt_red, gridDim.x)) return;
  if (threadIdx.x == 0) {
    int stop = 0;
    C->pouter += 1;
    if (acc) {
      const double fx = C->fx, ft = C->ft;
      const double rel = fabs(fx - ft) / fmax(fabs(fx), 1e-300);
      C->pk += 1;
      C->fx = ft;
      C->f_cur = ft;
      C->pstep = C->t;
      stop = (rel <= C->tol_df) || (C->f_target > 0.0 && ft <= C->f_target) ||
             (C->pk >= C->pgd_max_iter) || !isfinite(ft);
      if (!isfinite(ft)) C->diverged = 1;
      C->status = (rel <= C->tol_df) || (C->f_target > 0.0 && ft <= C->f_target);
    } else {
      stop = 1;
      C->f_cur = C->fx;
    }
    C->stop = stop;
    set_cond(houter, use_cond, !stop);
  }
}

// ---------------------------------------------------------------------------
// operator kernels
// ---------------------------------------------------------------------------

// grid (nchunk, N): out_s = partials of scenario s + half_rho * v_s.
__global__ void k_reduce_scen(DevPlan P, const float* __restrict__ partial,
                              const double* __restrict__ v, double half_rho, double* out) {
  const int s = blockIdx.y, j = blockIdx.x * VT + threadIdx.x;
  if (j >= P.n) return;
  const size_t o = (size_t)s * P.n + j;
  out[o] = sum_partials(P, partial, s, j) + half_rho * v[o];
}

// grid (nchunk, N).  out[s][j] = -(row-pass partials of scenario s)[j]; with the
// residual pass at v = 0 this is A~_s^T p~.
__global__ void k_neg_partials(DevPlan P, const float* __restrict__ partial, double* out) {
  const int s = blockIdx.y, j = blockIdx.x * VT + threadIdx.x;
  if (j >= P.n) return;
  out[(size_t)s * P.n + j] = -sum_partials(P, partial, s, j);
}

// Cached-factor x-update, part 1: c_s = A~_s^T p~ + (rho/2) z - y_s/2 as float
// (grid (nchunk, N)).
__global__ void k_chol_rhs(DevPlan P, const Ctl* __restrict__ C, const double* __restrict__ bchol,
                           const double* __restrict__ z, const double* __restrict__ y, float* c) {
  const int s = blockIdx.y, gi = s / P.Ns, j = blockIdx.x * VT + threadIdx.x;
  if (j >= P.n || C->g[gi].done) return;
  const size_t o = (size_t)s * P.n + j;
  c[(size_t)s * P.n_pad + j] = (float)(bchol[o] + 0.5 * C->g[gi].rho * z[(size_t)gi * P.n + j] - 0.5 * y[o]);
}

// Cached-factor x-update, part 2 (App. A): x_s = B_s^{-1} c_s.  grid (ceil(n /
// kCholRows), N), 256 threads: c_s staged in shared memory, each warp takes rows
// of B_s^{-1} (streamed once, evict-first) with four 16-byte loads in flight per
// lane, FP64 accumulation of FP32 products.
constexpr int kCholRows = 64;
__global__ void __launch_bounds__(256)
k_chol_x(DevPlan P, const Ctl* __restrict__ C, const float* __restrict__ binv, const float* __restrict__ c,
         double* x) {
  extern __shared__ float cbuf[];
  const int s = blockIdx.y, n = P.n;
  if (C->g[s / P.Ns].done) return;   // a stopped group keeps its x
  for (int j = threadIdx.x; j < n; j += blockDim.x) cbuf[j] = c[(size_t)s * P.n_pad + j];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float* Bs = binv + (size_t)s * n * n;
  const bool vec = (n & 3) == 0;
  for (int r = w; r < kCholRows; r += 8) {
    const int j = blockIdx.x * kCholRows + r;
    if (j >= n) break;
    const float* row = Bs + (size_t)j * n;
    double acc = 0.0;
    if (vec) {
      const float4* row4 = reinterpret_cast<const float4*>(row);
      const float4* c4 = reinterpret_cast<const float4*>(cbuf);
      const int nq = n >> 2;
      int k = lane;
      for (; k + 96 < nq; k += 128) {
        const float4 b0 = __ldcs(row4 + k), b1 = __ldcs(row4 + k + 32), b2 = __ldcs(row4 + k + 64),
                     b3 = __ldcs(row4 + k + 96);
        const float4 v0 = c4[k], v1 = c4[k + 32], v2 = c4[k + 64], v3 = c4[k + 96];
        float t = b0.x * v0.x + b0.y * v0.y + b0.z * v0.z + b0.w * v0.w;
        t += b1.x * v1.x + b1.y * v1.y + b1.z * v1.z + b1.w * v1.w;
        acc += (double)t;
        t = b2.x * v2.x + b2.y * v2.y + b2.z * v2.z + b2.w * v2.w;
        t += b3.x * v3.x + b3.y * v3.y + b3.z * v3.z + b3.w * v3.w;
        acc += (double)t;
      }
      for (; k < nq; k += 32) {
        const float4 b = __ldcs(row4 + k);
        const float4 v = c4[k];
        acc += (double)(b.x * v.x + b.y * v.y + b.z * v.z + b.w * v.w);
      }
    } else {
      for (int k = lane; k < n; k += 32) acc += (double)(__ldcs(row + k) * cbuf[k]);
    }
    acc = warp_sum_d(acc);
    if (lane == 0) x[(size_t)s * n + j] = acc;
  }
}

// grid (nchunk): out = scale * sum over all blocks.
__global__ void k_reduce_all(DevPlan P, const float* __restrict__ partial, double scale, double* out) {
  const int j = blockIdx.x * VT + threadIdx.x;
  if (j >= P.n) return;
  double v = 0.0;
  for (int s = 0; s < P.N; ++s) v += sum_partials(P, partial, s, j);
  out[j] = scale * v;
}

// ---------------------------------------------------------------------------
// host-side launch helpers: one code path that either launches into a stream
// or appends kernel nodes to a CUDA graph
// ---------------------------------------------------------------------------

struct Exec {
  cudaStream_t st = nullptr;       // stream mode
  cudaGraph_t g = nullptr;         // graph mode
  cudaGraphNode_t last = nullptr;
  cudaError_t err = cudaSuccess;

  bool graph() const { return g != nullptr; }

  void kernel(void* fn, dim3 grid, dim3 block, size_t smem, void** args) {
    if (err != cudaSuccess) return;
    if (!graph()) {
      err = cudaLaunchKernel(fn, grid, block, args, smem, st);
      return;
    }
    cudaKernelNodeParams kp{};
    kp.func = fn;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = (unsigned int)smem;
    kp.kernelParams = args;
    cudaGraphNode_t node;
    err = cudaGraphAddKernelNode(&node, g, last ? &last : nullptr, last ? 1 : 0, &kp);
    if (err == cudaSuccess) last = node;
  }

  // Append a WHILE node; returns an Exec that appends to its body.
  Exec while_body(cudaGraphConditionalHandle h) {
    Exec body;
    if (err != cudaSuccess) {
      body.err = err;
      return body;
    }
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    err = cudaGraphAddNode(&node, g, last ? &last : nullptr, nullptr, last ? 1 : 0, &np);
    if (err != cudaSuccess) {
      body.err = err;
      return body;
    }
    last = node;
    body.g = np.conditional.phGraph_out[0];
    return body;
  }
};

template <typename... A>
void launch(Exec& e, void (*fn)(A...), dim3 grid, dim3 block, size_t smem, A... args) {
  void* ptrs[] = {(void*)&args...};
  e.kernel((void*)fn, grid, block, smem, ptrs);
}

void rowpass(Exec& e, Plan* P, int mode, const float* v, int v_stride, const int* active,
             float* dose = nullptr) {
  const DevPlan& dp = P->dp;
  void* fn = rowpass_kernel(dp, mode);
  float* partial = P->partial;
  double* objp = P->objp;
  void* args[] = {(void*)&dp, (void*)&v, (void*)&v_stride, (void*)&active,
                  (void*)&partial, (void*)&objp, (void*)&dose};
  e.kernel(fn, dim3(dp.grid), dim3(rowpass_threads(dp)), rowpass_smem(dp, mode), args);
}

// ---- ADMM pieces ---------------------------------------------------------------

void admm_iteration_head(Exec& e, Plan* P, unsigned long long hcg, int uc) {
  const DevPlan& dp = P->dp;
  dim3 g2(P->nchunk, dp.N);
  // a batched plan skips the scenarios of problems that have stopped
  rowpass(e, P, kResid, P->v32, dp.n_pad, dp.G > 1 ? P->uact : nullptr);
  launch(e, k_cg_init, g2, dim3(VT), 0, dp, P->ctl, (const float*)P->partial, (const double*)P->x,
         (const double*)P->y, (const double*)P->z, (const double*)P->dinv, P->r, P->u, P->v32, P->dots,
         P->nchunk, P->gam, P->tol, P->r0n, P->act, P->cgi, P->cnt_s, hcg, uc);
}

void cg_body(Exec& e, Plan* P, unsigned long long hcg, int uc) {
  const DevPlan& dp = P->dp;
  rowpass(e, P, kNormal, P->v32, dp.n_pad, P->act);
  launch(e, k_cg_step, dim3(kCgCluster, dp.N), dim3(kCgThreads), 0, dp, P->ctl, P->x, P->r, P->u, P->p, P->q,
         (const float*)P->partial, (const double*)P->dinv, P->v32, P->gam, P->gprev, P->aprev,
         (const double*)P->tol, P->act, P->act_next, P->cgi, P->cgcnt, hcg, uc);
}

void admm_iteration_tail(Exec& e, Plan* P, int use_obj, unsigned long long hadmm, int uc, ConHook* con = nullptr) {
  const DevPlan& dp = P->dp;
  dim3 g1(P->nchunk, dp.G), g2(P->nchunk, dp.N);
  launch(e, k_admm_z, g1, dim3(VT), 0, dp, P->ctl, (const double*)P->x, (const double*)P->y,
         (const double*)P->z, P->znew, (const double*)P->lb, (const double*)P->ub, P->vpart, P->nchunk);
  if (con && e.err == cudaSuccess) e.err = con->after_z(P);
  launch(e, k_admm_d, g2, dim3(VT), 0, dp, P->ctl, (const double*)P->x, (const double*)P->z,
         (const double*)P->znew, (const double*)P->dprev, P->d, P->vpart, P->nchunk);
  launch(e, k_admm_y, g2, dim3(VT), 0, dp, P->ctl, (const double*)P->x, P->y, P->z,
         (const double*)P->znew, (const double*)P->d, P->dprev, P->v32, P->vz32, P->vpart, P->nchunk,
         hadmm, use_obj ? 0 : uc);
  if (use_obj) {
    rowpass(e, P, kObj, P->vz32, 0, nullptr);
    launch(e, k_admm_obj, dim3(1), dim3(32), 0, dp, P->ctl, hadmm, uc);
  }
}

void admm_tail_final(Exec& e, Plan* P) {
  if (P->dp.G > 1) {   // every group's own z
    launch(e, k_stage_z, dim3(P->nchunk, P->dp.N), dim3(VT), 0, P->dp, (const double*)P->z, P->v32);
    rowpass(e, P, kObj, P->v32, P->dp.n_pad, nullptr);
  } else {
    rowpass(e, P, kObj, P->vz32, 0, nullptr);
  }
  launch(e, k_final_obj, dim3(1), dim3(32), 0, P->dp, P->ctl);
}

void chol_iteration_head(Exec& e, Plan* P) {
  const DevPlan& dp = P->dp;
  launch(e, k_chol_rhs, dim3(P->nchunk, dp.N), dim3(VT), 0, dp, (const Ctl*)P->ctl, (const double*)P->bchol,
         (const double*)P->z, (const double*)P->y, P->v32);
  launch(e, k_chol_x, dim3((dp.n + kCholRows - 1) / kCholRows, dp.N), dim3(256), sizeof(float) * (size_t)dp.n_pad,
         dp, (const Ctl*)P->ctl, (const float*)P->binv, (const float*)P->v32, P->x);
}

cudaError_t build_admm_chol_graph(Plan* P, int use_obj) {
  cudaGraph_t g = nullptr;
  cudaError_t err = cudaGraphCreate(&g, 0);
  if (err != cudaSuccess) return err;
  cudaGraphConditionalHandle hadmm = 0;
  err = cudaGraphConditionalHandleCreate(&hadmm, g, 1, cudaGraphCondAssignDefault);
  Exec top;
  top.g = g;
  top.err = err;
  Exec body = top.while_body(hadmm);
  chol_iteration_head(body, P);
  admm_iteration_tail(body, P, use_obj, (unsigned long long)hadmm, 1);
  if (body.err != cudaSuccess) top.err = body.err;
  admm_tail_final(top, P);
  err = top.err;
  if (err == cudaSuccess) {
    if (P->admm_chol_exec) cudaGraphExecDestroy(P->admm_chol_exec);
    P->admm_chol_exec = nullptr;
    err = cudaGraphInstantiate(&P->admm_chol_exec, g, 0);
    if (err == cudaSuccess) P->admm_chol_exec_obj = use_obj;
  }
  cudaGraphDestroy(g);
  return err;
}

cudaError_t build_admm_graph(Plan* P, int use_obj, double* z0d, double* y0d) {
  (void)z0d;
  (void)y0d;
  cudaGraph_t g = nullptr;
  cudaError_t err = cudaGraphCreate(&g, 0);
  if (err != cudaSuccess) return err;
  cudaGraphConditionalHandle hadmm = 0, hcg = 0;
  err = cudaGraphConditionalHandleCreate(&hadmm, g, 1, cudaGraphCondAssignDefault);
  Exec top;
  top.g = g;
  top.err = err;
  Exec body = top.while_body(hadmm);
  if (body.err == cudaSuccess)
    body.err = cudaGraphConditionalHandleCreate(&hcg, body.g, 0, cudaGraphCondAssignDefault);
  admm_iteration_head(body, P, (unsigned long long)hcg, 1);
  Exec cg = body.while_body(hcg);
  cg_body(cg, P, (unsigned long long)hcg, 1);
  if (cg.err != cudaSuccess) body.err = cg.err;
  admm_iteration_tail(body, P, use_obj, (unsigned long long)hadmm, 1);
  if (body.err != cudaSuccess) top.err = body.err;
  admm_tail_final(top, P);
  err = top.err;
  if (err == cudaSuccess) {
    if (P->admm_exec) cudaGraphExecDestroy(P->admm_exec);
    P->admm_exec = nullptr;
    err = cudaGraphInstantiate(&P->admm_exec, g, 0);
    if (err == cudaSuccess) P->admm_exec_obj = use_obj;
  }
  cudaGraphDestroy(g);
  return err;
}

// ---- PGD pieces ------------------------------------------------------------------

void pgd_head(Exec& e, Plan* P, unsigned long long htrial, int uc) {
  const DevPlan& dp = P->dp;
  rowpass(e, P, kResid, P->vz32, 0, nullptr);
  launch(e, k_pgd_grad, dim3(P->nchunk), dim3(VT), 0, dp, P->ctl, (const float*)P->partial,
         P->g, htrial, uc);
}

void pgd_trial(Exec& e, Plan* P, unsigned long long htrial, int uc) {
  const DevPlan& dp = P->dp;
  launch(e, k_pgd_trial, dim3(P->nchunk), dim3(VT), 0, dp, P->ctl, (const double*)P->xp,
         (const double*)P->g, (const double*)P->lb, (const double*)P->ub, P->xt, P->v32, P->vpart);
  rowpass(e, P, kObj, P->v32, 0, nullptr);
  launch(e, k_pgd_accept, dim3(1), dim3(32), 0, dp, P->ctl, htrial, uc);
}

void pgd_tail(Exec& e, Plan* P, unsigned long long houter, int uc) {
  launch(e, k_pgd_finish, dim3(P->nchunk), dim3(VT), 0, P->dp, P->ctl, P->xp, (const double*)P->xt,
         P->vz32, houter, uc);
}

cudaError_t build_pgd_graph(Plan* P) {
  cudaGraph_t g = nullptr;
  cudaError_t err = cudaGraphCreate(&g, 0);
  if (err != cudaSuccess) return err;
  cudaGraphConditionalHandle hout = 0, htr = 0;
  err = cudaGraphConditionalHandleCreate(&hout, g, 1, cudaGraphCondAssignDefault);
  Exec top;
  top.g = g;
  top.err = err;
  Exec body = top.while_body(hout);
  if (body.err == cudaSuccess)
    body.err = cudaGraphConditionalHandleCreate(&htr, body.g, 0, cudaGraphCondAssignDefault);
  pgd_head(body, P, (unsigned long long)htr, 1);
  Exec tr = body.while_body(htr);
  pgd_trial(tr, P, (unsigned long long)htr, 1);
  if (tr.err != cudaSuccess) body.err = tr.err;
  pgd_tail(body, P, (unsigned long long)hout, 1);
  if (body.err != cudaSuccess) top.err = body.err;
  err = top.err;
  if (err == cudaSuccess) {
    if (P->pgd_exec) cudaGraphExecDestroy(P->pgd_exec);
    P->pgd_exec = nullptr;
    err = cudaGraphInstantiate(&P->pgd_exec, g, 0);
  }
  cudaGraphDestroy(g);
  return err;
}

// RPT_TIMEOUT if a row pass recorded a bounded wait that ran out (and clear it).
int check_err(Plan* P) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, P->err, sizeof(int), cudaMemcpyDeviceToHost, P->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) return cuda_fail(e, "read error word");
  if (h != 0) {
    cudaMemsetAsync(P->err, 0, sizeof(int), P->stream);
    if (h == kErrCgCluster) {
      set_error("the CG step kernel ran without its thread-block cluster");
      return RPT_ECUDA;
    }
    set_error("a row-pass pipeline wait ran out (code " + std::to_string(h) + ")");
    return RPT_TIMEOUT;
  }
  return RPT_OK;
}

cudaError_t read_ctl(Plan* P) {
  // the scalars and the plan's own groups (the rest of the group array is unused)
  const size_t bytes = offsetof(Ctl, g) + sizeof(Grp) * (size_t)P->dp.G;
  cudaError_t e = cudaMemcpyAsync(P->ctl_host, P->ctl, bytes, cudaMemcpyDeviceToHost, P->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(P->stream);
}

}  // namespace

// ===========================================================================
// entry points
// ===========================================================================

void destroy_graphs(Plan* P) {
  if (P->admm_exec) cudaGraphExecDestroy(P->admm_exec);
  if (P->admm_chol_exec) cudaGraphExecDestroy(P->admm_chol_exec);
  if (P->pgd_exec) cudaGraphExecDestroy(P->pgd_exec);
  P->admm_exec = nullptr;
  P->admm_chol_exec = nullptr;
  P->pgd_exec = nullptr;
}

namespace {
struct NvtxRange {            // NVTX range for tools (no cost without one attached)
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

int admm_solve_impl(Plan* P, const rpt_admm_params* prm, const double* z0, const double* y0, double* x_out,
                    rpt_solve_info* info, ConHook* con, rpt_solve_info* group_info);

int admm_solve(Plan* P, const rpt_admm_params* prm, const double* z0, const double* y0,
               double* x_out, rpt_solve_info* info, ConHook* con, rpt_solve_info* group_info) {
  NvtxRange r(con ? "rpt: ADMM-BB with dose constraints (cached factor)"
                  : (prm && prm->subproblem == RPT_SUB_CHOL ? "rpt: ADMM-BB (cached factor)" : "rpt: ADMM-BB (CG)"));
  return admm_solve_impl(P, prm, z0, y0, x_out, info, con, group_info);
}

// con: dose-constraint blocks; the solve then uses the cached factor (with the
// constraint terms in B_s) and the host-driven loop.  A batched plan (G > 1)
// solves its groups side by side, each with its own penalty, BB step and
// stopping test; z0, y0, resume, con and the objective tests need G = 1.
int admm_solve_impl(Plan* P, const rpt_admm_params* prm, const double* z0, const double* y0,
                    double* x_out, rpt_solve_info* info, ConHook* con, rpt_solve_info* group_info) {
  const DevPlan& dp = P->dp;
  const int n = dp.n, N = dp.N, G = dp.G;
  std::vector<double> rho(G);
  for (int g = 0; g < G; ++g) {
    rho[g] = prm->rho > 0 ? prm->rho : prm->rho_scale * P->grp_rho[g];
    if (!(rho[g] > 0) || !std::isfinite(rho[g])) {
      set_error("rho must be positive and finite (default rule gave " + std::to_string(rho[g]) +
                (G > 1 ? " for problem " + std::to_string(g) + ")" : ")"));
      return RPT_EINVAL;
    }
  }
  if (G > 1 && (z0 || y0 || prm->resume || con || std::isfinite(prm->tol_obj) || prm->f_target > 0.0)) {
    set_error("a batched plan solves from a cold start without objective tests or dose constraints");
    return RPT_EUNSUPPORTED;
  }
  if (prm->max_iter < 1 || prm->cg_max < 0 || prm->eps_abs < 0 || prm->eps_rel < 0 ||
      prm->bb_mode < 0 || prm->bb_mode > 2 || prm->z_mode < 0 || prm->z_mode > 1 ||
      prm->bb_per_scenario < 0 || prm->bb_per_scenario > 1 ||
      prm->cg_precond < 0 || prm->cg_precond > 1 || prm->subproblem < 0 || prm->subproblem > 1 ||
      !(prm->bb_kappa >= 1.0) || !(prm->cg_theta > 0) || !(prm->cg_eta0 > 0) ||
      !(prm->cg_floor_rel >= 0) || std::isnan(prm->tol_obj) || !(prm->f_target >= 0.0) ||
      !std::isfinite(prm->f_target)) {
    set_error("invalid ADMM parameters");
    return RPT_EINVAL;
  }
  if (prm->resume && !P->state_valid) {
    set_error("resume requested but the plan holds no ADMM state");
    return RPT_EINVAL;
  }
  for (int pass = 0; pass < 2; ++pass) {
    const double* a = pass ? y0 : z0;
    const size_t cnt = pass ? (size_t)N * n : (size_t)n;
    if (a)
      for (size_t i = 0; i < cnt; ++i)
        if (!std::isfinite(a[i])) {
          set_error(pass ? "y0 has a non-finite entry" : "z0 has a non-finite entry");
          return RPT_EINVAL;
        }
  }
  const int use_obj = (std::isfinite(prm->tol_obj) || prm->f_target > 0.0) ? 1 : 0;
  const bool chol = prm->subproblem == RPT_SUB_CHOL || con != nullptr;
  cudaStream_t st = P->stream;
  cudaError_t e;
  double setup_s = 0.0;
  if (chol) {
    if ((e = cudaFuncSetAttribute(k_chol_x, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(float) * (size_t)dp.n_pad))))
      return cuda_fail(e, "kernel attribute");
    const bool cached = !con && P->chol_ready && !P->chol_con && P->chol_rho == rho;
    const auto t0 = std::chrono::steady_clock::now();
    if (int rc = chol_prepare(P, rho, con)) return rc;
    if (!cached) setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  // inputs: z0 -> znew (scratch until the first z-update), y0 -> u (scratch until CG)
  if (z0 && (e = cudaMemcpyAsync(P->znew, z0, sizeof(double) * n, cudaMemcpyHostToDevice, st)))
    return cuda_fail(e, "copy z0");
  if (y0 && (e = cudaMemcpyAsync(P->u, y0, sizeof(double) * N * n, cudaMemcpyHostToDevice, st)))
    return cuda_fail(e, "copy y0");
  Ctl& c = *P->ctl_host;
  std::memset(&c, 0, sizeof(Ctl));
  for (int g = 0; g < G; ++g) {
    Grp& q = c.g[g];
    q.rho = rho[g];
    q.inv_rho = 1.0 / rho[g];
    q.step = q.step_prev = rho[g];
    q.first = 1;
    q.nn = (double)dp.Ns * (double)P->grp_n[g];
    q.cst = P->grp_const[g];
  }
  c.uact = G > 1 ? P->uact : nullptr;
  c.eps_abs = prm->eps_abs;
  c.eps_rel = prm->eps_rel;
  c.bb_kappa = prm->bb_kappa;
  c.cg_theta = prm->cg_theta;
  c.cg_eta0 = prm->cg_eta0;
  c.cg_floor = prm->cg_floor_rel;
  c.tol_obj = prm->tol_obj;
  c.f_goal = prm->f_target;
  c.const_term = P->stats.const_term;
  c.max_iter = prm->max_iter;
  c.cg_max = prm->cg_max;
  c.bb_mode = prm->bb_mode;
  c.bb_scen = prm->bb_per_scenario;
  c.step_s = P->bb_step;
  c.z_mode = prm->z_mode;
  c.precond = prm->cg_precond;
  c.use_obj = use_obj;
  if (prm->trace) {
    if (!P->trace) {
      if ((e = cudaMalloc(&P->trace, sizeof(double) * kTraceFields * kTraceCap))) return cuda_fail(e, "trace buffer");
      P->allocs.push_back(P->trace);
    }
    c.trace = P->trace;
    c.trace_cap = kTraceCap;
    c.trace_on = 1;
  }
  c.f_prev = HUGE_VAL;
  if (con) {
    c.con_q = con->q;
    c.con_t = con->t;
    c.con_sums = con->sums;
    c.con_K = con->K;
    c.con_on = 1;
  }
  if ((e = cudaMemcpyAsync(P->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, st)))
    return cuda_fail(e, "upload control block");
  if ((e = cudaMemsetAsync(P->cgcnt, 0, sizeof(int) * N, st))) return cuda_fail(e, "memset");
  if (G > 1) {   // every scenario active in the first residual pass
    std::vector<int> ones(N, 1);
    if ((e = cudaMemcpyAsync(P->uact, ones.data(), sizeof(int) * N, cudaMemcpyHostToDevice, st)) ||
        (e = cudaStreamSynchronize(st)))
      return cuda_fail(e, "activity");
  }
  if ((e = cudaEventRecord(P->ev0, st))) return cuda_fail(e, "event");
  {
    Exec ex;
    ex.st = st;
    launch(ex, k_admm_init, dim3(P->nchunk, N), dim3(VT), 0, dp, (const Ctl*)P->ctl,
           (const double*)P->znew, (const double*)P->u, z0 ? 1 : 0, y0 ? 1 : 0, prm->resume ? 1 : 0,
           (const double*)P->lb, (const double*)P->ub, (const float*)P->diag, P->dinv, P->x, P->y,
           P->z, P->dprev, P->v32);
    if (ex.err) return cuda_fail(ex.err, "launch init");
  }
  if (con && (e = con->init(P))) return cuda_fail(e, "dose-constraint initialisation");
  if (chol && prm->use_graph && !con) {
    if (!P->admm_chol_exec || P->admm_chol_exec_obj != use_obj) {
      if ((e = build_admm_chol_graph(P, use_obj))) return cuda_fail(e, "build ADMM graph");
    }
    if ((e = cudaGraphLaunch(P->admm_chol_exec, st))) return cuda_fail(e, "launch ADMM graph");
  } else if (chol) {
    const int every = prm->check_every > 0 ? prm->check_every : 1;
    for (int it = 1;; ++it) {
      Exec ex;
      ex.st = st;
      if (con) {
        if ((e = con->rhs(P))) return cuda_fail(e, "dose-constraint right-hand side");
        launch(ex, k_chol_x, dim3((dp.n + kCholRows - 1) / kCholRows, dp.N), dim3(256),
               sizeof(float) * (size_t)dp.n_pad, dp, (const Ctl*)P->ctl, (const float*)P->binv,
               (const float*)P->v32, P->x);
      } else {
        chol_iteration_head(ex, P);
      }
      admm_iteration_tail(ex, P, use_obj, 0, 0, con);
      if (ex.err) return cuda_fail(ex.err, "launch");
      if (it % every == 0 || it >= prm->max_iter) {
        if ((e = read_ctl(P))) return cuda_fail(e, "read control");
        if (P->ctl_host->stop) break;
      }
    }
    Exec ex;
    ex.st = st;
    admm_tail_final(ex, P);
    if (ex.err) return cuda_fail(ex.err, "launch");
  } else if (prm->use_graph) {
    if (!P->admm_exec || P->admm_exec_obj != use_obj) {
      if ((e = build_admm_graph(P, use_obj, nullptr, nullptr))) return cuda_fail(e, "build ADMM graph");
    }
    if ((e = cudaGraphLaunch(P->admm_exec, st))) return cuda_fail(e, "launch ADMM graph");
  } else {
    const int every = prm->check_every > 0 ? prm->check_every : 1;
    for (;;) {
      Exec ex;
      ex.st = st;
      admm_iteration_head(ex, P, 0, 0);
      if (ex.err) return cuda_fail(ex.err, "launch");
      if ((e = read_ctl(P))) return cuda_fail(e, "read control");
      while (P->ctl_host->cg_any > 0 && P->ctl_host->kcg < prm->cg_max) {
        cg_body(ex, P, 0, 0);
        if (ex.err) return cuda_fail(ex.err, "launch");
        if ((e = read_ctl(P))) return cuda_fail(e, "read control");
      }
      admm_iteration_tail(ex, P, use_obj, 0, 0);
      if (ex.err) return cuda_fail(ex.err, "launch");
      const int k_done = P->ctl_host->k + 1;
      if (k_done % every == 0 || k_done >= prm->max_iter) {
        if ((e = read_ctl(P))) return cuda_fail(e, "read control");
        if (P->ctl_host->stop) break;
      }
    }
    Exec ex;
    ex.st = st;
    admm_tail_final(ex, P);
    if (ex.err) return cuda_fail(ex.err, "launch");
  }
  if ((e = cudaEventRecord(P->ev1, st))) return cuda_fail(e, "event");
  if ((e = read_ctl(P))) return cuda_fail(e, "read control");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, P->ev0, P->ev1);
  const Ctl& h = *P->ctl_host;
  P->state_valid = true;
  if (int rc = check_err(P)) return rc;
  int status = h.diverged ? RPT_DIVERGED : (h.status ? RPT_OK : RPT_NOT_CONVERGED);
  // a batched plan returns every group's z (a diverged group's as it stands;
  // its own status says so)
  if ((status != RPT_DIVERGED || G > 1) && x_out) {
    if ((e = cudaMemcpyAsync(x_out, P->z, sizeof(double) * n * G, cudaMemcpyDeviceToHost, st)))
      return cuda_fail(e, "copy x_out");
    if ((e = cudaStreamSynchronize(st))) return cuda_fail(e, "sync");
  }
  // init + per iteration (residual pass, CG init, 2 per CG step, z/d/y, 2 for the
  // optional objective test) + final objective pass and its reduction (+ staging)
  const long long kernels = (chol ? 3 + 5LL * h.k : 3 + 5LL * h.k + 2LL * h.cg_steps) +
                            (use_obj ? 2LL * h.k : 0LL) + (G > 1 ? 1 : 0);
  auto fill = [&](rpt_solve_info* o, const Grp& q, int st_q) {
    std::memset(o, 0, sizeof(*o));
    o->status = st_q;
    o->iterations = q.k;
    o->inner = q.cg;
    o->row_passes = h.passes;
    o->kernels = kernels;
    o->setup_seconds = setup_s;
    o->seconds = ms * 1e-3;
    o->f = G > 1 ? q.f : h.f_cur;
    o->r_prim = q.r_prim;
    o->r_dual = q.r_dual;
    o->eps_prim = q.eps_prim;
    o->eps_dual = q.eps_dual;
    o->step = q.step;
    o->rho = q.rho;
  };
  if (info) {
    fill(info, h.g[0], status);
    if (G > 1) {
      // over all groups: the loop count, the CG steps, the total objective, and the
      // residual norms of the stacked vectors; step and rho are per group only
      double rp = 0, rd = 0, ep = 0, ed = 0;
      for (int g = 0; g < G; ++g) {
        rp += h.g[g].r_prim * h.g[g].r_prim;
        rd += h.g[g].r_dual * h.g[g].r_dual;
        ep += h.g[g].eps_prim * h.g[g].eps_prim;
        ed += h.g[g].eps_dual * h.g[g].eps_dual;
      }
      info->iterations = h.k;
      info->inner = h.cg_total;
      info->f = h.f_cur;
      info->r_prim = std::sqrt(rp);
      info->r_dual = std::sqrt(rd);
      info->eps_prim = std::sqrt(ep);
      info->eps_dual = std::sqrt(ed);
      info->step = 0.0;
      info->rho = 0.0;
    }
  }
  if (group_info)
    for (int g = 0; g < G; ++g)
      fill(&group_info[g], h.g[g],
           h.g[g].diverged ? RPT_DIVERGED : (h.g[g].status ? RPT_OK : RPT_NOT_CONVERGED));
  P->trace_count = prm->trace ? std::min(h.k, kTraceCap) : 0;
  if (status == RPT_DIVERGED) set_error("ADMM residuals became non-finite");
  return status;
}

int pgd_solve(Plan* P, const rpt_pgd_params* prm, const double* x0, double* x_out,
              rpt_solve_info* info) {
  NvtxRange range("rpt: PGD");
  const DevPlan& dp = P->dp;
  const int n = dp.n;
  if (!(prm->beta > 0 && prm->beta < 1) || !(prm->gamma > 0 && prm->gamma < 1) ||
      prm->max_iter < 1 || prm->max_trials < 1 || !(prm->tol_rel_df >= 0) || std::isnan(prm->alpha)) {
    set_error("invalid PGD parameters");
    return RPT_EINVAL;
  }
  if (x0)
    for (int j = 0; j < n; ++j)
      if (!std::isfinite(x0[j])) {
        set_error("x0 has a non-finite entry");
        return RPT_EINVAL;
      }
  double alpha = prm->alpha;
  double L = 0.0;
  if (!(alpha > 0)) {
    int rc = compute_lipschitz(P, &L);
    if (rc != RPT_OK) return rc;
    if (!(L > 0)) {
      set_error("Lipschitz estimate is zero (empty problem?)");
      return RPT_EINVAL;
    }
    alpha = 4.0 / L;
  }
  cudaStream_t st = P->stream;
  cudaError_t e;
  if (x0 && (e = cudaMemcpyAsync(P->xt, x0, sizeof(double) * n, cudaMemcpyHostToDevice, st)))
    return cuda_fail(e, "copy x0");
  Ctl& c = *P->ctl_host;
  std::memset(&c, 0, sizeof(Ctl));
  c.const_term = P->stats.const_term;
  c.alpha = alpha;
  c.beta_a = prm->beta;
  c.gamma = prm->gamma;
  c.tol_df = prm->tol_rel_df;
  c.f_target = prm->f_target;
  c.pgd_max_iter = prm->max_iter;
  c.max_trials = prm->max_trials;
  if ((e = cudaMemcpyAsync(P->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, st)))
    return cuda_fail(e, "upload control block");
  if ((e = cudaEventRecord(P->ev0, st))) return cuda_fail(e, "event");
  {
    Exec ex;
    ex.st = st;
    launch(ex, k_pgd_init, dim3(P->nchunk), dim3(VT), 0, dp, (const double*)P->xt, x0 ? 1 : 0,
           (const double*)P->lb, (const double*)P->ub, P->xp, P->vz32);
    if (ex.err) return cuda_fail(ex.err, "launch init");
  }
  if (prm->use_graph) {
    if (!P->pgd_exec && (e = build_pgd_graph(P))) return cuda_fail(e, "build PGD graph");
    if ((e = cudaGraphLaunch(P->pgd_exec, st))) return cuda_fail(e, "launch PGD graph");
  } else {
    for (;;) {
      Exec ex;
      ex.st = st;
      pgd_head(ex, P, 0, 0);
      do {
        pgd_trial(ex, P, 0, 0);
        if (ex.err) return cuda_fail(ex.err, "launch");
        if ((e = read_ctl(P))) return cuda_fail(e, "read control");
      } while (!P->ctl_host->accepted && !P->ctl_host->failed);
      pgd_tail(ex, P, 0, 0);
      if (ex.err) return cuda_fail(ex.err, "launch");
      if ((e = read_ctl(P))) return cuda_fail(e, "read control");
      if (P->ctl_host->stop) break;
    }
  }
  if ((e = cudaEventRecord(P->ev1, st))) return cuda_fail(e, "event");
  if ((e = read_ctl(P))) return cuda_fail(e, "read control");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, P->ev0, P->ev1);
  const Ctl& h = *P->ctl_host;
  if (int rc = check_err(P)) return rc;
  int status = h.diverged ? RPT_DIVERGED : (h.status ? RPT_OK : RPT_NOT_CONVERGED);
  if (status != RPT_DIVERGED && x_out) {
    if ((e = cudaMemcpyAsync(x_out, P->xp, sizeof(double) * n, cudaMemcpyDeviceToHost, st)))
      return cuda_fail(e, "copy x_out");
    if ((e = cudaStreamSynchronize(st))) return cuda_fail(e, "sync");
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = status;
    info->iterations = h.pk;
    info->inner = h.trials_total;
    info->row_passes = h.passes;
    // init + per iteration (residual pass, gradient, finish) + 3 per Armijo trial
    info->kernels = 1 + 3LL * h.pouter + 3LL * h.trials_total;
    info->seconds = ms * 1e-3;
    info->f = h.f_cur;
    info->step = h.pstep;
    info->rho = L > 0 ? L : P->lipschitz;
  }
  if (status == RPT_DIVERGED) set_error("PGD objective became non-finite");
  return status;
}

// ---- operators -----------------------------------------------------------------

static cudaError_t stage_host_vector(Plan* P, float* dst, const double* src, int count_vecs) {
  const DevPlan& dp = P->dp;
  std::vector<float> h((size_t)count_vecs * dp.n_pad, 0.f);
  for (int s = 0; s < count_vecs; ++s)
    for (int j = 0; j < dp.n; ++j) h[(size_t)s * dp.n_pad + j] = (float)src[(size_t)s * dp.n + j];
  cudaError_t e = cudaMemcpyAsync(dst, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, P->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(P->stream);
}

int op_apply_normal(Plan* P, const double* v, double rho, double* u_out) {
  const DevPlan& dp = P->dp;
  for (size_t i = 0; i < (size_t)dp.N * dp.n; ++i)
    if (!std::isfinite(v[i])) {
      set_error("v has a non-finite entry");
      return RPT_EINVAL;
    }
  if (!(rho >= 0) || !std::isfinite(rho)) {
    set_error("rho must be finite and >= 0");
    return RPT_EINVAL;
  }
  cudaError_t e;
  if ((e = stage_host_vector(P, P->v32, v, dp.N))) return cuda_fail(e, "stage");
  if ((e = cudaMemcpyAsync(P->x, v, sizeof(double) * dp.N * dp.n, cudaMemcpyHostToDevice, P->stream)))
    return cuda_fail(e, "copy");
  Exec ex;
  ex.st = P->stream;
  rowpass(ex, P, kNormal, P->v32, dp.n_pad, nullptr);
  launch(ex, k_reduce_scen, dim3(P->nchunk, dp.N), dim3(VT), 0, dp, (const float*)P->partial,
         (const double*)P->x, 0.5 * rho, P->u);
  if (ex.err) return cuda_fail(ex.err, "launch");
  if ((e = cudaMemcpyAsync(u_out, P->u, sizeof(double) * dp.N * dp.n, cudaMemcpyDeviceToHost, P->stream)))
    return cuda_fail(e, "copy out");
  if ((e = cudaStreamSynchronize(P->stream))) return cuda_fail(e, "sync");
  P->state_valid = false;   // x was used as scratch
  return check_err(P);
}

int op_gradient(Plan* P, const double* x, double* g_out, double* f_out) {
  const DevPlan& dp = P->dp;
  for (int j = 0; j < dp.n; ++j)
    if (!std::isfinite(x[j])) {
      set_error("x has a non-finite entry");
      return RPT_EINVAL;
    }
  cudaError_t e;
  if ((e = stage_host_vector(P, P->vz32, x, 1))) return cuda_fail(e, "stage");
  Exec ex;
  ex.st = P->stream;
  rowpass(ex, P, kResid, P->vz32, 0, nullptr);
  launch(ex, k_reduce_all, dim3(P->nchunk), dim3(VT), 0, dp, (const float*)P->partial, 2.0, P->g);
  if (ex.err) return cuda_fail(ex.err, "launch");
  std::vector<double> objp(dp.N);
  if ((e = cudaMemcpyAsync(g_out, P->g, sizeof(double) * dp.n, cudaMemcpyDeviceToHost, P->stream)))
    return cuda_fail(e, "copy out");
  if ((e = cudaMemcpyAsync(objp.data(), dp.objs, sizeof(double) * dp.N, cudaMemcpyDeviceToHost, P->stream)))
    return cuda_fail(e, "copy out");
  if ((e = cudaStreamSynchronize(P->stream))) return cuda_fail(e, "sync");
  if (int rc = check_err(P)) return rc;
  if (f_out) {
    double f = P->stats.const_term;
    for (double v : objp) f += v;
    *f_out = f;
  }
  return RPT_OK;
}

int op_objective(Plan* P, const double* x, double* f_out, double* dose_out) {
  const DevPlan& dp = P->dp;
  for (int j = 0; j < dp.n; ++j)
    if (!std::isfinite(x[j])) {
      set_error("x has a non-finite entry");
      return RPT_EINVAL;
    }
  cudaError_t e;
  if (dose_out && !P->dose) {
    if ((e = cudaMalloc(&P->dose, sizeof(float) * (size_t)dp.N * dp.m_act))) {
      P->dose = nullptr;
      set_error("out of device memory for doses");
      return RPT_ENOMEM;
    }
    P->allocs.push_back(P->dose);
  }
  if ((e = stage_host_vector(P, P->vz32, x, 1))) return cuda_fail(e, "stage");
  // rows that are empty in a scenario are not visited: their dose is zero
  if (dose_out && (e = cudaMemsetAsync(P->dose, 0, sizeof(float) * (size_t)dp.N * dp.m_act, P->stream)))
    return cuda_fail(e, "memset");
  Exec ex;
  ex.st = P->stream;
  rowpass(ex, P, dose_out ? kDose : kObj, P->vz32, 0, nullptr, P->dose);
  if (ex.err) return cuda_fail(ex.err, "launch");
  std::vector<double> objp(dp.N);
  if ((e = cudaMemcpyAsync(objp.data(), dp.objs, sizeof(double) * dp.N, cudaMemcpyDeviceToHost, P->stream)))
    return cuda_fail(e, "copy out");
  std::vector<float> dose;
  if (dose_out) {
    dose.resize((size_t)dp.N * dp.m_act);
    if ((e = cudaMemcpyAsync(dose.data(), P->dose, sizeof(float) * dose.size(), cudaMemcpyDeviceToHost, P->stream)))
      return cuda_fail(e, "copy out");
  }
  if ((e = cudaStreamSynchronize(P->stream))) return cuda_fail(e, "sync");
  if (int rc = check_err(P)) return rc;
  if (f_out) {
    double f = P->stats.const_term;
    for (double v : objp) f += v;
    *f_out = f;
  }
  if (dose_out) {
    std::memset(dose_out, 0, sizeof(double) * (size_t)dp.N * dp.m);
    for (int s = 0; s < dp.N; ++s)
      for (int k = 0; k < dp.m_act; ++k)
        dose_out[(size_t)s * dp.m + P->kept_rows[k]] = dose[(size_t)s * dp.m_act + k];
  }
  return RPT_OK;
}

int profile_row_pass(Plan* P, int mode, int reps, double* ms, double* bytes) {
  if ((mode != kNormal && mode != kResid) || reps < 1) {
    set_error("profile_row_pass: mode must be 0 or 1 and reps >= 1");
    return RPT_EINVAL;
  }
  const DevPlan& dp = P->dp;
  cudaError_t e;
  Exec ex;
  ex.st = P->stream;
  rowpass(ex, P, mode, P->v32, dp.n_pad, nullptr);   // warm-up launch
  if ((e = cudaEventRecord(P->ev0, P->stream))) return cuda_fail(e, "event");
  for (int r = 0; r < reps; ++r) rowpass(ex, P, mode, P->v32, dp.n_pad, nullptr);
  if (ex.err) return cuda_fail(ex.err, "launch");
  if ((e = cudaEventRecord(P->ev1, P->stream))) return cuda_fail(e, "event");
  if ((e = cudaEventSynchronize(P->ev1))) return cuda_fail(e, "sync");
  float t = 0.f;
  cudaEventElapsedTime(&t, P->ev0, P->ev1);
  if (int rc = check_err(P)) return rc;
  if (ms) *ms = (double)t / reps;
  if (bytes) {
    if (dp.path == 3) {
      // bundled: stored block columns (4 values + index) and the 64-byte bundle
      // records the ring copies, plus the spot vectors in and out
      const int bv = dp.value_format == RPT_F32 ? 4 : (dp.value_format == RPT_BF16 ? 2 : 1);
      const int bi = dp.index_width == 16 ? 2 : 4;
      *bytes = (double)P->stats.block_cols * (4.0 * bv + bi) + 64.0 * (double)(P->stats.bundles + dp.N) +
               2.0 * 4.0 * (double)dp.N * dp.n;
    } else {
      const double per_row = 4.0 * (mode == kResid ? 2 : 1);   // weight (+ prescription)
      *bytes = (double)P->stats.matrix_bytes + per_row * (double)dp.N * dp.m_act +
               2.0 * 4.0 * (double)dp.N * dp.n;
    }
  }
  return RPT_OK;
}

int compute_bconst(Plan* P) {
  const DevPlan& dp = P->dp;
  cudaError_t e;
  if ((e = cudaMemsetAsync(P->v32, 0, sizeof(float) * (size_t)dp.N * dp.n_pad, P->stream)))
    return cuda_fail(e, "memset");
  Exec ex;
  ex.st = P->stream;
  rowpass(ex, P, kResid, P->v32, dp.n_pad, nullptr);
  launch(ex, k_neg_partials, dim3(P->nchunk, dp.N), dim3(VT), 0, dp, (const float*)P->partial, P->bchol);
  if (ex.err) return cuda_fail(ex.err, "launch");
  return RPT_OK;
}

int compute_lipschitz(Plan* P, double* L) {
  if (P->lipschitz > 0) {
    *L = P->lipschitz;
    return RPT_OK;
  }
  const DevPlan& dp = P->dp;
  std::vector<double> v(dp.n, 1.0 / std::sqrt((double)dp.n)), u(dp.n);
  double lam = 0.0;
  cudaError_t e;
  for (int it = 0; it < 30; ++it) {
    if ((e = stage_host_vector(P, P->vz32, v.data(), 1))) return cuda_fail(e, "stage");
    Exec ex;
    ex.st = P->stream;
    rowpass(ex, P, kNormal, P->vz32, 0, nullptr);
    launch(ex, k_reduce_all, dim3(P->nchunk), dim3(VT), 0, dp, (const float*)P->partial, 1.0, P->g);
    if (ex.err) return cuda_fail(ex.err, "launch");
    if ((e = cudaMemcpyAsync(u.data(), P->g, sizeof(double) * dp.n, cudaMemcpyDeviceToHost, P->stream)))
      return cuda_fail(e, "copy");
    if ((e = cudaStreamSynchronize(P->stream))) return cuda_fail(e, "sync");
    double nrm = 0.0;
    for (double a : u) nrm += a * a;
    nrm = std::sqrt(nrm);
    lam = nrm;
    if (nrm == 0.0) break;
    for (int j = 0; j < dp.n; ++j) v[j] = u[j] / nrm;
  }
  P->lipschitz = 2.0 * lam;
  *L = P->lipschitz;
  return RPT_OK;
}

}  // namespace rpt
