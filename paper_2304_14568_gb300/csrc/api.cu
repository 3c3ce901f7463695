// C ABI of librpt: plan creation (validation, row compaction, row blocks,
// upload, optional quantisation) and the extern "C" wrappers.
#include <algorithm>
#include <cstdlib>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <chrono>
#include <exception>
#include <thread>
#include <vector>

#include "batch.h"
#include "layout.h"
#include "plan.h"

namespace rpt {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return RPT_ENOMEM;
  return RPT_ECUDA;
}

namespace {

// ---- quantisation kernels (plan creation only) ---------------------------------

// Values and columns: value k belongs to stored entry k >> sh (sh = 0 for CSR
// rows, 2 for row bundles with 4 values per block column).
__global__ void k_colmax(const float* __restrict__ val, const int32_t* __restrict__ col, int64_t nval, int sh,
                         unsigned int* __restrict__ mx) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nval;
       k += (int64_t)gridDim.x * blockDim.x)
    atomicMax(&mx[col[k >> sh]], __float_as_uint(fabsf(val[k])));   // |a| >= 0 orders like its bits
}

__global__ void k_scales(const unsigned int* __restrict__ mx, int n, int n_pad, float fmt_max,
                         float* __restrict__ scale) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_pad) return;
  float s = 1.f;
  if (j < n) {
    const float m = __uint_as_float(mx[j]);
    if (m > 0.f) s = m / fmt_max;
  }
  scale[j] = s;
}

template <typename Q>
__global__ void k_quantise(const float* __restrict__ val, const int32_t* __restrict__ col, int64_t nval, int sh,
                           const float* __restrict__ scale, Q* __restrict__ out);

template <>
__global__ void k_quantise<__nv_bfloat16>(const float* __restrict__ val, const int32_t* __restrict__ col,
                                          int64_t nval, int sh, const float* __restrict__ scale,
                                          __nv_bfloat16* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nval;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = __float2bfloat16_rn(val[k] / scale[col[k >> sh]]);
}

template <>
__global__ void k_quantise<__nv_fp8_e4m3>(const float* __restrict__ val, const int32_t* __restrict__ col,
                                          int64_t nval, int sh, const float* __restrict__ scale,
                                          __nv_fp8_e4m3* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nval;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = __nv_fp8_e4m3(val[k] / scale[col[k >> sh]]);   // round to nearest, saturating
}

__global__ void k_to_u16(const int32_t* __restrict__ in, int64_t nnz, uint16_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (uint16_t)in[k];
}

struct ScenarioCheck {
  std::string err;
  double trace = 0.0;          // sum_i w_i sum_j a_ij^2
  std::vector<double> diag;    // [n] sum_i w_i a_ij^2 (Jacobi preconditioner)
  double colsq_max = 0.0;      // max_j sum_i a_ij^2 (unweighted)
};

void check_scenario(const rpt_problem* pr, int s, ScenarioCheck* out) {
  const int m = pr->m, n = pr->n;
  const int32_t* rp = pr->row_ptr[s];
  const int32_t* ci = pr->col_idx[s];
  const float* va = pr->val[s];
  if (rp[0] != 0) {
    out->err = "row_ptr[" + std::to_string(s) + "][0] != 0";
    return;
  }
  double tr = 0.0;
  out->diag.assign(n, 0.0);
  std::vector<double> colsq(n, 0.0);
  for (int i = 0; i < m; ++i) {
    const int32_t a = rp[i], b = rp[i + 1];
    if (b < a) {
      out->err = "row_ptr of scenario " + std::to_string(s) + " decreases at row " + std::to_string(i);
      return;
    }
    double rs = 0.0;
    int32_t prev = -1;
    for (int32_t k = a; k < b; ++k) {
      const int32_t c = ci[k];
      const float v = va[k];
      if (c < 0 || c >= n) {
        out->err = "column index out of range in scenario " + std::to_string(s) + ", row " + std::to_string(i);
        return;
      }
      if (c <= prev) {
        out->err = "column indices not strictly increasing in scenario " + std::to_string(s) +
                   ", row " + std::to_string(i);
        return;
      }
      prev = c;
      if (!std::isfinite(v) || v < 0.f) {
        out->err = "value not finite or negative in scenario " + std::to_string(s) + ", row " + std::to_string(i);
        return;
      }
      rs += (double)v * (double)v;
      out->diag[c] += pr->voxel_w[i] * (double)v * (double)v;
      colsq[c] += (double)v * (double)v;
    }
    tr += pr->voxel_w[i] * rs;
  }
  out->trace = tr;
  for (int j = 0; j < n; ++j) out->colsq_max = std::max(out->colsq_max, colsq[j]);
}

// Device allocations of a plan.  cap (rpt_device_opts.device_mem_cap, bytes; 0:
// none) caps the plan's total, so that running out of device memory can be
// tested without exhausting the device: a request past it fails as cudaMalloc
// would.
struct Alloc {
  Plan* P;
  size_t cap = 0;
  cudaError_t err = cudaSuccess;
  size_t total = 0;
  template <typename T>
  T* get(size_t count) {
    if (err != cudaSuccess) return nullptr;
    void* p = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    if (cap && total + bytes > cap) {
      err = cudaErrorMemoryAllocation;
      return nullptr;
    }
    total += bytes;
    err = cudaMalloc(&p, bytes);
    if (err != cudaSuccess) return nullptr;
    P->allocs.push_back(p);
    return (T*)p;
  }
};

void free_plan(Plan* P) {
  if (!P) return;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(P->device);
  if (P->stream) cudaStreamSynchronize(P->stream);
  destroy_graphs(P);
  for (void* a : P->allocs) cudaFree(a);
  P->allocs.clear();
  if (P->ctl_host) cudaFreeHost(P->ctl_host);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  if (P->own_stream && P->stream) cudaStreamDestroy(P->stream);
  if (cur >= 0) cudaSetDevice(cur);
  delete P;
}

using namespace layout;   // lanes per row, row lists, bank balance, chunks (layout.h)

// One bulk-copy ring configuration and its chunk lists.
struct RingCfg {
  int cmax = 0, rmax = 0, stages = 0;
  int thr = kTmaThreads;             // bundled path: threads of a row-pass CTA
  std::vector<ChunkDesc> chunks;
  std::vector<int> scen_chunk;
};

// The caller's ring geometry (rpt_device_opts chunk_entries / chunk_rows /
// stages), as the only candidate; empty when the caller leaves all three to
// the library.  Unset fields take the given defaults.
std::vector<int3> ring_override(const rpt_device_opts* o, int cmax, int rmax, int stages) {
  if (!o || (o->chunk_entries <= 0 && o->chunk_rows <= 0 && o->stages <= 0)) return {};
  return {make_int3(std::max(64, o->chunk_entries > 0 ? o->chunk_entries : cmax) & ~15,
                    std::max(1, o->chunk_rows > 0 ? o->chunk_rows : rmax),
                    std::min(8, std::max(2, o->stages > 0 ? o->stages : stages)))};
}

// U (batched plans): pr is U->view, whose scenarios are the units (problem g,
// scenario s) of U->G problems; bounds come from U, one box per problem.
int create_plan(const rpt_problem* pr, const rpt_device_opts* opts, rpt_plan** out,
                const batch::Units* U = nullptr) {
  if (!pr || !out) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  // phase times of the creation (rpt_plan_stats): host layout, device work, autotuning
  using clock = std::chrono::steady_clock;
  auto secs = [](clock::time_point a, clock::time_point b) { return std::chrono::duration<double>(b - a).count(); };
  const clock::time_point t_begin = clock::now();
  const int m = pr->m, n = pr->n, N = pr->N;
  const int G = U ? U->G : 1, Ns = U ? U->Ns : N;
  static_assert(batch::kMaxProblems == kMaxGroups, "batched problems = solver groups");
  // group of a row (batched plans: the problem that owns it) and of a scenario
  std::vector<int32_t> rgrp;
  if (U) {
    rgrp.resize(m);
    for (int g = 0; g < G; ++g)
      for (int i = U->row_off[g]; i < U->row_off[g + 1]; ++i) rgrp[i] = g;
  }
  auto row_group = [&](int i) { return U ? rgrp[i] : 0; };
  if (m < 1 || n < 1 || N < 1) {
    set_error("m, n and N must be >= 1");
    return RPT_EINVAL;
  }
  if (n > RPT_MAX_SPOTS) {
    set_error("n = " + std::to_string(n) + " exceeds RPT_MAX_SPOTS = " + std::to_string(RPT_MAX_SPOTS));
    return RPT_EUNSUPPORTED;
  }
  if (pr->value_format < RPT_F32 || pr->value_format > RPT_FP8E4M3) {
    set_error("unknown value_format");
    return RPT_EUNSUPPORTED;
  }
  if (pr->index_width != 32 && pr->index_width != 16) {
    set_error("index_width must be 32 or 16");
    return RPT_EUNSUPPORTED;
  }
  if (pr->index_width == 16 && n > 65535) {
    set_error("index_width 16 needs n <= 65535");
    return RPT_EINVAL;
  }
  if (opts && (opts->row_path < 0 || opts->row_path > 4 || opts->accumulate < 0 || opts->accumulate > 2 ||
               (opts->ring_threads != 0 && opts->ring_threads != 1024 && opts->ring_threads != 768 &&
                opts->ring_threads != 640))) {
    set_error("row_path must be 0..4, accumulate 0..2 and ring_threads 0, 640, 768 or 1024");
    return RPT_EINVAL;
  }
  if (!pr->row_ptr || !pr->col_idx || !pr->val || !pr->voxel_w || !pr->presc) {
    set_error("null array in rpt_problem");
    return RPT_EINVAL;
  }
  for (int s = 0; s < N; ++s)
    if (!pr->row_ptr[s] || (!pr->col_idx[s] && pr->row_ptr[s][m] > 0) || (!pr->val[s] && pr->row_ptr[s][m] > 0)) {
      set_error("null CSR array for scenario " + std::to_string(s));
      return RPT_EINVAL;
    }
  for (int i = 0; i < m; ++i) {
    if (!std::isfinite(pr->voxel_w[i]) || pr->voxel_w[i] < 0) {
      set_error("voxel_w[" + std::to_string(i) + "] not finite or negative");
      return RPT_EINVAL;
    }
    if (!std::isfinite(pr->presc[i]) || pr->presc[i] < 0) {
      set_error("presc[" + std::to_string(i) + "] not finite or negative");
      return RPT_EINVAL;
    }
  }
  std::vector<double> cs(N, 1.0);
  if (pr->scen_weight)
    for (int s = 0; s < N; ++s) {
      if (!std::isfinite(pr->scen_weight[s]) || pr->scen_weight[s] < 0) {
        set_error("scen_weight[" + std::to_string(s) + "] not finite or negative");
        return RPT_EINVAL;
      }
      cs[s] = pr->scen_weight[s];
    }
  std::vector<double> lb((size_t)G * n, 0.0), ub((size_t)G * n, HUGE_VAL);
  for (size_t j = 0; j < (size_t)G * n; ++j) {
    if (U) {
      lb[j] = U->lb[j];
      ub[j] = U->ub[j];
    } else {
      if (pr->lb) lb[j] = pr->lb[j];
      if (pr->ub) ub[j] = pr->ub[j];
    }
    if (!std::isfinite(lb[j]) || std::isnan(ub[j]) || ub[j] == -HUGE_VAL || lb[j] > ub[j]) {
      set_error("bounds invalid at spot " + std::to_string(j % n) +
                (U ? " of problem " + std::to_string(j / n) : std::string()) + " (need finite lb <= ub)");
      return RPT_EINVAL;
    }
  }
  // ---- CSR validation (scenarios spread over the host threads) ----
  std::vector<ScenarioCheck> chk(N);
  parallel_for(N, std::min<int>(std::max(1u, std::thread::hardware_concurrency()), 32),
               [&](int s, int) { check_scenario(pr, s, &chk[s]); });
  for (int s = 0; s < N; ++s)
    if (!chk[s].err.empty()) {
      set_error(chk[s].err);
      return RPT_EINVAL;
    }
  // ---- row compaction: drop rows with no entry in any scenario ----
  std::vector<uint8_t> keep(m, 0);
  for (int s = 0; s < N; ++s) {
    const int32_t* rp = pr->row_ptr[s];
    for (int i = 0; i < m; ++i)
      if (rp[i + 1] > rp[i]) keep[i] = 1;
  }
  // a row's constant c_s w p^2 counts in the scenarios of its own group only
  std::vector<int32_t> kept;
  kept.reserve(m);
  std::vector<double> gconst(G, 0.0);
  std::vector<int32_t> dropped;
  for (int i = 0; i < m; ++i) {
    if (keep[i]) {
      kept.push_back(i);
    } else {
      dropped.push_back(i);
      const int g = row_group(i);
      for (int s = g * Ns; s < (g + 1) * Ns; ++s) gconst[g] += cs[s] * pr->voxel_w[i] * pr->presc[i] * pr->presc[i];
    }
  }
  if (kept.empty()) {   // keep one (empty) row so every launch has work items
    kept.push_back(0);
    dropped.erase(dropped.begin());
    const int g = row_group(0);
    for (int s = g * Ns; s < (g + 1) * Ns; ++s) gconst[g] -= cs[s] * pr->voxel_w[0] * pr->presc[0] * pr->presc[0];
  }
  const int m_act = (int)kept.size();
  // On the device every row is padded with zero entries (column 0, value 0) to a
  // multiple of 4 entries, so rows start on 16-byte boundaries and lanes can load
  // 4 entries at once; pnnz[s] counts scenario s's stored (padded) entries.
  std::vector<int64_t> nnz(N), pnnz(N), base(N);
  int64_t NNZ = 0, NNZp = 0;
  for (int s = 0; s < N; ++s) {
    const int32_t* rp = pr->row_ptr[s];
    nnz[s] = rp[m];
    int64_t pn = 0;
    for (int i = 0; i < m; ++i) pn += ((int64_t)(rp[i + 1] - rp[i]) + 3) & ~(int64_t)3;
    // row records hold a scenario's entry offsets as int32
    if (pn > (int64_t)INT32_MAX - 64) {
      set_error("scenario " + std::to_string(s) + " has " + std::to_string(pn) +
                " entries after row padding; at most 2^31 - 65 per scenario are supported");
      return RPT_EUNSUPPORTED;
    }
    pnnz[s] = pn;
    base[s] = NNZp;
    NNZ += nnz[s];
    NNZp += pn;
  }

  const clock::time_point t_host0 = clock::now();
  Plan* P = new (std::nothrow) Plan();
  if (!P) {
    set_error("out of host memory");
    return RPT_ENOMEM;
  }
  // an exception from here on (out of host memory) releases the plan while it
  // unwinds; every error return releases it itself
  struct ReleaseOnThrow {
    Plan* p;
    int before = std::uncaught_exceptions();
    ~ReleaseOnThrow() {
      if (std::uncaught_exceptions() > before) free_plan(p);
    }
  } release_on_throw{P};
  P->device = opts ? opts->device : 0;
  cudaError_t e = cudaSetDevice(P->device);
  if (e != cudaSuccess) {
    free_plan(P);
    return cuda_fail(e, "cudaSetDevice");
  }
  cudaDeviceGetAttribute(&P->sm_count, cudaDevAttrMultiProcessorCount, P->device);
  if (opts && opts->stream) {
    P->stream = (cudaStream_t)opts->stream;
  } else {
    if ((e = cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking))) {
      free_plan(P);
      return cuda_fail(e, "cudaStreamCreate");
    }
    P->own_stream = true;
  }
  const clock::time_point t_dev0 = clock::now();
  const int n_pad = (n + 31) / 32 * 32;
  DevPlan& dp = P->dp;
  dp.m = m;
  dp.n = n;
  dp.N = N;
  dp.G = G;
  dp.Ns = Ns;
  dp.m_act = m_act;
  dp.n_pad = n_pad;
  dp.value_format = pr->value_format;
  // testing hook: the bulk-copy rings' producer issues no copy, so every
  // consumer wait runs out (after its one-second bound) and the pass reports
  // RPT_TIMEOUT; the bounded waits are tested without a GPU fault
  dp.inject_timeout = (opts && opts->inject_timeout) ? 1 : 0;
  dp.index_width = pr->index_width;
  P->nchunk = (n + kVecThreads - 1) / kVecThreads;
  P->kept_rows = kept;
  const int bi = pr->index_width == 16 ? 2 : 4;
  const int bv = pr->value_format == RPT_F32 ? 4 : (pr->value_format == RPT_BF16 ? 2 : 1);

  int min_lanes = std::min(32, std::max(1, (opts && opts->min_lanes > 0) ? opts->min_lanes : 8));
  min_lanes = 1 << (31 - __builtin_clz((unsigned)min_lanes));   // power of two
  // row path: the caller's choice, else the bundled ring when its stage fits the
  // plan, else the bulk-copy ring when it fits, else the register path
  const int want_path = opts ? opts->row_path : 0;
  const int want_thr = opts ? opts->ring_threads : 0;   // checked on entry
  const bool exact = opts && opts->accumulate == 1;      // bundled path: fixed-point sums on request
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
  const bool autotune = opts && opts->autotune;
  // each scenario's non-empty rows in kept order (rows empty in a scenario add
  // c_s w p^2 to the constant)
  std::vector<std::vector<int32_t>> order(N);
  P->empty_kept.assign(N, {});
  for (int s = 0; s < N; ++s) {
    const int32_t* rp = pr->row_ptr[s];
    const int g = s / Ns;
    for (int k = 0; k < m_act; ++k) {
      if (row_group(kept[k]) != g) continue;   // another problem's row (batched plans)
      const int len = rp[kept[k] + 1] - rp[kept[k]];
      if (len > 0) {
        order[s].push_back(k);
      } else {
        gconst[g] += cs[s] * pr->voxel_w[kept[k]] * pr->presc[kept[k]] * pr->presc[kept[k]];
        P->empty_kept[s].push_back(k);
      }
    }
  }
  double const_term = 0.0;
  for (int g = 0; g < G; ++g) const_term += gconst[g];
  P->nz_index.assign((size_t)N * m_act, -1);
  for (int s = 0; s < N; ++s)
    for (size_t q = 0; q < order[s].size(); ++q) P->nz_index[(size_t)s * m_act + order[s][q]] = (int32_t)q;
  P->scen_c = cs;
  P->dropped_rows = dropped;
  P->colsq_max.assign(N, 0.0);
  for (int s = 0; s < N; ++s) P->colsq_max[s] = chk[s].colsq_max;
  // stored layout, filled by one of the branches below
  RowLists R;                        // per scenario: rows (CSR) or bundles, with entry offsets
  std::vector<int32_t> col_h;        // [NE] spot index per stored entry (block column)
  std::vector<float> val_h;          // [NE * vpe]
  // bundled layout: each scenario's block columns stay in their own arrays and
  // are uploaded to their offsets (no host-side concatenation)
  std::vector<std::vector<int32_t>> bcol;
  std::vector<std::vector<float>> bval;
  std::vector<int4> rec_h;           // records uploaded to the device
  std::vector<int> recbase_h(N + 1, 0);
  std::vector<int64_t> ebase(N, 0), ecount(N, 0);   // first stored entry and count per scenario
  std::vector<int> rec_of_h((size_t)N * m_act, -1);
  int64_t NE = 0;
  int vpe = 1;
  bool bundled = false, dyn = false;
  int64_t n_bundles = 0;
  std::vector<int4> blocks;
  std::vector<int> blk_first(N + 1, 0);
  std::vector<ChunkDesc> chunks;
  std::vector<int> scen_chunk;
  bool use_tma = false, use_stream = false;
  int ctas = 0;
  std::vector<RingCfg> ring_cfgs;   // ring configurations that fit (all of them when autotuning)
  // ---- bundled layout (path 4) ----
  if (want_path == 4 || want_path == 0) {
    std::vector<int3> cands = ring_override(opts, 3072, 192, 2);
    if (cands.empty())
      // wide stages first: fewer, longer phases of the ring measured fastest (a
      // stage holds at most 128 bundle records, enough for 4096 block columns of
      // the average bundle); the list goes down to stages that fit wide plans
      cands = {make_int3(4096, 128, 2), make_int3(2560, 128, 3), make_int3(3072, 192, 2), make_int3(2048, 128, 3),
               make_int3(4096, 256, 2), make_int3(2048, 128, 2), make_int3(1536, 96, 3), make_int3(1024, 64, 3),
               make_int3(1024, 64, 2), make_int3(512, 32, 2),
               make_int3(6144, 384, 2), make_int3(4096, 256, 3)};   // these two fit narrow formats
    std::vector<int3> fit;
    for (const int3& c : cands)
      if (tma_smem_bytes(n_pad, c.x, c.y, c.z, bv, bi, true, true, exact) + 1024 <= (size_t)smem_optin)
        fit.push_back(c);
    if (!fit.empty()) {
      std::vector<BundleScen> B;
      {
        // each scenario's rows in kept order, then the bundles of all scenarios
        // with their work spread over every host thread
        const int nt = std::min<int>(std::max(1u, std::thread::hardware_concurrency()), 32);
        std::vector<std::vector<BundleInRow>> rows(N);
        parallel_for(N, nt, [&](int s, int) {
          const int32_t* rp = pr->row_ptr[s];
          rows[s].reserve(order[s].size());
          for (int32_t k : order[s]) {
            const int32_t i = kept[k], a0 = rp[i];
            BundleInRow br;
            br.kept = k;
            br.col = pr->col_idx[s] + a0;
            br.val = pr->val[s] + a0;
            br.len = rp[i + 1] - a0;
            br.wc = (float)(cs[s] * pr->voxel_w[i]);
            br.p = (float)pr->presc[i];
            rows[s].push_back(br);
          }
        });
        build_bundles_all(rows, &B, nt);
      }
      RowLists RB;
      RB.rec_base.assign(N + 1, 0);
      RB.nrows.assign(N, 0);
      int64_t nbc = 0, recs = 0;
      bool too_many = false;
      for (int s = 0; s < N; ++s) {
        ebase[s] = nbc;
        ecount[s] = B[s].nbc;
        nbc += B[s].nbc;
        if (B[s].nbc > (int64_t)INT32_MAX - 64) too_many = true;
        RB.nrows[s] = B[s].nb;
        RB.rec_base[s + 1] = RB.rec_base[s] + B[s].nb + 1;
        recbase_h[s] = (int)recs;
        recs += 4 * (int64_t)(B[s].nb + 1);
        n_bundles += B[s].nb;
      }
      recbase_h[N] = (int)recs;
      RB.rec.resize(RB.rec_base[N]);
      for (int s = 0; s < N; ++s)
        for (int q = 0; q <= B[s].nb; ++q) RB.rec[RB.rec_base[s] + q] = B[s].rec[(size_t)4 * q];
      if (!too_many && recs < (int64_t)INT32_MAX) {
        // CTA sizes: the caller's, else 1024 threads, or all three when autotuning.
        // A bundle's lanes are chosen as for 1024 threads whatever the size (the
        // larger register budgets of the smaller CTAs only shorten the tail), so
        // that a lane's dot product runs in the same order on every CTA size and
        // exact-sum passes give the same bits on all of them
        std::vector<int> thr_list;
        if (want_thr) thr_list = {want_thr};
        else if (autotune) thr_list = {1024, 768, 640};
        else thr_list = {1024};
        // (the chunks of a shape are the same for every CTA size: cut them once)
        for (const int3& c : fit) {
          std::vector<ChunkDesc> ch;
          std::vector<int> sc;
          if (!build_chunks(RB, ebase, N, c.x, c.y, false, kBunMinLanes, &ch, &sc, kBunKeep)) continue;
          for (int t : thr_list) {
            RingCfg rc;
            rc.cmax = c.x;
            rc.rmax = c.y;
            rc.stages = c.z;
            rc.thr = t;
            rc.chunks = ch;
            rc.scen_chunk = sc;
            ring_cfgs.push_back(std::move(rc));
          }
          if (!autotune) break;
        }
      }
      if (!ring_cfgs.empty()) {
        bundled = true;
        vpe = kBunRows;
        NE = nbc;
        rec_h.resize((size_t)recs);
        bcol.resize(N);
        bval.resize(N);
        for (int s = 0; s < N; ++s) {
          std::copy(B[s].rec.begin(), B[s].rec.end(), rec_h.begin() + recbase_h[s]);
          for (int q = 0; q < B[s].nb; ++q) rec_of_h[(size_t)s * m_act + q] = B[s].pos_of[q];
          std::vector<int4>().swap(B[s].rec);
          bcol[s] = std::move(B[s].col);
          bval[s] = std::move(B[s].val);
        }
        R = std::move(RB);
        ctas = 1;
        dp.ring_threads = ring_cfgs[0].thr;
        dp.cmax = ring_cfgs[0].cmax;
        dp.rmax = ring_cfgs[0].rmax;
        dp.stages = ring_cfgs[0].stages;
        chunks = ring_cfgs[0].chunks;
        scen_chunk = ring_cfgs[0].scen_chunk;
      }
    }
    if (!bundled && want_path == 4) {
      free_plan(P);
      set_error("bundled row path not possible for this plan (shared memory, or a bundle wider than a stage)");
      return RPT_EUNSUPPORTED;
    }
  }
  if (!bundled) {
  // ---- per-scenario row lists, sorted by decreasing length; entries permuted to match ----
  R.rec_base.assign(N + 1, 0);
  R.nrows.assign(N, 0);
  for (int s = 0; s < N; ++s) {
    const int32_t* rp = pr->row_ptr[s];
    std::stable_sort(order[s].begin(), order[s].end(), [&](int32_t a, int32_t b) {
      return rp[kept[a] + 1] - rp[kept[a]] > rp[kept[b] + 1] - rp[kept[b]];
    });
    R.nrows[s] = (int)order[s].size();
    R.rec_base[s + 1] = R.rec_base[s] + R.nrows[s] + 1;
  }
  R.rec.resize(R.rec_base[N]);
  col_h.assign((size_t)NNZp, 0);
  val_h.assign((size_t)NNZp, 0.f);
  {
    // streaming-path plans store rows lane-interleaved (interleave_row)
    const bool interleave = (want_path == 3);
    auto fill = [&](int s) {
      const int32_t* rp = pr->row_ptr[s];
      int4* out = &R.rec[R.rec_base[s]];
      int32_t pos = 0;
      std::vector<int32_t> lc;
      std::vector<float> lv;
      BankScratch bb;
      for (int q = 0; q < R.nrows[s]; ++q) {
        const int k = order[s][q];
        const int32_t a = rp[kept[k]], len = rp[kept[k] + 1] - a;
        const float wc = (float)(cs[s] * pr->voxel_w[kept[k]]);
        const float pp = (float)pr->presc[kept[k]];
        int4 r4;
        r4.x = pos;
        std::memcpy(&r4.y, &wc, 4);
        std::memcpy(&r4.z, &pp, 4);
        r4.w = k;
        out[q] = r4;
        const int32_t plen = (len + 3) & ~3;
        lc.assign(plen, 0);
        lv.assign(plen, 0.f);
        std::memcpy(lc.data(), pr->col_idx[s] + a, sizeof(int32_t) * len);
        std::memcpy(lv.data(), pr->val[s] + a, sizeof(float) * len);
        bank_balance(lc.data(), lv.data(), len, interleave ? stream_lanes(plen) : lanes_for(plen, min_lanes), bb);
        if (!interleave) {
          std::memcpy(&col_h[base[s] + pos], lc.data(), sizeof(int32_t) * plen);
          std::memcpy(&val_h[base[s] + pos], lv.data(), sizeof(float) * plen);
        } else {
          interleave_row(lc.data(), lv.data(), plen, stream_lanes(plen), &col_h[base[s] + pos],
                         &val_h[base[s] + pos]);
        }
        pos += plen;
      }
      out[R.nrows[s]] = make_int4(pos, 0, 0, 0);
    };
    parallel_for(N, std::min<int>(std::max(1u, std::thread::hardware_concurrency()), 32),
                 [&](int s, int) { fill(s); });
  }
  // ---- work decomposition: register-direct row blocks (default) or bulk-copy ring ----
  const double per_lane = 4.0;   // register path: per-row overhead per lane, in entries
  if (want_path == 3) {
    dp.cmax = std::max(16, (opts && opts->chunk_entries > 0) ? opts->chunk_entries : 1536) & ~15;
    dp.rmax = std::max(1, (opts && opts->chunk_rows > 0) ? opts->chunk_rows : 128);
    dp.stages = 0;
    ctas = 1;
    if (stream_smem_bytes(n_pad, dp.rmax, true) + 1024 <= (size_t)smem_optin)
      use_stream = build_chunks(R, base, N, dp.cmax, dp.rmax, true, min_lanes, &chunks, &scen_chunk);
    if (!use_stream) {
      free_plan(P);
      set_error("streaming row path not possible for this plan (shared memory)");
      return RPT_EUNSUPPORTED;
    }
  } else if (want_path != 1) {
    ctas = (opts && opts->ctas_per_sm > 0) ? opts->ctas_per_sm : 1;
    // ring configurations {entries per stage, rows per stage, stages}: the
    // caller's, else the default followed by smaller ones for wide plans
    // (the spot vector and the accumulator share the shared memory with the ring)
    std::vector<int3> cands = ring_override(opts, 6144, 512, 3);
    if (cands.empty())
      cands = {make_int3(6144, 512, 3), make_int3(8192, 512, 2), make_int3(4096, 512, 4),
               make_int3(4096, 512, 3), make_int3(4096, 512, 2), make_int3(3072, 256, 3),
               make_int3(3072, 256, 2), make_int3(2048, 256, 4), make_int3(2048, 256, 2)};
    for (const int3& c : cands) {
      if (tma_smem_bytes(n_pad, c.x, c.y, c.z, bv, bi, true) + 1024 > (size_t)smem_optin) continue;
      RingCfg rc;
      rc.cmax = c.x;
      rc.rmax = c.y;
      rc.stages = c.z;
      if (!build_chunks(R, base, N, rc.cmax, rc.rmax, false, min_lanes, &rc.chunks, &rc.scen_chunk)) continue;
      ring_cfgs.push_back(std::move(rc));
      if (!autotune) break;   // first that fits
    }
    if (!ring_cfgs.empty()) {
      use_tma = true;
      dp.cmax = ring_cfgs[0].cmax;
      dp.rmax = ring_cfgs[0].rmax;
      dp.stages = ring_cfgs[0].stages;
      chunks = ring_cfgs[0].chunks;
      scen_chunk = ring_cfgs[0].scen_chunk;
    }
    if (!use_tma && want_path == 2) {
      free_plan(P);
      set_error("bulk-copy row path not possible for this plan (shared memory, or a row longer than a stage)");
      return RPT_EUNSUPPORTED;
    }
  }
  dyn = use_tma || use_stream;   // chunk queues
  if (dyn) {
    dp.path = use_tma ? 1 : 2;
    dp.grid = P->sm_count * ctas;
    dp.nblocks = dp.grid * N;          // one slot per (CTA, scenario)
    dp.slot_cap = dp.grid;
  } else {
    dp.path = 0;
    ctas = (opts && opts->ctas_per_sm > 0) ? opts->ctas_per_sm : 2;
    double total = 0.0;
    for (int s = 0; s < N; ++s) {
      const int4* r = &R.rec[R.rec_base[s]];
      for (int q = 0; q < R.nrows[s]; ++q) total += row_cost(r[q + 1].x - r[q].x, per_lane, min_lanes);
    }
    const double target = std::max(1.0, total / (double)(P->sm_count * ctas));
    for (int s = 0; s < N; ++s) {
      const int4* r = &R.rec[R.rec_base[s]];
      blk_first[s] = (int)blocks.size();
      // runs of equal lanes-per-row, each cut into blocks of about `target` cost
      int q = 0;
      while (q < R.nrows[s]) {
        const int g0 = lanes_for(r[q + 1].x - r[q].x, min_lanes);
        int q1 = q;
        double run = 0.0;
        while (q1 < R.nrows[s] && lanes_for(r[q1 + 1].x - r[q1].x, min_lanes) == g0) {
          run += row_cost(r[q1 + 1].x - r[q1].x, per_lane, min_lanes);
          ++q1;
        }
        const int nb = std::max(1, (int)std::lround(run / target));
        double acc = 0.0, goal = run / nb;
        int qb = q;
        for (int k = q; k < q1; ++k) {
          acc += row_cost(r[k + 1].x - r[k].x, per_lane, min_lanes);
          if (acc >= goal - 1e-9 && (int)blocks.size() - blk_first[s] < 1 << 30) {
            blocks.push_back(make_int4(s, qb, k + 1, g0));
            qb = k + 1;
            acc = 0.0;
          }
        }
        if (qb < q1) blocks.push_back(make_int4(s, qb, q1, g0));
        q = q1;
      }
      if ((int)blocks.size() == blk_first[s]) blocks.push_back(make_int4(s, 0, 0, 1));   // empty scenario
    }
    blk_first[N] = (int)blocks.size();
    dp.nblocks = (int)blocks.size();
    dp.grid = dp.nblocks;
    dp.slot_cap = 1;
    for (int s = 0; s < N; ++s) dp.slot_cap = std::max(dp.slot_cap, blk_first[s + 1] - blk_first[s]);
  }
    NE = NNZp;
    ebase = base;
    ecount = pnnz;
    rec_h = R.rec;
    recbase_h = R.rec_base;
    for (int s = 0; s < N; ++s)
      for (int q = 0; q < R.nrows[s]; ++q) rec_of_h[(size_t)s * m_act + R.rec[R.rec_base[s] + q].w] = q;
  }
  if (bundled) {
    dyn = true;
    dp.path = 3;
    dp.grid = P->sm_count * ctas;
    dp.nblocks = dp.grid * N;
    dp.slot_cap = dp.grid;
  }
  // slot lists: static for the register path (block b of scenario s), written
  // by the kernel for the bulk-copy path
  std::vector<int> slot_count(N, 0), slot_list((size_t)N * dp.slot_cap, 0);
  if (!dyn)
    for (int s = 0; s < N; ++s) {
      slot_count[s] = blk_first[s + 1] - blk_first[s];
      for (int k = 0; k < slot_count[s]; ++k) slot_list[(size_t)s * dp.slot_cap + k] = blk_first[s] + k;
    }
  std::vector<float> diag_h((size_t)N * n);
  for (int s = 0; s < N; ++s)
    for (int j = 0; j < n; ++j) diag_h[(size_t)s * n + j] = (float)(cs[s] * chk[s].diag[j]);

  const clock::time_point t_host1 = clock::now();
  // ---- device memory ----
  // entry arrays are padded so that 16-entry aligned bulk copies stay inside them
  constexpr int64_t kPad = 64;
  Alloc A{P, (opts && opts->device_mem_cap > 0) ? (size_t)opts->device_mem_cap : 0};
  int64_t* d_base = A.get<int64_t>(N);
  int32_t* d_col32 = A.get<int32_t>(NE + kPad);            // replaced by 16-bit indices if requested
  float* d_val32 = A.get<float>((NE + kPad) * vpe);        // replaced by quantised values if requested
  int4* d_rec = A.get<int4>(rec_h.size());
  int* d_recbase = A.get<int>(N + 1);
  size_t chunk_cap = chunks.size();
  for (const RingCfg& rc : ring_cfgs) chunk_cap = std::max(chunk_cap, rc.chunks.size());
  ChunkDesc* d_chunks = dyn ? A.get<ChunkDesc>(chunk_cap) : nullptr;
  int* d_scen_chunk = dyn ? A.get<int>(N + 1) : nullptr;
  int* d_qnext = dyn ? A.get<int>(N) : nullptr;
  unsigned char* d_visited = dyn ? A.get<unsigned char>((size_t)N * dp.grid) : nullptr;
  int* d_slot_count = A.get<int>(N);
  int* d_slot_list = A.get<int>(slot_list.size());
  double* d_objs = A.get<double>(N);
  unsigned int* d_done = A.get<unsigned int>(1);
  P->err = A.get<int>(1);
  P->diag = A.get<float>(diag_h.size());
  int4* d_blocks = dyn ? nullptr : A.get<int4>(blocks.size());
  P->rec_of = A.get<int>((size_t)N * m_act);
  P->lb = A.get<double>((size_t)G * n);
  P->ub = A.get<double>((size_t)G * n);
  const size_t Nn = (size_t)N * n;
  P->x = A.get<double>(Nn);
  P->r = A.get<double>(Nn);
  P->p = A.get<double>(Nn);
  P->u = A.get<double>(Nn);
  P->y = A.get<double>(Nn);
  P->d = A.get<double>(Nn);
  P->dprev = A.get<double>(Nn);
  P->q = A.get<double>(Nn);
  P->dinv = A.get<double>(Nn);
  P->z = A.get<double>((size_t)G * n);
  P->znew = A.get<double>((size_t)G * n);
  P->uact = A.get<int>(N);
  P->v32 = A.get<float>((size_t)N * n_pad);
  P->vz32 = A.get<float>(n_pad);
  // partial slots: float (paths 1-3) or 64-bit fixed point (bundled path), n_pad each
  P->partial = A.get<float>((size_t)dp.nblocks * n_pad * 2);
  int* d_fexp = A.get<int>(N);
  double* d_kbound = A.get<double>(2 * (size_t)N);
  P->objp = A.get<double>(dp.nblocks);
  P->gam = A.get<double>(N);
  P->tol = A.get<double>(N);
  P->r0n = A.get<double>(N);
  P->alpha = A.get<double>(N);
  P->gprev = A.get<double>(N);
  P->aprev = A.get<double>(N);
  P->cgi = A.get<int>(N);
  P->beta = A.get<double>(N);
  P->bb_step = A.get<double>(N);
  P->act = A.get<int>(N);
  P->act_next = A.get<int>(N);
  P->cgcnt = A.get<int>(N);
  P->cnt_s = A.get<unsigned int>(N);
  P->dots = A.get<double>((size_t)N * P->nchunk * 4);
  P->vpart = A.get<double>((size_t)(N + G) * P->nchunk * 8);
  P->g = A.get<double>(n);
  P->xt = A.get<double>(n);
  P->xp = A.get<double>(n);
  P->ctl = A.get<Ctl>(1);
  if (A.err != cudaSuccess) {
    free_plan(P);
    return cuda_fail(A.err, "device allocation");
  }
  if ((e = cudaMallocHost(&P->ctl_host, sizeof(Ctl)))) {
    free_plan(P);
    return cuda_fail(e, "pinned allocation");
  }
  if ((e = cudaEventCreate(&P->ev0)) || (e = cudaEventCreate(&P->ev1))) {
    free_plan(P);
    return cuda_fail(e, "event");
  }
  cudaStream_t st = P->stream;
#define RPT_CP(dst, src, bytes)                                                            \
  do {                                                                                     \
    if ((bytes) > 0 && (e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st))) { \
      free_plan(P);                                                                        \
      return cuda_fail(e, "upload");                                                       \
    }                                                                                      \
  } while (0)
  RPT_CP(d_base, ebase.data(), N * sizeof(int64_t));
  if (bundled) {
    for (int s = 0; s < N; ++s) {
      RPT_CP(d_col32 + ebase[s], bcol[s].data(), bcol[s].size() * sizeof(int32_t));
      RPT_CP(d_val32 + ebase[s] * vpe, bval[s].data(), bval[s].size() * sizeof(float));
    }
  } else {
    RPT_CP(d_col32, col_h.data(), (size_t)NE * sizeof(int32_t));
    RPT_CP(d_val32, val_h.data(), (size_t)NE * vpe * sizeof(float));
  }
  RPT_CP(d_rec, rec_h.data(), rec_h.size() * sizeof(int4));
  RPT_CP(d_recbase, recbase_h.data(), (N + 1) * sizeof(int));
  RPT_CP(P->rec_of, rec_of_h.data(), rec_of_h.size() * sizeof(int));
  P->rec_of_host = rec_of_h;
  if (!dyn) RPT_CP(d_blocks, blocks.data(), blocks.size() * sizeof(int4));
  RPT_CP(P->diag, diag_h.data(), diag_h.size() * sizeof(float));
  if (dyn) {
    RPT_CP(d_chunks, chunks.data(), chunks.size() * sizeof(ChunkDesc));
    RPT_CP(d_scen_chunk, scen_chunk.data(), (N + 1) * sizeof(int));
  }
  RPT_CP(d_slot_count, slot_count.data(), N * sizeof(int));
  RPT_CP(d_slot_list, slot_list.data(), slot_list.size() * sizeof(int));
  RPT_CP(P->lb, lb.data(), lb.size() * sizeof(double));
  RPT_CP(P->ub, ub.data(), ub.size() * sizeof(double));
#undef RPT_CP
  if ((e = cudaMemsetAsync(P->cnt_s, 0, sizeof(unsigned int) * N, st)) ||
      (e = cudaMemsetAsync(P->err, 0, sizeof(int), st)) ||
      (e = cudaMemsetAsync(d_done, 0, sizeof(unsigned int), st)) ||
      (e = cudaMemsetAsync(d_objs, 0, sizeof(double) * N, st)) ||
      (dyn && (e = cudaMemsetAsync(d_qnext, 0, sizeof(int) * N, st))) ||
      (dyn && (e = cudaMemsetAsync(d_visited, 0, (size_t)N * dp.grid, st))) ||
      (e = cudaMemsetAsync(d_col32 + NE, 0, sizeof(int32_t) * kPad, st)) ||
      (e = cudaMemsetAsync(d_val32 + NE * vpe, 0, sizeof(float) * kPad * vpe, st)) ||
      (e = cudaMemsetAsync(P->ctl, 0, sizeof(Ctl), st)) ||
      (e = cudaMemsetAsync(d_fexp, 0, sizeof(int) * N, st)) ||
      (e = cudaMemsetAsync(d_kbound, 0, sizeof(double) * 2 * N, st)) ||
      (e = cudaMemsetAsync(P->v32, 0, sizeof(float) * (size_t)N * n_pad, st)) ||
      (e = cudaMemsetAsync(P->vz32, 0, sizeof(float) * n_pad, st))) {
    free_plan(P);
    return cuda_fail(e, "memset");
  }
  dp.nnz_base = d_base;
  dp.blocks = d_blocks;
  dp.rowrec = d_rec;
  dp.rec_base = d_recbase;
  dp.chunks = d_chunks;
  dp.scen_chunk = d_scen_chunk;
  dp.qnext = d_qnext;
  dp.visited = d_visited;
  dp.slot_count = d_slot_count;
  dp.slot_list = d_slot_list;
  dp.objs = d_objs;
  dp.objp = P->objp;
  dp.done_ctr = d_done;
  dp.err = P->err;
  dp.col32 = d_col32;
  dp.val32 = d_val32;
  dp.acc64 = (bundled && exact) ? 1 : 0;
  dp.fexp = d_fexp;
  dp.kbound = d_kbound;
  // ---- quantised values / narrow indices ----
  const int qgrid = std::max(1, P->sm_count * 8), qblock = 256;
  if (pr->value_format != RPT_F32) {
    float* scale = A.get<float>((size_t)N * n_pad);
    unsigned int* mx = A.get<unsigned int>(n_pad);
    void* q = pr->value_format == RPT_BF16 ? (void*)A.get<__nv_bfloat16>((NE + kPad) * vpe)
                                           : (void*)A.get<__nv_fp8_e4m3>((NE + kPad) * vpe);
    if (A.err != cudaSuccess) {
      free_plan(P);
      return cuda_fail(A.err, "device allocation");
    }
    const float fmt_max = pr->value_format == RPT_BF16 ? 1.0f : 448.0f;
    for (int s = 0; s < N && e == cudaSuccess; ++s) {
      e = cudaMemsetAsync(mx, 0, sizeof(unsigned int) * n_pad, st);
      if (e) break;
      const int sh = vpe == 4 ? 2 : 0;   // value e of the scenario belongs to stored entry e >> sh
      if (ecount[s] > 0)
        k_colmax<<<qgrid, qblock, 0, st>>>(d_val32 + ebase[s] * vpe, d_col32 + ebase[s], ecount[s] * vpe, sh, mx);
      k_scales<<<(n_pad + 255) / 256, 256, 0, st>>>(mx, n, n_pad, fmt_max, scale + (size_t)s * n_pad);
      if (ecount[s] > 0) {
        if (pr->value_format == RPT_BF16)
          k_quantise<__nv_bfloat16><<<qgrid, qblock, 0, st>>>(d_val32 + ebase[s] * vpe, d_col32 + ebase[s],
                                                              ecount[s] * vpe, sh, scale + (size_t)s * n_pad,
                                                              (__nv_bfloat16*)q + ebase[s] * vpe);
        else
          k_quantise<__nv_fp8_e4m3><<<qgrid, qblock, 0, st>>>(d_val32 + ebase[s] * vpe, d_col32 + ebase[s],
                                                              ecount[s] * vpe, sh, scale + (size_t)s * n_pad,
                                                              (__nv_fp8_e4m3*)q + ebase[s] * vpe);
      }
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      free_plan(P);
      return cuda_fail(e, "quantise");
    }
    dp.colscale = scale;
    if (pr->value_format == RPT_BF16) dp.valbf = (const __nv_bfloat16*)q;
    else dp.val8 = (const __nv_fp8_e4m3*)q;
    dp.val32 = nullptr;
  }
  if (pr->index_width == 16) {
    uint16_t* c16 = A.get<uint16_t>(NE + kPad);
    if (A.err != cudaSuccess) {
      free_plan(P);
      return cuda_fail(A.err, "device allocation");
    }
    k_to_u16<<<qgrid, qblock, 0, st>>>(d_col32, NE + kPad, c16);
    if ((e = cudaGetLastError())) {
      free_plan(P);
      return cuda_fail(e, "index conversion");
    }
    dp.col16 = c16;
    dp.col32 = nullptr;
  }
  if ((e = cudaStreamSynchronize(st))) {
    free_plan(P);
    return cuda_fail(e, "plan upload");
  }
  // release the float32 / int32 staging copies that the stored format replaced
  auto release = [&](void* ptr) {
    auto it = std::find(P->allocs.begin(), P->allocs.end(), ptr);
    if (it != P->allocs.end()) {
      cudaFree(ptr);
      P->allocs.erase(it);
    }
  };
  if (pr->value_format != RPT_F32) release(d_val32);
  if (pr->index_width == 16) release(d_col32);
  if (dp.acc64) {
    // bounds of the fixed-point accumulation, from the stored values
    double* kc = nullptr;
    if ((e = cudaMalloc(&kc, sizeof(double) * 2 * n_pad))) {
      free_plan(P);
      return cuda_fail(e, "device allocation");
    }
    e = bundle_bounds(dp, kc, kc + n_pad, d_kbound, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(kc);
    if (e != cudaSuccess) {
      free_plan(P);
      return cuda_fail(e, "fixed-point bounds");
    }
  }
  if ((e = rowpass_prepare(dp))) {
    free_plan(P);
    return cuda_fail(e, "kernel attributes");
  }
  // ---- statistics ----
  // default penalty rho = 2 mean_s tr(A~_s^T A~_s) / n, per group on the group's
  // own scenarios and spot count; the plan's figure on all problems stacked
  double tr = 0.0;
  int n_all = 0;
  P->grp_rho.assign(G, 0.0);
  P->grp_n.assign(G, n);
  P->grp_const = gconst;
  for (int g = 0; g < G; ++g) {
    double t = 0.0;
    for (int s = g * Ns; s < (g + 1) * Ns; ++s) t += cs[s] * chk[s].trace;
    if (U) P->grp_n[g] = U->n_g[g];
    P->grp_rho[g] = 2.0 * (t / Ns) / P->grp_n[g];
    tr += t;
    n_all += P->grp_n[g];
  }
  rpt_plan_stats& S = P->stats;
  S.m = m;
  S.n = n_all;
  S.N = Ns;
  S.m_active = m_act;
  S.nnz = NNZ;
  // values and indices, plus one 4-byte row offset per stored row (the records'
  // weight and prescription are counted by the kernels' algorithmic bytes)
  S.matrix_bytes = bundled ? NE * (int64_t)(bi + kBunRows * bv) + (n_bundles + N) * 4
                           : NNZ * (int64_t)(bi + bv) + (int64_t)(R.rec_base[N]) * 4;
  S.bundles = bundled ? n_bundles : 0;
  S.block_cols = bundled ? NE : 0;
  S.bundle_fill = (bundled && NE > 0) ? (double)NNZ / (double)(kBunRows * NE) : 0.0;
  S.exact_sums = dp.acc64;
  S.ring_threads = bundled ? dp.ring_threads : 0;
  S.value_format = pr->value_format;
  S.index_width = pr->index_width;
  S.row_blocks = dp.nblocks;
  S.sm_count = P->sm_count;
  S.default_rho = 2.0 * (tr / Ns) / n_all;
  S.const_term = const_term;
  S.row_path = dp.path + 1;
  S.min_lanes = min_lanes;
  S.chunk_entries = dp.path >= 1 ? dp.cmax : 0;
  S.chunk_rows = dp.path >= 1 ? dp.rmax : 0;
  S.stages = (dp.path == 1 || dp.path == 3) ? dp.stages : 0;
  S.autotuned = 0;
  S.autotune_ms = 0.0;
  if ((e = cudaStreamSynchronize(st))) {
    free_plan(P);
    return cuda_fail(e, "sync");
  }
  const clock::time_point t_dev1 = clock::now();
  S.layout_seconds = secs(t_begin, t_host0) + secs(t_dev0, t_host1);
  S.device_seconds = secs(t_host0, t_dev0) + secs(t_host1, t_dev1);
  S.autotune_seconds = 0.0;
  // ---- autotuning: time every fitting ring configuration on this plan, keep the fastest ----
  if ((use_tma || bundled) && ring_cfgs.size() > 1) {
    std::vector<double> ms(ring_cfgs.size(), 1e30);
    auto apply = [&](const RingCfg& rc) -> cudaError_t {
      cudaError_t ee = cudaMemcpyAsync(d_chunks, rc.chunks.data(), rc.chunks.size() * sizeof(ChunkDesc),
                                       cudaMemcpyHostToDevice, st);
      if (ee == cudaSuccess)
        ee = cudaMemcpyAsync(d_scen_chunk, rc.scen_chunk.data(), (N + 1) * sizeof(int), cudaMemcpyHostToDevice, st);
      if (ee == cudaSuccess) ee = cudaStreamSynchronize(st);
      P->dp.cmax = rc.cmax;
      P->dp.rmax = rc.rmax;
      P->dp.stages = rc.stages;
      if (bundled) P->dp.ring_threads = rc.thr;
      if (ee == cudaSuccess) ee = rowpass_prepare(P->dp);
      return ee;
    };
    // time on a nonzero vector (a zero vector makes every scatter add zeros)
    {
      std::vector<float> ones((size_t)N * n_pad, 1.0f);
      if ((e = cudaMemcpy(P->v32, ones.data(), sizeof(float) * ones.size(), cudaMemcpyHostToDevice))) {
        free_plan(P);
        return cuda_fail(e, "autotune");
      }
    }
    // every configuration timed over 4 launches, then the four fastest again over
    // 10 launches each, keeping each one's best (one short timing per
    // configuration let clock and queue noise pick a slower ring)
    auto time_cfg = [&](size_t c, int reps) -> int {
      if ((e = apply(ring_cfgs[c]))) return cuda_fail(e, "autotune");
      double t = 0.0, by = 0.0;
      if (int rc = profile_row_pass(P, kNormal, reps, &t, &by)) return rc;
      ms[c] = std::min(ms[c], t);
      return RPT_OK;
    };
    for (size_t c = 0; c < ring_cfgs.size(); ++c)
      if (int rc = time_cfg(c, 4)) {
        free_plan(P);
        return rc;
      }
    std::vector<size_t> order(ring_cfgs.size());
    for (size_t c = 0; c < order.size(); ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return ms[a] < ms[b]; });
    for (size_t k = 0; k < std::min<size_t>(4, order.size()); ++k)
      if (int rc = time_cfg(order[k], 10)) {
        free_plan(P);
        return rc;
      }
    const size_t best = (size_t)(std::min_element(ms.begin(), ms.end()) - ms.begin());
    if ((e = apply(ring_cfgs[best]))) {
      free_plan(P);
      return cuda_fail(e, "autotune");
    }
    S.chunk_entries = ring_cfgs[best].cmax;
    S.chunk_rows = ring_cfgs[best].rmax;
    S.stages = ring_cfgs[best].stages;
    S.ring_threads = bundled ? ring_cfgs[best].thr : 0;
    S.autotuned = (int32_t)ring_cfgs.size();
    S.autotune_ms = ms[best];
    S.autotune_seconds = secs(t_dev1, clock::now());
  }
  *out = reinterpret_cast<rpt_plan*>(P);
  return RPT_OK;
}

template <typename F>
int guarded(F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    set_error("out of host memory");
    return RPT_ENOMEM;
  } catch (...) {
    set_error("internal error");
    return RPT_ECUDA;
  }
}

Plan* as_plan(rpt_plan* p) { return reinterpret_cast<Plan*>(p); }

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace rpt

using namespace rpt;

extern "C" {

void rpt_admm_params_default(rpt_admm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->rho = 0.0;
  p->rho_scale = 1.0;
  p->eps_abs = 1e-4;
  p->eps_rel = 1e-4;
  p->tol_obj = HUGE_VAL;
  p->max_iter = 5000;
  p->bb_mode = RPT_BB_PAPER;
  p->bb_kappa = 10.0;
  p->z_mode = RPT_Z_STD;
  p->cg_max = 50;
  p->cg_theta = 0.15;
  p->cg_eta0 = 1e-2;
  p->cg_floor_rel = 1e-6;
  p->use_graph = 1;
  p->check_every = 1;
  p->resume = 0;
  p->cg_precond = 1;
  p->subproblem = RPT_SUB_CG;
  p->trace = 0;
  p->bb_per_scenario = 0;
  p->f_target = 0.0;
}

void rpt_pgd_params_default(rpt_pgd_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->alpha = 0.0;
  p->beta = 1e-4;
  p->gamma = 0.5;
  p->tol_rel_df = 1e-5;
  p->f_target = 0.0;
  p->max_iter = 20000;
  p->max_trials = 30;
  p->use_graph = 1;
}

int rpt_plan_create(const rpt_problem* prob, const rpt_device_opts* opts, rpt_plan** out) {
  return guarded([&] { return create_plan(prob, opts, out); });
}

int rpt_plans_create_batched(int32_t n_plans, const rpt_problem* const* probs, const rpt_device_opts* opts,
                             rpt_plan** out) {
  if (!out || !probs || n_plans < 1) {
    set_error("n_plans >= 1 and non-null probs and out needed");
    return RPT_EINVAL;
  }
  return guarded([&] {
    // every problem valid on its own (a column index is checked against its own
    // problem's spot count, before the stacking offsets hide it)
    for (int k = 0; k < n_plans; ++k) {
      const rpt_problem* q = probs[k];
      if (!q || q->m < 1 || q->n < 1 || q->N < 1 || !q->row_ptr || !q->col_idx || !q->val || !q->voxel_w ||
          !q->presc) {
        set_error("problem " + std::to_string(k) + ": null or empty");
        return RPT_EINVAL;
      }
      for (int s = 0; s < q->N; ++s) {
        if (!q->row_ptr[s] || (q->row_ptr[s][q->m] > 0 && (!q->col_idx[s] || !q->val[s]))) {
          set_error("problem " + std::to_string(k) + ": null CSR array for scenario " + std::to_string(s));
          return RPT_EINVAL;
        }
        ScenarioCheck chk;
        check_scenario(q, s, &chk);
        if (!chk.err.empty()) {
          set_error("problem " + std::to_string(k) + ": " + chk.err);
          return RPT_EINVAL;
        }
      }
    }
    batch::Units un;
    std::string err;
    int rc = batch::stack_units(n_plans, probs, &un, &err);
    if (rc != RPT_OK) {
      set_error(err);
      return rc;
    }
    rpt_plan* h = nullptr;
    rc = create_plan(&un.view, opts, &h, &un);
    if (rc != RPT_OK) return rc;
    as_plan(h)->batch_col_off = un.col_off;
    *out = h;
    return RPT_OK;
  });
}

int rpt_plan_batch_query(const rpt_plan* plan, int32_t* n_plans, int32_t* col_offsets) {
  if (!plan || !n_plans) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  const Plan* P = reinterpret_cast<const Plan*>(plan);
  const bool batched = !P->batch_col_off.empty();
  *n_plans = batched ? (int32_t)P->batch_col_off.size() - 1 : 1;
  if (col_offsets) {
    if (batched) {
      for (size_t k = 0; k < P->batch_col_off.size(); ++k) col_offsets[k] = P->batch_col_off[k];
    } else {
      col_offsets[0] = 0;
      col_offsets[1] = P->dp.n;
    }
  }
  return RPT_OK;
}

int rpt_admm_bb_solve_batched(rpt_plan* plan, const rpt_admm_params* params, double* const* x_out,
                              rpt_solve_info* info, rpt_solve_info* plan_info) {
  if (!plan || !params || !x_out) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  Plan* P = as_plan(plan);
  const int G = P->dp.G, n = P->dp.n;
  for (int k = 0; k < G; ++k)
    if (!x_out[k]) {
      set_error("x_out[" + std::to_string(k) + "] is NULL");
      return RPT_EINVAL;
    }
  return guarded([&] {
    DeviceScope ds(P->device);
    std::vector<double> z((size_t)G * n);
    const int rc = admm_solve(P, params, nullptr, nullptr, z.data(), info, nullptr, plan_info);
    if (rc != RPT_OK && rc != RPT_NOT_CONVERGED && !(rc == RPT_DIVERGED && G > 1)) return rc;
    for (int k = 0; k < G; ++k)
      std::memcpy(x_out[k], z.data() + (size_t)k * n, sizeof(double) * (size_t)P->grp_n[k]);
    return rc;
  });
}

int rpt_plan_set_weights(rpt_plan* plan, const double* voxel_w, const double* presc) {
  if (!plan || !voxel_w || !presc) {
    set_error("rpt_plan_set_weights: null argument");
    return RPT_EINVAL;
  }
  Plan* P = as_plan(plan);
  if (int rc = refuse_batched(P, "rpt_plan_set_weights")) return rc;
  const int m = P->dp.m, N = P->dp.N, n = P->dp.n, m_act = P->dp.m_act, n_pad = P->dp.n_pad;
  for (int i = 0; i < m; ++i)
    if (!std::isfinite(voxel_w[i]) || voxel_w[i] < 0 || !std::isfinite(presc[i]) || presc[i] < 0) {
      set_error("rpt_plan_set_weights: voxel_w[" + std::to_string(i) + "] or presc not finite or negative");
      return RPT_EINVAL;
    }
  return guarded([&] {
    DeviceScope ds(P->device);
    cudaStream_t st = P->stream;
    std::vector<double> wk(m_act), pk(m_act);
    double wmax = 0.0;
    for (int k = 0; k < m_act; ++k) {
      wk[k] = voxel_w[P->kept_rows[k]];
      pk[k] = presc[P->kept_rows[k]];
      wmax = std::max(wmax, wk[k]);
    }
    double* d = nullptr;                     // [wk | pk] then the fixed-point sums
    cudaError_t e = cudaMalloc(&d, sizeof(double) * (2 * (size_t)m_act + n_pad));
    if (e != cudaSuccess) return cuda_fail(e, "rpt_plan_set_weights");
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(d + 2 * (size_t)m_act);
    e = cudaMemcpyAsync(d, wk.data(), sizeof(double) * m_act, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + m_act, pk.data(), sizeof(double) * m_act, cudaMemcpyHostToDevice, st);
    std::vector<unsigned long long> h(n_pad);
    std::vector<float> diag((size_t)N * n);
    double tr = 0.0;
    for (int s = 0; s < N && e == cudaSuccess; ++s) {
      // sum_i c_s w_i a_ij^2 <= c_s max(w) max_j sum_i a_ij^2: scale so that 4x that stays below 2^62
      const double bound = P->scen_c[s] * wmax * P->colsq_max[s] * 4.0;
      int ex = 0;
      if (bound > 0.0) std::frexp(bound, &ex);
      const double scale = std::ldexp(1.0, 60 - ex);
      e = plan_reweight(P->dp, s, P->scen_c[s], d, d + m_act, scale, acc, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), acc, sizeof(unsigned long long) * n_pad,
                                                cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      for (int j = 0; j < n; ++j) {   // each sum is exact; the trace adds them in column order
        const double dj = (double)(long long)h[j] / scale;
        diag[(size_t)s * n + j] = (float)dj;
        tr += dj;
      }
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(P->diag, diag.data(), sizeof(float) * diag.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && P->dp.path == 3) e = bundle_bounds(P->dp, d, d + n_pad, const_cast<double*>(P->dp.kbound), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "rpt_plan_set_weights");
    // the constant of Eq. 2 in the order plan creation sums it
    double c = 0.0;
    for (int32_t i : P->dropped_rows)
      for (int s = 0; s < N; ++s) c += P->scen_c[s] * voxel_w[i] * presc[i] * presc[i];
    for (int s = 0; s < N; ++s)
      for (int32_t k : P->empty_kept[s]) {
        const int32_t i = P->kept_rows[k];
        c += P->scen_c[s] * voxel_w[i] * presc[i] * presc[i];
      }
    P->stats.const_term = c;
    P->stats.default_rho = 2.0 * (tr / N) / n;
    P->grp_const.assign(1, c);
    P->grp_rho.assign(1, P->stats.default_rho);
    P->lipschitz = 0.0;
    P->chol_ready = false;
    P->chol_con = false;
    return RPT_OK;
  });
}

void rpt_plan_destroy(rpt_plan* plan) {
  if (plan) free_plan(as_plan(plan));
}

int rpt_plan_query(const rpt_plan* plan, rpt_plan_stats* out) {
  if (!plan || !out) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  *out = reinterpret_cast<const Plan*>(plan)->stats;
  return RPT_OK;
}

int rpt_admm_bb_solve(rpt_plan* plan, const rpt_admm_params* params, const double* z0,
                      const double* y0, double* x_out, rpt_solve_info* info) {
  if (!plan || !params) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  return guarded([&] {
    if (int rc = refuse_batched(as_plan(plan), "rpt_admm_bb_solve")) return rc;
    DeviceScope ds(as_plan(plan)->device);
    return admm_solve(as_plan(plan), params, z0, y0, x_out, info);
  });
}

int rpt_pgd_solve(rpt_plan* plan, const rpt_pgd_params* params, const double* x0, double* x_out,
                  rpt_solve_info* info) {
  if (!plan || !params) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  return guarded([&] {
    if (int rc = refuse_batched(as_plan(plan), "rpt_pgd_solve")) return rc;
    DeviceScope ds(as_plan(plan)->device);
    return pgd_solve(as_plan(plan), params, x0, x_out, info);
  });
}

int rpt_objective(rpt_plan* plan, const double* x, double* f_out, double* dose_out) {
  if (!plan || !x) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  return guarded([&] {
    if (int rc = refuse_batched(as_plan(plan), "rpt_objective")) return rc;
    DeviceScope ds(as_plan(plan)->device);
    return op_objective(as_plan(plan), x, f_out, dose_out);
  });
}

int rpt_gradient(rpt_plan* plan, const double* x, double* g_out, double* f_out) {
  if (!plan || !x || !g_out) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  return guarded([&] {
    if (int rc = refuse_batched(as_plan(plan), "rpt_gradient")) return rc;
    DeviceScope ds(as_plan(plan)->device);
    return op_gradient(as_plan(plan), x, g_out, f_out);
  });
}

int rpt_apply_normal(rpt_plan* plan, const double* v, double rho, double* u_out) {
  if (!plan || !v || !u_out) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  return guarded([&] {
    if (int rc = refuse_batched(as_plan(plan), "rpt_apply_normal")) return rc;
    DeviceScope ds(as_plan(plan)->device);
    return op_apply_normal(as_plan(plan), v, rho, u_out);
  });
}

int rpt_profile_row_pass(rpt_plan* plan, int mode, int reps, double* ms_per_pass,
                         double* bytes_per_pass) {
  if (!plan) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  return guarded([&] {
    DeviceScope ds(as_plan(plan)->device);
    return profile_row_pass(as_plan(plan), mode, reps, ms_per_pass, bytes_per_pass);
  });
}

int rpt_state_get(rpt_plan* plan, double* z, double* x, double* y) {
  if (!plan) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  return guarded([&] {
    Plan* P = as_plan(plan);
    if (int rc = refuse_batched(P, "rpt_state_get")) return rc;
    if (!P->state_valid) {
      set_error("the plan holds no ADMM state");
      return RPT_EINVAL;
    }
    DeviceScope ds(P->device);
    const size_t Nn = (size_t)P->dp.N * P->dp.n;
    cudaError_t e = cudaSuccess;
    if (z && !e) e = cudaMemcpyAsync(z, P->z, sizeof(double) * P->dp.n, cudaMemcpyDeviceToHost, P->stream);
    if (x && !e) e = cudaMemcpyAsync(x, P->x, sizeof(double) * Nn, cudaMemcpyDeviceToHost, P->stream);
    if (y && !e) e = cudaMemcpyAsync(y, P->y, sizeof(double) * Nn, cudaMemcpyDeviceToHost, P->stream);
    if (!e) e = cudaStreamSynchronize(P->stream);
    return e ? cuda_fail(e, "state copy") : RPT_OK;
  });
}

int rpt_state_set(rpt_plan* plan, const double* z, const double* x, const double* y) {
  if (!plan || !z || !x || !y) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  return guarded([&] {
    Plan* P = as_plan(plan);
    if (int rc = refuse_batched(P, "rpt_state_set")) return rc;
    const size_t Nn = (size_t)P->dp.N * P->dp.n;
    for (int j = 0; j < P->dp.n; ++j)
      if (!std::isfinite(z[j])) {
        set_error("z has a non-finite entry");
        return RPT_EINVAL;
      }
    for (size_t i = 0; i < Nn; ++i)
      if (!std::isfinite(x[i]) || !std::isfinite(y[i])) {
        set_error("x or y has a non-finite entry");
        return RPT_EINVAL;
      }
    DeviceScope ds(P->device);
    cudaError_t e = cudaMemcpyAsync(P->z, z, sizeof(double) * P->dp.n, cudaMemcpyHostToDevice, P->stream);
    if (!e) e = cudaMemcpyAsync(P->x, x, sizeof(double) * Nn, cudaMemcpyHostToDevice, P->stream);
    if (!e) e = cudaMemcpyAsync(P->y, y, sizeof(double) * Nn, cudaMemcpyHostToDevice, P->stream);
    if (!e) e = cudaStreamSynchronize(P->stream);
    if (e) return cuda_fail(e, "state copy");
    P->state_valid = true;
    return RPT_OK;
  });
}

const char* rpt_status_string(int status) {
  switch (status) {
    case RPT_OK: return "ok";
    case RPT_NOT_CONVERGED: return "not converged (iteration cap reached)";
    case RPT_EINVAL: return "invalid argument";
    case RPT_ENOMEM: return "out of memory";
    case RPT_ECUDA: return "CUDA error";
    case RPT_TIMEOUT: return "device wait timed out";
    case RPT_DIVERGED: return "diverged (non-finite residual)";
    case RPT_EUNSUPPORTED: return "unsupported by this build";
    default: return "unknown status";
  }
}

const char* rpt_last_error(void) { return g_last_error.c_str(); }

const char* rpt_version(void) { return "librpt 0.1 (sm_103a)"; }

}  // extern "C"

extern "C" int rpt_trace_get(rpt_plan* plan, double* out, int32_t cap, int32_t* count) {
  if (!plan || !count || cap < 0) {
    rpt::set_error("rpt_trace_get: bad argument");
    return RPT_EINVAL;
  }
  rpt::Plan* P = reinterpret_cast<rpt::Plan*>(plan);
  *count = P->trace_count;
  if (!out || P->trace_count == 0) return RPT_OK;
  const int k = std::min(cap, P->trace_count);
  cudaError_t e = cudaSetDevice(P->device);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, P->trace, sizeof(double) * rpt::kTraceFields * (size_t)k, cudaMemcpyDeviceToHost,
                        P->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
  return e == cudaSuccess ? RPT_OK : rpt::cuda_fail(e, "rpt_trace_get");
}
