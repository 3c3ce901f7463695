// Cached-factor x-update (App. A; the subproblem solver of the paper): for a
// fixed rho,
//     B_s = A~_s^T A~_s + (rho/2) I
// is formed once per (plan, rho), factored (Cholesky, B_s = L L^T) and inverted
// (B_s^{-1} = L^{-T} L^{-1}); every ADMM iteration then takes
//     x_s = B_s^{-1} c_s,   c_s = A~_s^T p~ + (rho/2) z - y_s / 2
// as one dense matrix-vector product per scenario, without a pass over the
// sparse matrices.  The paper factors in double precision on the CPU; here the
// factor, its inverse and the products are FP32 on the device (the solver state
// stays FP64), which bounds the relative error of an x-update by about
// cond(B_s) * n * eps32.
//
// Forming B_s uses the sparsity: rows are taken kRB at a time in voxel order
// (neighbouring voxels share most of their spots), their union of columns U is
// built in shared memory with the dense kRB x |U| block of A~, and every nonzero
// pair sum over the block goes to the lower triangle of B_s with one global
// atomic.  Factorisation and inversion are blocked (64) right-looking
// algorithms: small diagonal-block kernels plus, for the trailing updates and
// the products of the inverse, the FP32-accurate tensor-core GEMM of
// gemm_tf32.cuh (error-compensated TF32), batched over scenarios.
#include <cmath>
#include <vector>

#include "gemm_tf32.cuh"
#include "plan.h"
#include "rowcommon.cuh"

namespace rpt {
namespace {

constexpr int kRB = 16;       // rows per outer-product block
constexpr int kUMax = 1536;   // columns a block may touch (more: the per-row path)
constexpr int kNB = 64;       // Cholesky / inverse block size
constexpr int kPB = 4;        // blocks per panel: the trailing matrix is updated once per panel (rank 256)
constexpr unsigned kFull = 0xffffffffu;

// Lower triangle of B_s (row-major n x n, zero on entry) += sum over kept rows k
// in [blockIdx.x * kRB, +kRB) of c_s w_k a_k a_k^T (A~ = diag(sqrt(c_s w)) A).
// BUN = false: CSR rows, rec_of[s][k] = position of kept row k in the row list.
// BUN = true: row bundles, rec_of[s][q] = position of the q-th bundle in creation
// (kept-row) order; the block takes kRB / 4 consecutive bundles.
template <typename VT, typename IT, bool BUN>
__global__ void __launch_bounds__(256)
k_btb(DevPlan P, int s, const int* __restrict__ rec_of, float* __restrict__ B) {
  constexpr int RPU = BUN ? kBundleRows : 1;    // rows per unit (bundle or row)
  constexpr int UPB = kRB / RPU;                // units per block
  extern __shared__ __align__(16) unsigned char smem[];
  int* map = reinterpret_cast<int*>(smem);            // [n_pad]: flag, then position in U (-1: absent)
  int* U = map + P.n_pad;                             // [kUMax] sorted union of columns
  float* D = reinterpret_cast<float*>(U + kUMax);     // [kRB][kUMax] dense block of A~
  __shared__ int rlo[UPB], rhi[UPB];
  __shared__ float rw[kRB];
  __shared__ int wsum[8];
  __shared__ int running;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int n = P.n;
  const int4* rec = P.rowrec + P.rec_base[s];
  const long long base = P.nnz_base[s];
  const VT* val = vals<VT>(P) + base * RPU;
  const IT* col = cols<IT>(P) + base;
  const float* cs = P.colscale ? P.colscale + (size_t)s * P.n_pad : nullptr;
  const int nunits = BUN ? (P.rec_base[s + 1] - P.rec_base[s]) / 4 - 1 : P.m_act;
  if (tid < UPB) {
    const int k = blockIdx.x * UPB + tid;
    const int q = k < nunits ? rec_of[(size_t)s * P.m_act + k] : -1;
    rlo[tid] = q >= 0 ? rec[q * RPU].x : 0;
    rhi[tid] = q >= 0 ? rec[(q + 1) * RPU].x : 0;
  }
  if (tid < kRB) {
    const int u = tid / RPU, r = tid % RPU;
    const int k = blockIdx.x * UPB + u;
    const int q = k < nunits ? rec_of[(size_t)s * P.m_act + k] : -1;
    const float wc = q < 0 ? 0.f
                     : BUN ? __int_as_float(reinterpret_cast<const int*>(&rec[4 * q + 1])[r])
                           : __int_as_float(rec[q].y);
    rw[tid] = sqrtf(wc);
  }
  if (tid == 0) running = 0;
  for (int j = tid; j < P.n_pad; j += blockDim.x) map[j] = 0;
  __syncthreads();
  auto entry = [&](int e, float (&a)[RPU]) {     // the unit's values at stored entry e
    if constexpr (BUN) {
      quad_v<true, VT>(val + 4 * (size_t)e, a);
    } else {
      a[0] = to_f<VT>(val[e]);
    }
  };
  for (int u = 0; u < UPB; ++u)
    for (int e = rlo[u] + tid; e < rhi[u]; e += blockDim.x) {
      float a[RPU];
      entry(e, a);
      bool nz = false;
      for (int r = 0; r < RPU; ++r) nz |= a[r] != 0.f;
      if (nz) map[(int)col[e]] = 1;
    }
  __syncthreads();
  // ordered compaction of the flags: map[c] = position in U, U[position] = c
  for (int c0 = 0; c0 < P.n_pad; c0 += blockDim.x) {
    const int c = c0 + tid;
    const int f = c < P.n_pad ? map[c] : 0;
    const unsigned bal = __ballot_sync(kFull, f != 0);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int off = running;
    for (int i = 0; i < w; ++i) off += wsum[i];
    if (c < P.n_pad) {
      const int pos = off + __popc(bal & ((1u << lane) - 1u));
      map[c] = f ? pos : -1;
      if (f && pos < kUMax) U[pos] = c;
    }
    __syncthreads();
    if (tid == 0) {
      int t = running;
      for (int i = 0; i < 8; ++i) t += wsum[i];
      running = t;
    }
    __syncthreads();
  }
  const int nu = running;
  if (nu > kUMax) {
    // rare: rows too spread out for one dense block; add each unit's pairs directly
    for (int u = 0; u < UPB; ++u) {
      const int lo = rlo[u], len = rhi[u] - rlo[u];
      const long long pairs = (long long)len * len;
      for (long long p = tid; p < pairs; p += blockDim.x) {
        const int e1 = lo + (int)(p / len), e2 = lo + (int)(p % len);
        const int c1 = (int)col[e1], c2 = (int)col[e2];
        if (c1 < c2) continue;
        float a1[RPU], a2[RPU];
        entry(e1, a1);
        entry(e2, a2);
        float v = 0.f;
        for (int r = 0; r < RPU; ++r) v += rw[u * RPU + r] * rw[u * RPU + r] * a1[r] * a2[r];
        if (cs) v *= cs[c1] * cs[c2];
        if (v != 0.f) atomicAdd(&B[(size_t)c1 * n + c2], v);
      }
    }
    return;
  }
  for (int e = tid; e < kRB * nu; e += blockDim.x) D[(e / nu) * kUMax + (e % nu)] = 0.f;
  __syncthreads();
  for (int u = 0; u < UPB; ++u)
    for (int e = rlo[u] + tid; e < rhi[u]; e += blockDim.x) {
      const int c = (int)col[e];
      float a[RPU];
      entry(e, a);
      for (int r = 0; r < RPU; ++r)
        if (a[r] != 0.f) D[(u * RPU + r) * kUMax + map[c]] = rw[u * RPU + r] * (cs ? a[r] * cs[c] : a[r]);
    }
  __syncthreads();
  // pairs a >= b of U (row U[a] >= column U[b]: the lower triangle): a warp takes
  // a row a (its D column broadcast), its lanes the columns b <= a
  const int nwarps = blockDim.x >> 5;
  for (int a = w; a < nu; a += nwarps) {
    float da[kRB];
#pragma unroll
    for (int r = 0; r < kRB; ++r) da[r] = D[r * kUMax + a];
    const size_t rowoff = (size_t)U[a] * n;
    for (int b = lane; b <= a; b += 32) {
      float sum = 0.f;
#pragma unroll
      for (int r = 0; r < kRB; ++r) sum = fmaf(da[r], D[r * kUMax + b], sum);
      if (sum != 0.f) atomicAdd(&B[rowoff + U[b]], sum);
    }
  }
}

// B_s[j][j] += half_rho for every scenario (grid.y = scenario).
__global__ void k_add_diag(float* B, int n, float half_rho) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) B[(size_t)blockIdx.y * n * n + (size_t)j * n + j] += half_rho;
}

// Upper triangle of every B_s^{-1} from its lower triangle (32 x 32 tiles through
// shared memory; grid (tiles, tiles, scenario), only tiles with row block >= column block).
__global__ void k_mirror_lower(float* X, int n) {
  __shared__ float t[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;
  if (bj > bi) return;
  float* Xs = X + (size_t)blockIdx.z * n * n;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int i = bi * 32 + r, j = bj * 32 + threadIdx.x;
    if (i < n && j < n) t[r][threadIdx.x] = Xs[(size_t)i * n + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int i = bj * 32 + r, j = bi * 32 + threadIdx.x;       // (i, j) = transposed position
    if (i < n && j < n && j > i) Xs[(size_t)i * n + j] = t[threadIdx.x][r];
  }
}

// Y_s = I (all scenarios; Y zero on entry).
__global__ void k_set_identity(float* Y, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) Y[(size_t)blockIdx.y * n * n + (size_t)j * n + j] = 1.f;
}

// Cholesky of the diagonal block kb of every scenario (grid.x = scenario), in place
// (lower).  A pivot <= 0 sets *err and is replaced by 1 so that the factorisation ends.
__global__ void __launch_bounds__(256) k_potrf_diag(float* B, int n, int kb, int* err) {
  __shared__ float a[kNB][kNB + 1];
  float* Bs = B + (size_t)blockIdx.x * n * n;
  const int r0 = kb * kNB, nb = min(kNB, n - r0);
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, k = e % nb;
    a[i][k] = Bs[(size_t)(r0 + i) * n + r0 + k];
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      float d = a[j][j];
      if (!(d > 0.f)) {
        atomicExch(err, 1);
        d = 1.f;
      }
      a[j][j] = sqrtf(d);
    }
    __syncthreads();
    const float ljj = a[j][j];
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][j] /= ljj;
    __syncthreads();
    const int m = nb - j - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k <= i) a[i][k] -= a[i][j] * a[k][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, k = e % nb;
    if (k <= i) Bs[(size_t)(r0 + i) * n + r0 + k] = a[i][k];
  }
}

// Panel below diagonal block kb: each row x solves x L_kk^T = a (grid (row blocks,
// scenario), one row per thread).
__global__ void __launch_bounds__(64) k_trsm_panel(float* B, int n, int kb) {
  __shared__ float L[kNB][kNB + 1];
  __shared__ float x[64][kNB + 1];
  float* Bs = B + (size_t)blockIdx.y * n * n;
  const int r0 = kb * kNB, nb = min(kNB, n - r0);
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, k = e % nb;
    L[i][k] = Bs[(size_t)(r0 + i) * n + r0 + k];
  }
  const int i = r0 + nb + blockIdx.x * 64 + threadIdx.x;
  if (i < n)
    for (int k = 0; k < nb; ++k) x[threadIdx.x][k] = Bs[(size_t)i * n + r0 + k];
  __syncthreads();
  if (i >= n) return;
  for (int j = 0; j < nb; ++j) {
    float t = x[threadIdx.x][j];
    for (int k = 0; k < j; ++k) t -= x[threadIdx.x][k] * L[j][k];
    x[threadIdx.x][j] = t / L[j][j];
  }
  for (int k = 0; k < nb; ++k) Bs[(size_t)i * n + r0 + k] = x[threadIdx.x][k];
}

// Rows of block kb of Y: Y[R, 0:cols] = L_kk^{-1} Y[R, 0:cols] (forward
// substitution down the block's rows; one column per thread; grid (column blocks,
// scenario)).
__global__ void __launch_bounds__(64) k_trsm_left(const float* L, float* Y, int n, int kb, int cols) {
  __shared__ float Lk[kNB][kNB + 1];
  __shared__ float y[kNB][64 + 1];
  const float* Ls = L + (size_t)blockIdx.y * n * n;
  float* Ys = Y + (size_t)blockIdx.y * n * n;
  const int r0 = kb * kNB, nb = min(kNB, n - r0);
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, k = e % nb;
    Lk[i][k] = Ls[(size_t)(r0 + i) * n + r0 + k];
  }
  const int c = blockIdx.x * 64 + threadIdx.x;
  if (c < cols)
    for (int j = 0; j < nb; ++j) y[j][threadIdx.x] = Ys[(size_t)(r0 + j) * n + c];
  __syncthreads();
  if (c >= cols) return;
  for (int j = 0; j < nb; ++j) {
    float t = y[j][threadIdx.x];
    for (int k = 0; k < j; ++k) t -= Lk[j][k] * y[k][threadIdx.x];
    y[j][threadIdx.x] = t / Lk[j][j];
  }
  for (int j = 0; j < nb; ++j) Ys[(size_t)(r0 + j) * n + c] = y[j][threadIdx.x];
}

}  // namespace

// Form, factor and invert B_s for every scenario into P->binv (allocating it on
// first use); also A~_s^T p~ into P->bchol (compute_bconst, solver.cu).
int chol_prepare(Plan* P, const std::vector<double>& rho, CholExtra* extra) {
  if (!extra && P->chol_ready && !P->chol_con && P->chol_rho == rho) return RPT_OK;
  const DevPlan& dp = P->dp;
  const int n = dp.n, N = dp.N;
  const size_t nn = (size_t)n * n;
  cudaStream_t st = P->stream;
  cudaError_t e;
  if (!P->binv) {
    if ((e = cudaMalloc(&P->binv, sizeof(float) * nn * N))) return cuda_fail(e, "allocate the factor");
    P->allocs.push_back(P->binv);
  }
  if (!P->bchol) {
    if ((e = cudaMalloc(&P->bchol, sizeof(double) * (size_t)n * N))) return cuda_fail(e, "allocate A~'p~");
    P->allocs.push_back(P->bchol);
  }
  float* Y = nullptr;
  if ((e = cudaMalloc(&Y, sizeof(float) * nn * N))) return cuda_fail(e, "allocate the inverse workspace");
  auto done = [&](int rc) {
    cudaStreamSynchronize(st);
    cudaFree(Y);
    return rc;
  };
  if ((e = cudaMemsetAsync(P->binv, 0, sizeof(float) * nn * N, st))) return done(cuda_fail(e, "memset"));
  if ((e = cudaMemsetAsync(Y, 0, sizeof(float) * nn * N, st))) return done(cuda_fail(e, "memset"));
  if ((e = cudaMemsetAsync(P->err, 0, sizeof(int), st))) return done(cuda_fail(e, "memset"));
  // 1. B_s = A~_s^T A~_s (lower), + (rho/2) I
  const size_t smem = sizeof(int) * ((size_t)dp.n_pad + kUMax) + sizeof(float) * kRB * kUMax;
  void* fn;
  if (dp.path == 3) {
    if (dp.index_width == 16)
      fn = dp.value_format == 1 ? (void*)k_btb<__nv_bfloat16, uint16_t, true>
         : dp.value_format == 2 ? (void*)k_btb<__nv_fp8_e4m3, uint16_t, true> : (void*)k_btb<float, uint16_t, true>;
    else
      fn = dp.value_format == 1 ? (void*)k_btb<__nv_bfloat16, int32_t, true>
         : dp.value_format == 2 ? (void*)k_btb<__nv_fp8_e4m3, int32_t, true> : (void*)k_btb<float, int32_t, true>;
  } else if (dp.index_width == 16) {
    fn = dp.value_format == 1 ? (void*)k_btb<__nv_bfloat16, uint16_t, false>
       : dp.value_format == 2 ? (void*)k_btb<__nv_fp8_e4m3, uint16_t, false> : (void*)k_btb<float, uint16_t, false>;
  } else {
    fn = dp.value_format == 1 ? (void*)k_btb<__nv_bfloat16, int32_t, false>
       : dp.value_format == 2 ? (void*)k_btb<__nv_fp8_e4m3, int32_t, false> : (void*)k_btb<float, int32_t, false>;
  }
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return done(cuda_fail(e, "kernel attribute"));
  const dim3 gb((dp.m_act + kRB - 1) / kRB);
  for (int s = 0; s < N; ++s) {
    DevPlan dpc = dp;
    float* Bs = P->binv + nn * s;
    const int* ro = P->rec_of;
    int ss = s;
    void* args[] = {(void*)&dpc, (void*)&ss, (void*)&ro, (void*)&Bs};
    if ((e = cudaLaunchKernel(fn, gb, dim3(256), args, smem, st))) return done(cuda_fail(e, "launch"));
  }
  const dim3 gd((n + 255) / 256, N);
  for (int g = 0; g < dp.G; ++g)   // each group's scenarios with the group's penalty
    k_add_diag<<<dim3((n + 255) / 256, dp.Ns), 256, 0, st>>>(P->binv + nn * (size_t)g * dp.Ns, n,
                                                              (float)(0.5 * rho[g]));
  if (extra && (e = extra->add(P, P->binv))) return done(cuda_fail(e, "constraint terms of B_s"));
  // 2. Cholesky, lower, in place, right-looking in panels of kPB blocks: inside a
  //    panel each block is factored (diagonal block, then the rows below it) and
  //    its rank-64 update goes to the rest of the panel's columns only; the
  //    matrix right of the panel gets the panel's rank-256 update once
  const int nblk = (n + kNB - 1) / kNB;
  const long long snn = (long long)nn;
  for (int KB = 0; KB < nblk; KB += kPB) {
    const int kend = std::min(KB + kPB, nblk);
    for (int kb = KB; kb < kend; ++kb) {
      k_potrf_diag<<<N, 256, 0, st>>>(P->binv, n, kb, P->err);
      const int c0 = (kb + 1) * kNB;            // first row and column after block kb
      if (c0 >= n) continue;
      k_trsm_panel<<<dim3((n - c0 + 63) / 64, N), 64, 0, st>>>(P->binv, n, kb);
      const int c1 = std::min(kend * kNB, n);   // the panel's remaining columns c0 .. c1
      if (c1 > c0) {
        const float* L21 = P->binv + (size_t)c0 * n + (size_t)kb * kNB;
        gemm_tf32x3<false, true>(st, n - c0, c1 - c0, kNB, L21, n, L21, n, P->binv + (size_t)c0 * n + c0, n,
                                 -1.f, 1.f, N, snn, snn, snn, /*lower=*/true);
      }
    }
    const int t0 = kend * kNB;
    if (t0 < n) {
      const float* Lp = P->binv + (size_t)t0 * n + (size_t)KB * kNB;   // rows t0.., the panel's columns
      gemm_tf32x3<false, true>(st, n - t0, n - t0, (kend - KB) * kNB, Lp, n, Lp, n, P->binv + (size_t)t0 * n + t0,
                               n, -1.f, 1.f, N, snn, snn, snn, /*lower=*/true);
    }
  }
  // 3. Y = L^{-1} (forward substitution on I), in panels of kPB block rows: the
  //    panel's rows first take -L Y over all earlier columns in one product
  //    (Y is lower triangular, so the earlier rows of Y end at the panel), then
  //    block row by block row the rest of the sum and the diagonal block's solve
  k_set_identity<<<gd, 256, 0, st>>>(Y, n);
  for (int KB = 0; KB < nblk; KB += kPB) {
    const int kend = std::min(KB + kPB, nblk);
    const int R0 = KB * kNB, R1 = std::min(kend * kNB, n);
    if (R0 > 0)
      gemm_tf32x3<false, false>(st, R1 - R0, R0, R0, P->binv + (size_t)R0 * n, n, Y, n, Y + (size_t)R0 * n, n,
                                -1.f, 1.f, N, snn, snn, snn, false, /*kdiag=*/1);
    for (int kb = KB; kb < kend; ++kb) {
      const int r0 = kb * kNB, nb = std::min(kNB, n - r0);
      if (r0 > R0)
        gemm_tf32x3<false, false>(st, nb, r0, r0 - R0, P->binv + (size_t)r0 * n + R0, n, Y + (size_t)R0 * n, n,
                                  Y + (size_t)r0 * n, n, -1.f, 1.f, N, snn, snn, snn);
      const int cols = r0 + nb;
      k_trsm_left<<<dim3((cols + 63) / 64, N), 64, 0, st>>>(P->binv, Y, n, kb, cols);
    }
  }
  // 4. B^{-1} = Y^T Y into binv (the factor is no longer needed): lower tiles, the
  //    sum starting at max(i, j) since Y is lower triangular; then mirrored
  gemm_tf32x3<true, false>(st, n, n, n, Y, n, Y, n, P->binv, n, 1.f, 0.f, N, (long long)nn, (long long)nn,
                           (long long)nn, /*lower=*/true, /*kdiag=*/2);
  k_mirror_lower<<<dim3((n + 31) / 32, (n + 31) / 32, N), dim3(32, 8), 0, st>>>(P->binv, n);
  if ((e = cudaGetLastError())) return done(cuda_fail(e, "launch"));
  // 5. A~_s^T p~
  if (int rc = compute_bconst(P)) return done(rc);
  if ((e = cudaStreamSynchronize(st))) return done(cuda_fail(e, "sync"));
  int herr = 0;
  if ((e = cudaMemcpy(&herr, P->err, sizeof(int), cudaMemcpyDeviceToHost))) return done(cuda_fail(e, "copy"));
  if (herr) {
    cudaMemset(P->err, 0, sizeof(int));
    set_error("cached-factor subproblem: B_s is not positive definite in float32");
    return done(RPT_EINVAL);
  }
  P->chol_ready = true;
  P->chol_con = extra != nullptr;
  P->chol_rho = rho;
  return done(RPT_OK);
}

}  // namespace rpt
