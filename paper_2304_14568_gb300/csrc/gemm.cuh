// A small FP32 GEMM for the library's dense side work (the learned warm start's
// network and the cached-factor subproblem setup): 64 x 64 output tiles, 16-deep
// shared-memory staging, 4 x 4 outputs per thread, optional transposes, batched
// over blockIdx.z with element strides.
//   C = alpha * op(A) op(B) + beta * C (+ bias[N], ReLU)
//   op(A)(i,k) = TA ? A[k*lda + i] : A[i*lda + k];  op(B)(k,j) = TB ? B[j*ldb + k] : B[k*ldb + j]
// beta == 0 never reads C.  Structure flags for triangular operands:
//   lower: compute only output tiles that reach the lower triangle (j <= i);
//   kdiag 1: op(B)(k, j) is zero for k < j (K starts at the tile's first column);
//   kdiag 2: also op(A)(i, k) is zero for k < i (K starts at max of both).
#pragma once
#include <cuda_runtime.h>

namespace rpt {
namespace {

constexpr int kGemmTM = 64, kGemmTN = 64, kGemmTK = 16;
constexpr int kGemmThreads = 256;

template <bool TA, bool TB>
__global__ void __launch_bounds__(kGemmThreads)
k_gemm(int M, int N, int K, const float* __restrict__ A, int lda, long long sA, const float* __restrict__ B,
       int ldb, long long sB, float* __restrict__ C, int ldc, long long sC, const float* __restrict__ bias,
       int relu, float alpha, float beta, int lower, int kdiag) {
  __shared__ float As[kGemmTK][kGemmTM + 4];
  __shared__ float Bs[kGemmTK][kGemmTN + 4];
  A += (long long)blockIdx.z * sA;
  B += (long long)blockIdx.z * sB;
  C += (long long)blockIdx.z * sC;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * kGemmTM, j0 = blockIdx.x * kGemmTN;
  if (lower && j0 > i0 + kGemmTM - 1) return;
  float acc[4][4] = {};
  const int kfirst = kdiag == 2 ? max(i0, j0) : (kdiag == 1 ? j0 : 0);
  for (int k0 = (kfirst / kGemmTK) * kGemmTK; k0 < K; k0 += kGemmTK) {
    for (int e = threadIdx.x; e < kGemmTK * kGemmTM; e += kGemmThreads) {
      const int kk = e / kGemmTM, ii = e % kGemmTM;
      const int i = i0 + ii, k = k0 + kk;
      float a = 0.f;
      if (i < M && k < K) a = TA ? A[(size_t)k * lda + i] : A[(size_t)i * lda + k];
      As[kk][ii] = a;
    }
    for (int e = threadIdx.x; e < kGemmTK * kGemmTN; e += kGemmThreads) {
      const int kk = e / kGemmTN, jj = e % kGemmTN;
      const int j = j0 + jj, k = k0 + kk;
      float b = 0.f;
      if (j < N && k < K) b = TB ? B[(size_t)j * ldb + k] : B[(size_t)k * ldb + j];
      Bs[kk][jj] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGemmTK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty * 4 + r;
    if (i >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx * 4 + c;
      if (j >= N) continue;
      float v = alpha * acc[r][c];
      if (beta != 0.f) v = fmaf(beta, C[(size_t)i * ldc + j], v);
      if (bias) v += bias[j];
      if (relu) v = fmaxf(v, 0.f);
      C[(size_t)i * ldc + j] = v;
    }
  }
}

template <bool TA, bool TB>
inline void gemm(cudaStream_t st, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                 int ldc, const float* bias = nullptr, bool relu = false, float alpha = 1.f, float beta = 0.f,
                 int batch = 1, long long sA = 0, long long sB = 0, long long sC = 0, bool lower = false,
                 int kdiag = 0) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + kGemmTN - 1) / kGemmTN, (M + kGemmTM - 1) / kGemmTM, batch);
  k_gemm<TA, TB><<<grid, kGemmThreads, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, bias, relu ? 1 : 0,
                                                alpha, beta, lower ? 1 : 0, kdiag);
}

}  // namespace
}  // namespace rpt
