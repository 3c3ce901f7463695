// bfloat16 tensor-core GEMM for the learned warm start's network (the BF16
// compute form): warp-level mma.sync m16n8k16 with FP32 accumulation.
//   C = alpha * op(A) op(B) + beta * C (+ bias[N], ReLU), and optionally a
//   bfloat16 copy Cb of the result (the next layer's input);
//   op(A)(i,k) = TA ? A[k*lda + i] : A[i*lda + k];  op(B)(k,j) = TB ? B[j*ldb + k] : B[k*ldb + j]
// (the same operand conventions as gemm.cuh).  A CTA computes a 64 x 64 tile with
// 4 warps of 32 x 32 (2 x 4 mma tiles each); K advances in steps of 32 staged in
// shared memory as [row][k] for op(A) and [column][k] for op(B), so that every
// fragment register is one 32-bit shared-memory load in the layout the PTX ISA
// gives for m16n8k16 (A row-major, B column-major).  The network's GEMMs are
// small (hundreds of rows), so the tiles are staged with plain loads; beta == 0
// never reads C.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rpt {
namespace {

constexpr int kTcBM = 64, kTcBN = 64, kTcBK = 32, kTcPad = 8;
constexpr int kTcThreads = 128;

__device__ __forceinline__ void mma_bf16_m16n8k16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(kTcThreads)
k_gemm_bf16(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda, const __nv_bfloat16* __restrict__ B,
            int ldb, float* __restrict__ C, int ldc, __nv_bfloat16* __restrict__ Cb, const float* __restrict__ bias,
            int relu, float alpha, float beta) {
  __shared__ __align__(16) __nv_bfloat16 As[kTcBM][kTcBK + kTcPad];
  __shared__ __align__(16) __nv_bfloat16 Bs[kTcBN][kTcBK + kTcPad];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = blockIdx.y * kTcBM, j0 = blockIdx.x * kTcBN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;   // the warp's 32 x 32 quarter
  const int g = lane >> 2, t = lane & 3;                    // mma group and thread in group
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int k0 = 0; k0 < K; k0 += kTcBK) {
    // loads run along each operand's contiguous dimension
    for (int e = tid; e < kTcBM * kTcBK; e += kTcThreads) {
      const int ii = TA ? e % kTcBM : e / kTcBK, kk = TA ? e / kTcBM : e % kTcBK;
      const int i = i0 + ii, k = k0 + kk;
      __nv_bfloat16 v = zero;
      if (i < M && k < K) v = TA ? A[(size_t)k * lda + i] : A[(size_t)i * lda + k];
      As[ii][kk] = v;
    }
    for (int e = tid; e < kTcBN * kTcBK; e += kTcThreads) {
      const int jj = TB ? e / kTcBK : e % kTcBN, kk = TB ? e % kTcBK : e / kTcBN;
      const int j = j0 + jj, k = k0 + kk;
      __nv_bfloat16 v = zero;
      if (j < N && k < K) v = TB ? B[(size_t)j * ldb + k] : B[(size_t)k * ldb + j];
      Bs[jj][kk] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kTcBK; ks += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = wm + mt * 16 + g;
        af[mt][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * t]);
        af[mt][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * t]);
        af[mt][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * t + 8]);
        af[mt][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = wn + nt * 8 + g;
        bf[nt][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * t]);
        bf[nt][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16_m16n8k16(acc[mt][nt], af[mt], bf[nt]);
    }
    __syncthreads();
  }
  // accumulator layout: regs 0,1 at (row g, cols 2t, 2t+1), regs 2,3 at row g + 8
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + wm + mt * 16 + g + (q >> 1) * 8;
        const int j = j0 + wn + nt * 8 + 2 * t + (q & 1);
        if (i >= M || j >= N) continue;
        float v = alpha * acc[mt][nt][q];
        if (beta != 0.f) v = fmaf(beta, C[(size_t)i * ldc + j], v);
        if (bias) v += bias[j];
        if (relu) v = fmaxf(v, 0.f);
        C[(size_t)i * ldc + j] = v;
        if (Cb) Cb[(size_t)i * ldc + j] = __float2bfloat16_rn(v);
      }
}

template <bool TA, bool TB>
inline void gemm_bf16(cudaStream_t st, int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B,
                      int ldb, float* C, int ldc, __nv_bfloat16* Cb = nullptr, const float* bias = nullptr,
                      bool relu = false, float alpha = 1.f, float beta = 0.f) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + kTcBN - 1) / kTcBN, (M + kTcBM - 1) / kTcBM);
  k_gemm_bf16<TA, TB><<<grid, kTcThreads, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, Cb, bias, relu ? 1 : 0, alpha,
                                                   beta);
}

}  // namespace
}  // namespace rpt
