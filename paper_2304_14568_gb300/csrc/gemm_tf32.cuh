// FP32-accurate GEMM on the tensor cores for the cached-factor setup (the
// Cholesky trailing updates and the inverse of the factor).  Each FP32 operand x
// is split into a TF32 high part h = tf32(x) and a TF32 low part l = tf32(x - h)
// (x = h + l to about 22 significant bits), and a product is formed as
// h_a h_b + h_a l_b + l_a h_b on mma.sync m16n8k8 tf32 with FP32 accumulation;
// the dropped l_a l_b term is below 2^-22 of the product.  The tensor cores
// accumulate only over one 32-deep K tile; the tiles' sums are added in FP32
// with round-to-nearest outside them, so that the tensor cores' own rounding
// of the accumulator does not build up over long K.  This is the
// error-compensated TF32 scheme of Ootomo and Yokota ("Recovering single
// precision accuracy from Tensor Cores while surpassing the FP32 theoretical
// peak performance", 2022).
//   C = alpha * op(A) op(B) + beta * C, batched over blockIdx.z with element strides;
//   op(A)(i,k) = TA ? A[k*lda + i] : A[i*lda + k];  op(B)(k,j) = TB ? B[j*ldb + k] : B[k*ldb + j]
// with the structure flags of gemm.cuh:
//   lower: compute only output tiles that reach the lower triangle (j <= i);
//   kdiag 1: op(B)(k, j) is zero for k < j (K starts at the tile's first column);
//   kdiag 2: also op(A)(i, k) is zero for k < i (K starts at max of both).
// A CTA computes a 64 x 64 tile with 4 warps of 32 x 32 (2 x 4 mma tiles each);
// K advances in steps of 32 staged in shared memory as [row][k] for op(A) and
// [column][k] for op(B) (a row stride of 36 floats keeps the fragment loads of a
// warp on 32 distinct banks).  The next K step's tiles are loaded from global
// memory into registers while the tensor cores work on the current one.
// beta == 0 never reads C.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rpt {
namespace {

constexpr int kT3BM = 64, kT3BN = 64, kT3BK = 32, kT3Pad = 4;
constexpr int kT3Threads = 128;

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x = hi + lo in TF32 (hi's bits are a float whose low 13 bits are zero)
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32_m16n8k8(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(kT3Threads)
k_gemm_tf32x3(int M, int N, int K, const float* __restrict__ A, int lda, long long sA, const float* __restrict__ B,
              int ldb, long long sB, float* __restrict__ C, int ldc, long long sC, float alpha, float beta,
              int lower, int kdiag) {
  __shared__ __align__(16) float As[kT3BM][kT3BK + kT3Pad];
  __shared__ __align__(16) float Bs[kT3BN][kT3BK + kT3Pad];
  A += (long long)blockIdx.z * sA;
  B += (long long)blockIdx.z * sB;
  C += (long long)blockIdx.z * sC;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = blockIdx.y * kT3BM, j0 = blockIdx.x * kT3BN;
  if (lower && j0 > i0 + kT3BM - 1) return;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;   // the warp's 32 x 32 quarter
  const int g = lane >> 2, t = lane & 3;                    // mma group and thread in group
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const int kfirst = kdiag == 2 ? max(i0, j0) : (kdiag == 1 ? j0 : 0);
  constexpr int kPer = kT3BM * kT3BK / kT3Threads;   // tile elements per thread and operand (16)
  float ra[kPer], rb[kPer];
  // loads run along each operand's contiguous dimension
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = tid + q * kT3Threads;
      const int ii = TA ? e % kT3BM : e / kT3BK, kk = TA ? e / kT3BM : e % kT3BK;
      const int i = i0 + ii, k = k0 + kk;
      ra[q] = (i < M && k < K) ? (TA ? A[(size_t)k * lda + i] : A[(size_t)i * lda + k]) : 0.f;
      const int jj = TB ? e / kT3BK : e % kT3BN, kb = TB ? e % kT3BK : e / kT3BN;
      const int j = j0 + jj, kj = k0 + kb;
      rb[q] = (j < N && kj < K) ? (TB ? B[(size_t)j * ldb + kj] : B[(size_t)kj * ldb + j]) : 0.f;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = tid + q * kT3Threads;
      const int ii = TA ? e % kT3BM : e / kT3BK, kk = TA ? e / kT3BM : e % kT3BK;
      As[ii][kk] = ra[q];
      const int jj = TB ? e / kT3BK : e % kT3BN, kb = TB ? e % kT3BK : e / kT3BN;
      Bs[jj][kb] = rb[q];
    }
  };
  int k0 = (kfirst / kT3BK) * kT3BK;
  if (k0 < K) {
    load(k0);
    store();
  }
  __syncthreads();
  for (; k0 < K; k0 += kT3BK) {
    const bool more = k0 + kT3BK < K;
    if (more) load(k0 + kT3BK);   // in flight during the products below
    float part[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c) part[a][b][c] = 0.f;
#pragma unroll
    for (int ks = 0; ks < kT3BK; ks += 8) {
      // fragments of m16n8k8 (tf32): A (row-major 16 x 8): a0 (g, t), a1 (g + 8, t),
      // a2 (g, t + 4), a3 (g + 8, t + 4); B (column-major 8 x 8): b0 (t, g), b1 (t + 4, g)
      uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = wm + mt * 16 + g;
        split_tf32(As[r][ks + t], ah[mt][0], al[mt][0]);
        split_tf32(As[r + 8][ks + t], ah[mt][1], al[mt][1]);
        split_tf32(As[r][ks + t + 4], ah[mt][2], al[mt][2]);
        split_tf32(As[r + 8][ks + t + 4], ah[mt][3], al[mt][3]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int c = wn + nt * 8 + g;
        split_tf32(Bs[c][ks + t], bh[nt][0], bl[nt][0]);
        split_tf32(Bs[c][ks + t + 4], bh[nt][1], bl[nt][1]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          mma_tf32_m16n8k8(part[mt][nt], al[mt], bh[nt]);   // small terms first
          mma_tf32_m16n8k8(part[mt][nt], ah[mt], bl[nt]);
          mma_tf32_m16n8k8(part[mt][nt], ah[mt], bh[nt]);
        }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][b][c] += part[a][b][c];
    __syncthreads();   // every warp is done with the current tiles
    if (more) store();
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
        C[(size_t)i * ldc + j] = v;
      }
}

template <bool TA, bool TB>
inline void gemm_tf32x3(cudaStream_t st, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                        float* C, int ldc, float alpha = 1.f, float beta = 0.f, int batch = 1, long long sA = 0,
                        long long sB = 0, long long sC = 0, bool lower = false, int kdiag = 0) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((N + kT3BN - 1) / kT3BN, (M + kT3BM - 1) / kT3BM, batch);
  k_gemm_tf32x3<TA, TB><<<grid, kT3Threads, 0, st>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, alpha, beta,
                                                     lower ? 1 : 0, kdiag);
}

}  // namespace
}  // namespace rpt
