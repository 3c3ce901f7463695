// Internal definitions shared by the librpt translation units.
//
// Layout in HBM (one plan):
//   rows      : the m_act voxel rows kept on the device (rows with no entry in
//               any scenario are dropped; their constant w p^2 goes to const_term)
//   row_ptr   : int32 [N][m_act+1], offsets within scenario s
//   rowrec    : int4  [N][m_act+1] per-row record {row_ptr, c_s w_i, p_i, 0}
//               (16 bytes, so a run of rows is one bulk copy)
//   col, val  : concatenated over scenarios, scenario s starts at nnz_base[s];
//               allocations are padded so that 16-entry aligned bulk copies
//               never leave them
//   w, p      : float32 [m_act] voxel weight and prescription (shared by scenarios)
//   cs        : float32 [N] scenario weights c_s
//   colscale  : float32 [N][n_pad] per-column scales of quantised values
// Work decomposition of one row pass:
//   path 0 (register): `blocks` = nnz-balanced row blocks, one CTA each
//   path 1 (TMA ring): the scenario-major sequence of all rows is cut into
//               `grid` equal-cost slices, one persistent CTA each; a slice is
//               1..3 `segs` (one scenario each), a segment is a run of
//               row-aligned `chunks` that each fit one shared-memory stage.
//   Either way every work unit (block or segment) owns one partial slot of
//   n_pad floats; the slots of scenario s are [blk_first[s], blk_first[s+1]).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

namespace rpt {

constexpr int kRowThreads = 512;      // threads of a register-path row-pass CTA
constexpr int kTmaThreads = 512;      // threads of a TMA-path CTA (1 producer + 15 consumer warps)
constexpr int kVecThreads = 256;      // threads of a vector CTA (one column each)

struct ChunkDesc {
  long long g_al;                     // first copied entry (global index, multiple of 16)
  int row_begin;                      // first row of the chunk (scenario-relative)
  int n_rows;                         // rows in the chunk
  int n_ent;                          // copied entries (multiple of 16)
  int pad;
};

struct DevPlan {
  int m, n, N, m_act, n_pad, nblocks;  // nblocks = partial slots
  int value_format;                   // RPT_F32 / RPT_BF16 / RPT_FP8E4M3
  int index_width;                    // 32 or 16
  int path;                           // 0 register, 1 TMA ring
  int grid;                           // CTAs of one row pass
  int cmax, rmax, stages;             // TMA path: entries / rows per stage, ring depth
  int pad0;
  const int32_t* row_ptr;             // [N][m_act+1]
  const int64_t* nnz_base;            // [N]
  const int32_t* col32;               // [NNZ] (index_width 32)
  const uint16_t* col16;              // [NNZ] (index_width 16)
  const float* val32;                 // [NNZ] (RPT_F32)
  const __nv_bfloat16* valbf;         // [NNZ] (RPT_BF16)
  const __nv_fp8_e4m3* val8;          // [NNZ] (RPT_FP8E4M3)
  const float* colscale;              // [N][n_pad] (quantised formats) or null
  const float* w;                     // [m_act]
  const float* p;                     // [m_act]
  const float* cs;                    // [N]
  const int4* blocks;                 // path 0: [nblocks] (s, row_begin, row_end, 0)
  const int* blk_first;               // [N+1]
  const int4* rowrec;                 // [N][m_act+1]
  const ChunkDesc* chunks;            // path 1
  const int4* segs;                   // path 1: (s, chunk_begin, chunk_end, slot)
  const int* cta_seg;                 // path 1: [grid+1]
  int* err;                           // device error word (bounded waits that ran out)
};

// ---- row-pass modes ---------------------------------------------------------
enum RowMode : int {
  kNormal = 0,   // acc_s  = sum_i c_s w_i a_i (a_i' v_s)
  kResid  = 1,   // acc_s  = sum_i c_s w_i a_i (a_i' v_s - p_i);  obj += c_s w_i (a_i' v_s - p_i)^2
  kObj    = 2,   // obj   += c_s w_i (a_i' v - p_i)^2 only
  kDose   = 3,   // dose[s][row] = a_i' v (physical dose) and obj
};

// ---- small device helpers -----------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of K doubles per thread; result valid in thread 0.
template <int K>
__device__ __forceinline__ void block_sum_d(double (&v)[K], double* sh /* [K*32] */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum_d(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k * 32 + wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = lane < nw ? sh[k * 32 + lane] : 0.0;
      v[k] = warp_sum_d(t);
    }
  }
  __syncthreads();
}

// Error-free transformation: s + e == a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

}  // namespace rpt

// ---- launchers implemented in rowpass.cu -----------------------------------------
namespace rpt {
// v:      staged spot vectors, float32 [N][n_pad] (v_stride = n_pad) or one shared
//         vector (v_stride = 0)
// active: [N] int flags or null (work of inactive scenarios is skipped)
// partial: [nblocks][n_pad] per-slot accumulators (modes kNormal, kResid)
// objp:    [nblocks] per-slot objective partial sums (modes kResid, kObj, kDose)
// dose:    [N][m_act] (mode kDose)
void* rowpass_kernel(const DevPlan& P, int mode);
size_t rowpass_smem(const DevPlan& P, int mode);
int rowpass_threads(const DevPlan& P);
cudaError_t rowpass_prepare(const DevPlan& P);
size_t tma_smem_bytes(int n_pad, int cmax, int rmax, int stages, int value_bytes, int index_bytes,
                      bool scatter);
}  // namespace rpt
