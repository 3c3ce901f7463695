// Internal definitions shared by the librpt translation units.
//
// Layout in HBM (one plan):
//   rows      : the m_act voxel rows kept on the device (rows with no entry in
//               any scenario are dropped; their constant w p^2 goes to const_term)
//   row lists : per scenario, its non-empty rows sorted by decreasing length
//               (rows empty in that scenario add c_s w p^2 to const_term); the
//               entries are stored permuted into that order, so each row is
//               contiguous and consecutive rows are adjacent
//   rowrec    : int4 per listed row {entry offset, c_s w_i, p_i, kept-row index},
//               rec_base[s]..: scenario s's rows plus a terminator record
//               holding its entry count (16 bytes: a run of rows is one bulk copy)
//   col, val  : concatenated over scenarios, scenario s starts at nnz_base[s];
//               allocations are padded so that 16-entry aligned bulk copies
//               never leave them
//   colscale  : float32 [N][n_pad] per-column scales of quantised values
// Work decomposition of one row pass:
//   path 0 (register): `blocks` = cost-balanced runs of rows, one CTA and one
//               partial slot each
//   path 1 (TMA ring): every scenario's row list is cut into row-aligned
//               `chunks` that each fit one shared-memory stage; one persistent
//               CTA per SM pulls chunks from per-scenario queues (starting at a
//               home scenario, moving on when it is exhausted), and keeps one
//               partial slot per scenario it visited (slot = cta * N + s).
//   path 2 (streaming): the same chunk queues (chunks cut by row-length class),
//               but every warp of the persistent CTA claims chunks on its own.
//   path 3 (bundled ring): the ring of path 1 over row bundles (layout.h):
//               rows grouped 4 at a time, one spot index per block column of a
//               bundle, records of 4 int4 per bundle; 64-bit fixed-point
//               accumulators (exact, order-independent sums).
//   The CTA that finishes last compacts the slots of every scenario into an
//   ordered list, sums the objective per scenario and resets the queues.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "chunk.h"

namespace rpt {

constexpr int kRowThreads = 512;      // threads of a register-path row-pass CTA
constexpr int kTmaThreads = 1024;     // threads of a TMA-path CTA (1 producer + 31 consumer warps)
constexpr int kStrThreads = 512;      // threads of a streaming-path CTA (16 independent warps)
constexpr int kVecThreads = 256;      // threads of a vector CTA (one column each)

struct DevPlan {
  int m, n, N, m_act, n_pad, nblocks;  // nblocks = partial slots
  int G, Ns;                          // groups (problems of a batched plan) and scenarios per
                                      // group: scenario u belongs to group u / Ns (G = 1, Ns = N
                                      // for a plan of one problem)
  int value_format;                   // RPT_F32 / RPT_BF16 / RPT_FP8E4M3
  int index_width;                    // 32 or 16
  int path;                           // 0 register, 1 TMA ring, 2 streaming, 3 bundled ring
  int grid;                           // CTAs of one row pass
  int cmax, rmax, stages;             // TMA path: entries / rows per stage, ring depth
  int ring_threads;                   // path 3: threads of a row-pass CTA (1024, 768, 640)
  int slot_cap;                       // capacity of each scenario's slot list
  const int64_t* nnz_base;            // [N]
  const int32_t* col32;               // [NNZ] (index_width 32)
  const uint16_t* col16;              // [NNZ] (index_width 16)
  const float* val32;                 // [NNZ] (RPT_F32)
  const __nv_bfloat16* valbf;         // [NNZ] (RPT_BF16)
  const __nv_fp8_e4m3* val8;          // [NNZ] (RPT_FP8E4M3)
  const float* colscale;              // [N][n_pad] (quantised formats) or null
  const int4* blocks;                 // path 0: [grid] (s, first row, end row, lanes per row)
  // Partial slots of the last pass, per scenario: slot_count[s] slots listed in
  // slot_list[s * slot_cap ...] in increasing order (static for path 0, written
  // by the finishing CTA of every pass for path 1); objs[s] = objective of
  // scenario s in the last objective pass.
  int* slot_count;                    // [N]
  int* slot_list;                     // [N][slot_cap]
  double* objs;                       // [N]
  double* objp;                       // [nblocks] per-slot objective partial sums
  unsigned int* done_ctr;             // finishing-CTA counter (self-resetting)
  int* qnext;                         // path 1: [N] per-scenario chunk queues (self-resetting)
  unsigned char* visited;             // path 1: [N][grid] slots written in this pass
  const int* scen_chunk;              // path 1: [N+1] chunk range of each scenario
  const int4* rowrec;                 // row records {start, c_s w_i, p_i, kept-row index}
  const int* rec_base;                // [N+1] first record of each scenario's row list
  const ChunkDesc* chunks;            // path 1: scenario-major chunk list
  int* err;                           // device error word (bounded waits that ran out)
  int inject_timeout;                 // testing: the ring's producer issues nothing (waits run out)
  // path 3 (bundled ring): partial slots hold exact 64-bit fixed-point sums.  A
  // pass on scenario s scales every contribution by 2^fexp[s], chosen from the
  // bound |acc_c| <= kbound[2s] max|v_s| (+ kbound[2s+1] with the prescription
  // term) so that no sum can overflow; the reducers scale back by 2^-fexp[s].
  int acc64;                          // 1: partial slots are int64 fixed point (path 3 with exact sums;
                                      //    0 on path 3: float32 shared atomics, like paths 0-2)
  int* fexp;                          // [N] scale exponent of the last scatter pass per scenario
  const double* kbound;               // [2N] max_c sum_i c_s w_i |a_ic| ||a_i||_1 and max_c sum_i c_s w_i |a_ic| p_i
};

// Fixed-point exponent that marks a scenario whose staged vector was not finite
// (the reducers then return NaN, so that divergence is still detected).
constexpr int kFexpNaN = -100000;

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

// ---- launchers implemented in rowpass.cu / rowstream.cu ---------------------------
namespace rpt {
// v:      staged spot vectors, float32 [N][n_pad] (v_stride = n_pad) or one shared
//         vector (v_stride = 0)
// active: [N] int flags or null (work of inactive scenarios is skipped)
// partial: [nblocks][n_pad] per-slot accumulators (modes kNormal, kResid)
// dose:    [N][m_act] (mode kDose)
// The per-slot objective sums go to P.objp and, per scenario, to P.objs.
void* rowpass_kernel(const DevPlan& P, int mode);
size_t rowpass_smem(const DevPlan& P, int mode);
int rowpass_threads(const DevPlan& P);
cudaError_t rowpass_prepare(const DevPlan& P);
size_t tma_smem_bytes(int n_pad, int cmax, int rmax, int stages, int value_bytes, int index_bytes,
                      bool scatter, bool bundled = false, bool fixed = false);
size_t stream_smem_bytes(int n_pad, int rmax, bool scatter);
void* stream_rowpass_kernel(const DevPlan& P, int mode);   // rowstream.cu
// Bundled layout, at plan creation: kbound[2s], kbound[2s+1] of every scenario
// (DevPlan::kbound) from the stored values; kc, pc: scratch [n_pad] doubles.
cudaError_t bundle_bounds(const DevPlan& P, double* kc, double* pc, double* kbound, cudaStream_t st);
// New weights for scenario s (rpt_plan_set_weights): rewrite its row records from
// wk, pk (per kept row) and c_s, and add sum_i c_s w_i a_ij^2 * scale to acc
// (int64 fixed point, [n_pad], zeroed here).
cudaError_t plan_reweight(const DevPlan& P, int s, double cs, const double* wk, const double* pk, double scale,
                          unsigned long long* acc, cudaStream_t st);
}  // namespace rpt
