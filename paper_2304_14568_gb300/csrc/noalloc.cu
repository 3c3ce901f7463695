// Allocation-free scenario operator: u = A^T diag(w) A v + (rho/2) v for one
// scenario whose CSR matrix the caller already holds in device memory.
//
// For callers that must not allocate device memory: code running where
// cudaMalloc is not available or not allowed (inside a memory pool that owns all
// device memory, in a real-time loop that may not block on the allocator, or in
// a process whose allocations are accounted by someone else).  Such a caller
// passes its own device inputs and output; the only working memory is a
// file-scope device array of fixed size, the per-CTA partial sums.
//
// The scratch array lives in every device that loads the library, for the life
// of the process.  In host code its name is only a host-side stand-in, so the
// device address is looked up once per device (cudaGetSymbolAddress) and passed
// to the kernels.  Every call overwrites each scratch slot it later reads, so
// nothing has to be cleared between calls; calls that overlap on the GPU share
// the array and race.
#include <mutex>
#include <string>

#include "plan.h"

namespace rpt {
namespace {

constexpr int kNaThreads = 512;
constexpr int kNaMaxCtas = 128;
constexpr int kNaMaxCols = 8192;           // largest n (columns padded to a multiple of 32)

// Per-CTA partial accumulators: kNaMaxCtas x kNaMaxCols floats (4 MiB).
static __device__ __align__(256) float g_noalloc_scratch[kNaMaxCtas * kNaMaxCols];

// Rows of CTA c: an nnz-balanced split found by binary search on row_ptr.
__device__ int first_row_with_offset(const int32_t* __restrict__ rp, int m, long long target) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((long long)rp[mid] >= target) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kNaThreads)
k_noalloc_pass(int m, int n, int n_pad, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
               const float* __restrict__ val, const float* __restrict__ w, const float* __restrict__ v,
               float* __restrict__ scratch) {
  extern __shared__ float sm[];
  float* sv = sm;
  float* acc = sm + n_pad;
  __shared__ int rows[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kNaThreads / 32;
  for (int j = tid; j < n_pad; j += kNaThreads) {
    sv[j] = j < n ? v[j] : 0.f;
    acc[j] = 0.f;
  }
  if (tid == 0) {
    const long long nnz = rp[m];
    rows[0] = first_row_with_offset(rp, m, nnz * blockIdx.x / gridDim.x);
    rows[1] = blockIdx.x + 1 == gridDim.x ? m : first_row_with_offset(rp, m, nnz * (blockIdx.x + 1) / gridDim.x);
  }
  __syncthreads();
  for (int i = rows[0] + warp; i < rows[1]; i += nw) {
    const int a = rp[i], b = rp[i + 1];
    float t = 0.f;
    for (int k = a + lane; k < b; k += 32) {
      const int c = col[k];
      if ((unsigned)c < (unsigned)n) t = fmaf(val[k], sv[c], t);   // entries outside [0, n) are ignored
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    const float coef = w[i] * t;
    for (int k = a + lane; k < b; k += 32) {
      const int c = col[k];
      if ((unsigned)c < (unsigned)n) atomicAdd(&acc[c], coef * val[k]);
    }
  }
  __syncthreads();
  float* out = scratch + (size_t)blockIdx.x * kNaMaxCols;
  for (int j = tid; j < n_pad; j += kNaThreads) out[j] = acc[j];
}

// u[j] = sum over CTAs c of scratch[c][j] + (rho/2) v[j].  The sum over the CTAs
// runs in a fixed order with compensation; the partial of each CTA comes from
// shared-memory float atomics whose order varies between runs, so results are
// not bitwise reproducible (they stay within the float32 bound of the sums).
__global__ void k_noalloc_reduce(int n, int ctas, const float* __restrict__ scratch, const float* __restrict__ v,
                                 float half_rho, float* __restrict__ u) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float s = 0.f, c = 0.f;
  for (int k = 0; k < ctas; ++k) {
    float t, e;
    two_sum(s, scratch[(size_t)k * kNaMaxCols + j], t, e);
    s = t;
    c += e;
  }
  u[j] = (s + c) + half_rho * v[j];
}

std::mutex g_na_mutex;
// device address of the scratch array, per device ordinal; looked up by the first
// call on a device and kept for the process (not valid across a cudaDeviceReset
// of that device, which the rpt.h entry rules out)
float* g_na_ptr[64] = {nullptr};

}  // namespace
}  // namespace rpt

using namespace rpt;

extern "C" int rpt_normal_apply_noalloc(int32_t m, int32_t n, const int32_t* row_ptr_dev,
                                        const int32_t* col_idx_dev, const float* val_dev,
                                        const float* row_w_dev, const float* v_dev, double rho, float* u_dev,
                                        void* stream) {
  if (m < 1 || n < 1 || !row_ptr_dev || !col_idx_dev || !val_dev || !row_w_dev || !v_dev || !u_dev ||
      !(rho >= 0.0)) {
    set_error("rpt_normal_apply_noalloc: bad argument (sizes, null pointer or rho)");
    return RPT_EINVAL;
  }
  if (n > kNaMaxCols) {
    set_error("rpt_normal_apply_noalloc: n = " + std::to_string(n) + " exceeds the scratch limit of " +
              std::to_string(kNaMaxCols) + " spots");
    return RPT_EUNSUPPORTED;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    set_error("rpt_normal_apply_noalloc: device ordinal out of range");
    return RPT_EUNSUPPORTED;
  }
  float* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      // one-time set-up on this device (must happen outside stream capture)
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
      g_na_ptr[dev] = static_cast<float*>(p);
    }
    scratch = g_na_ptr[dev];
  }
  const int n_pad = (n + 31) / 32 * 32;
  const size_t smem = (size_t)n_pad * 2 * sizeof(float);
  if ((e = cudaFuncSetAttribute(k_noalloc_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return cuda_fail(e, "kernel attribute");
  int ctas = 0;
  if ((e = cudaDeviceGetAttribute(&ctas, cudaDevAttrMultiProcessorCount, dev)))
    return cuda_fail(e, "device attribute");
  ctas = ctas < kNaMaxCtas ? ctas : kNaMaxCtas;
  if (ctas > m) ctas = m;
  cudaStream_t st = (cudaStream_t)stream;
  k_noalloc_pass<<<ctas, kNaThreads, smem, st>>>(m, n, n_pad, row_ptr_dev, col_idx_dev, val_dev, row_w_dev, v_dev,
                                                 scratch);
  if ((e = cudaGetLastError())) return cuda_fail(e, "launch");
  k_noalloc_reduce<<<(n + 255) / 256, 256, 0, st>>>(n, ctas, scratch, v_dev, (float)(0.5 * rho), u_dev);
  if ((e = cudaGetLastError())) return cuda_fail(e, "launch");
  return RPT_OK;
}
