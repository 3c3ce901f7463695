// Learned warm start: a small multilayer perceptron that maps a plan's
// objective weights (features chosen by the caller, e.g. the log structure
// weights and the prescription) to a spot vector, used as z^0 of ADMM-BB.  The
// paper has no learned part; this is the library's optional warm-start form.
//
// Network: n_in -> H -> ... -> H (L hidden layers, ReLU) -> n_out (linear).
// Loss: mean squared error over the batch and the outputs.  Training: Adam on
// minibatches drawn from a seeded permutation every epoch.  Everything runs in
// the library's kernels: the GEMMs with their fused bias/ReLU epilogue, the ReLU
// and bias gradients, the loss gradient and the Adam update.  Two compute forms:
//   BF16 (default): weights, activations and activation gradients enter the
//     GEMMs as bfloat16 and the tensor cores accumulate in FP32 (gemm_bf16.cuh,
//     mma.sync); the FP32 master weights take the Adam step and are rounded to
//     the bfloat16 copy after it; biases, losses and gradients stay FP32.
//   F32: the tiled shared-memory FP32 GEMM of gemm.cuh on the CUDA cores.
// The network is small (under a million weights, batches of a few hundred rows),
// so its GEMMs are latency- and launch-bound either way.
//
// Parameter layout (one float array): for each layer l, W_l (row-major,
// [out_l][in_l]) followed by b_l ([out_l]).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "gemm.cuh"
#include "gemm_bf16.cuh"
#include "plan.h"

namespace rpt {
namespace {

// dH *= (H > 0)   (ReLU backward; H is the layer's output after ReLU)
__global__ void k_relu_bwd(int64_t n, const float* __restrict__ H, float* __restrict__ dH) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    if (!(H[k] > 0.f)) dH[k] = 0.f;
}

// db[j] = sum_i dH[i][j]  (one block per 256 columns; fixed summation order)
__global__ void k_bias_grad(int M, int N, const float* __restrict__ dH, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int i = 0; i < M; ++i) s += dH[(size_t)i * N + j];
  db[j] = s;
}

// dOut = 2 (Out - Y) / (M N); loss += sum (Out - Y)^2 / (M N)  (FP64 partial sums)
__global__ void k_mse(int64_t n, const float* __restrict__ out, const float* __restrict__ y, float* __restrict__ d,
                      double inv, double* __restrict__ loss) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const float e = out[k] - y[k];
    d[k] = (float)(2.0 * inv) * e;
    acc += (double)e * e;
  }
  double v[1] = {acc};
  block_sum_d<1>(v, sh);
  if (threadIdx.x == 0) atomicAdd(loss, v[0] * inv);
}

// Adam (Kingma & Ba, Algorithm 1) with bias correction folded into the step size.
__global__ void k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr_t, float b1, float b2, float eps, float wd) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const float gk = g[k] + wd * p[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr_t * mk / (sqrtf(vk) + eps);
  }
}

__global__ void k_to_bf16(int64_t n, const float* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = __float2bfloat16_rn(src[k]);
}

__global__ void k_gather_rows(int rows, int cols, const int* __restrict__ idx, const float* __restrict__ src,
                              float* __restrict__ dst) {
  const int64_t n = (int64_t)rows * cols;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(k / cols), c = (int)(k % cols);
    dst[k] = src[(size_t)idx[r] * cols + c];
  }
}

}  // namespace

struct Mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<int> dims;              // n_in, H, ..., H, n_out
  std::vector<int64_t> woff, boff;    // offsets of W_l, b_l in the parameter array
  int64_t nparam = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  int bf16 = 1;                       // compute form: 1 bfloat16 tensor cores, 0 FP32 CUDA cores
  __nv_bfloat16* pb = nullptr;        // bfloat16 copy of p (the weights the BF16 GEMMs read)
  std::vector<__nv_bfloat16*> actb, dactb;   // bfloat16 copies of act / dact
  int cap = 0;                        // rows the activation buffers hold
  std::vector<float*> act;            // act[0] = input batch, act[l+1] = output of layer l
  std::vector<float*> dact;           // gradients w.r.t. act[l+1]
  float* y = nullptr;                 // target batch
  double* loss = nullptr;
  int* idx = nullptr;
  float *xall = nullptr, *yall = nullptr;
  int nall = 0;
  int64_t step = 0;                   // Adam steps taken
};

namespace {

void free_acts(Mlp* M) {
  for (float* a : M->act) cudaFree(a);
  for (float* a : M->dact) cudaFree(a);
  for (__nv_bfloat16* a : M->actb) cudaFree(a);
  for (__nv_bfloat16* a : M->dactb) cudaFree(a);
  M->act.clear();
  M->dact.clear();
  M->actb.clear();
  M->dactb.clear();
  cudaFree(M->y);
  M->y = nullptr;
  cudaFree(M->idx);
  M->idx = nullptr;
  M->cap = 0;
}

cudaError_t ensure_cap(Mlp* M, int rows) {
  if (rows <= M->cap) return cudaSuccess;
  free_acts(M);
  const int L = (int)M->dims.size() - 1;
  cudaError_t e = cudaSuccess;
  M->act.assign(L + 1, nullptr);
  M->dact.assign(L + 1, nullptr);
  M->actb.assign(L + 1, nullptr);
  M->dactb.assign(L + 1, nullptr);
  for (int l = 0; l <= L && e == cudaSuccess; ++l) {
    e = cudaMalloc(&M->act[l], sizeof(float) * (size_t)rows * M->dims[l]);
    if (e == cudaSuccess) e = cudaMalloc(&M->dact[l], sizeof(float) * (size_t)rows * M->dims[l]);
    if (e == cudaSuccess) e = cudaMalloc(&M->actb[l], sizeof(__nv_bfloat16) * (size_t)rows * M->dims[l]);
    if (e == cudaSuccess) e = cudaMalloc(&M->dactb[l], sizeof(__nv_bfloat16) * (size_t)rows * M->dims[l]);
  }
  if (e == cudaSuccess) e = cudaMalloc(&M->y, sizeof(float) * (size_t)rows * M->dims[L]);
  if (e == cudaSuccess) e = cudaMalloc(&M->idx, sizeof(int) * (size_t)rows);
  if (e == cudaSuccess) M->cap = rows;
  return e;
}

int blocks_for(int64_t n) { return (int)std::min<int64_t>(4096, std::max<int64_t>(1, (n + 255) / 256)); }

// Forward pass of `rows` rows already in act[0].
void forward(Mlp* M, int rows) {
  const int L = (int)M->dims.size() - 1;
  if (M->bf16) {
    const int64_t n0 = (int64_t)rows * M->dims[0];
    k_to_bf16<<<blocks_for(n0), 256, 0, M->stream>>>(n0, M->act[0], M->actb[0]);
  }
  for (int l = 0; l < L; ++l) {
    const int in = M->dims[l], out = M->dims[l + 1];
    if (M->bf16)
      gemm_bf16<false, true>(M->stream, rows, out, in, M->actb[l], in, M->pb + M->woff[l], in, M->act[l + 1], out,
                             M->actb[l + 1], M->p + M->boff[l], l + 1 < L);
    else
      gemm<false, true>(M->stream, rows, out, in, M->act[l], in, M->p + M->woff[l], in, M->act[l + 1], out,
                        M->p + M->boff[l], l + 1 < L);
  }
}

// Loss and gradient of the batch (targets in M->y) into M->g; returns through M->loss.
void backward(Mlp* M, int rows) {
  const int L = (int)M->dims.size() - 1;
  const int nout = M->dims[L];
  const int64_t n = (int64_t)rows * nout;
  cudaMemsetAsync(M->loss, 0, sizeof(double), M->stream);
  k_mse<<<blocks_for(n), 256, 0, M->stream>>>(n, M->act[L], M->y, M->dact[L], 1.0 / (double)n, M->loss);
  for (int l = L - 1; l >= 0; --l) {
    const int in = M->dims[l], out = M->dims[l + 1];
    if (l + 1 < L) {
      const int64_t k = (int64_t)rows * out;
      k_relu_bwd<<<blocks_for(k), 256, 0, M->stream>>>(k, M->act[l + 1], M->dact[l + 1]);
    }
    k_bias_grad<<<(out + 255) / 256, 256, 0, M->stream>>>(rows, out, M->dact[l + 1], M->g + M->boff[l]);
    if (M->bf16) {
      const int64_t k = (int64_t)rows * out;
      k_to_bf16<<<blocks_for(k), 256, 0, M->stream>>>(k, M->dact[l + 1], M->dactb[l + 1]);
      // dW_l = dAct_{l+1}^T act_l   ([out][rows] x [rows][in])
      gemm_bf16<true, false>(M->stream, out, in, rows, M->dactb[l + 1], out, M->actb[l], in, M->g + M->woff[l],
                             in);
      // dAct_l = dAct_{l+1} W_l   ([rows][out] x [out][in]); not needed for the input
      if (l > 0)
        gemm_bf16<false, false>(M->stream, rows, in, out, M->dactb[l + 1], out, M->pb + M->woff[l], in,
                                M->dact[l], in);
    } else {
      gemm<true, false>(M->stream, out, in, rows, M->dact[l + 1], out, M->act[l], in, M->g + M->woff[l], in,
                        nullptr, false);
      if (l > 0)
        gemm<false, false>(M->stream, rows, in, out, M->dact[l + 1], out, M->p + M->woff[l], in, M->dact[l], in,
                           nullptr, false);
    }
  }
}

int check(cudaError_t e, const char* what) { return e == cudaSuccess ? RPT_OK : cuda_fail(e, what); }

// the bfloat16 copy of the weights, after every change of the FP32 ones
cudaError_t refresh_bf16(Mlp* M) {
  k_to_bf16<<<blocks_for(M->nparam), 256, 0, M->stream>>>(M->nparam, M->p, M->pb);
  return cudaGetLastError();
}

}  // namespace
}  // namespace rpt

using namespace rpt;

extern "C" {

int rpt_mlp_train_params_default(rpt_mlp_train_params* tp) {
  if (!tp) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  tp->epochs = 300;
  tp->batch = 128;
  tp->lr = 1e-3;
  tp->beta1 = 0.9;
  tp->beta2 = 0.999;
  tp->eps = 1e-8;
  tp->weight_decay = 0.0;
  tp->seed = 1;
  return RPT_OK;
}

int rpt_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_hidden_layers, int32_t n_out, uint64_t seed,
                   int32_t device, rpt_mlp** out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_hidden_layers < 0 || n_out < 1 || n_hidden_layers > 16) {
    set_error("rpt_mlp_create: bad argument");
    return RPT_EINVAL;
  }
  *out = nullptr;
  Mlp* M = new (std::nothrow) Mlp();
  if (!M) {
    set_error("out of host memory");
    return RPT_ENOMEM;
  }
  M->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking);
  M->dims.push_back(n_in);
  for (int l = 0; l < n_hidden_layers; ++l) M->dims.push_back(n_hidden);
  M->dims.push_back(n_out);
  const int L = (int)M->dims.size() - 1;
  for (int l = 0; l < L; ++l) {
    M->woff.push_back(M->nparam);
    M->nparam += (int64_t)M->dims[l] * M->dims[l + 1];
    M->boff.push_back(M->nparam);
    M->nparam += M->dims[l + 1];
  }
  // Glorot-uniform weights, zero biases, from a seeded host generator
  std::vector<float> h((size_t)M->nparam, 0.f);
  std::mt19937_64 gen(seed);
  for (int l = 0; l < L; ++l) {
    const float a = std::sqrt(6.f / (float)(M->dims[l] + M->dims[l + 1]));
    std::uniform_real_distribution<float> U(-a, a);
    for (int64_t k = 0; k < (int64_t)M->dims[l] * M->dims[l + 1]; ++k) h[(size_t)(M->woff[l] + k)] = U(gen);
  }
  const size_t bytes = sizeof(float) * (size_t)M->nparam;
  if (e == cudaSuccess) e = cudaMalloc(&M->p, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&M->g, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&M->m, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&M->v, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&M->loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&M->pb, sizeof(__nv_bfloat16) * (size_t)M->nparam);
  if (e == cudaSuccess) e = cudaMemcpy(M->p, h.data(), bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = refresh_bf16(M);
  if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
  if (e == cudaSuccess) e = cudaMemset(M->m, 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(M->v, 0, bytes);
  if (e != cudaSuccess) {
    rpt_mlp_destroy(reinterpret_cast<rpt_mlp*>(M));
    return cuda_fail(e, "rpt_mlp_create");
  }
  *out = reinterpret_cast<rpt_mlp*>(M);
  return RPT_OK;
}

int rpt_mlp_destroy(rpt_mlp* mlp) {
  if (!mlp) return RPT_OK;
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  cudaSetDevice(M->device);
  if (M->stream) cudaStreamSynchronize(M->stream);
  free_acts(M);
  cudaFree(M->p);
  cudaFree(M->g);
  cudaFree(M->m);
  cudaFree(M->v);
  cudaFree(M->loss);
  cudaFree(M->pb);
  cudaFree(M->xall);
  cudaFree(M->yall);
  if (M->stream) cudaStreamDestroy(M->stream);
  delete M;
  return RPT_OK;
}

int rpt_mlp_param_count(const rpt_mlp* mlp, int64_t* count) {
  if (!mlp || !count) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  *count = reinterpret_cast<const Mlp*>(mlp)->nparam;
  return RPT_OK;
}

int rpt_mlp_get_params(rpt_mlp* mlp, float* params) {
  if (!mlp || !params) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  cudaSetDevice(M->device);
  cudaError_t e = cudaMemcpyAsync(params, M->p, sizeof(float) * (size_t)M->nparam, cudaMemcpyDeviceToHost,
                                  M->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
  return check(e, "rpt_mlp_get_params");
}

int rpt_mlp_set_params(rpt_mlp* mlp, const float* params) {
  if (!mlp || !params) {
    set_error("null argument");
    return RPT_EINVAL;
  }
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  cudaSetDevice(M->device);
  const size_t bytes = sizeof(float) * (size_t)M->nparam;
  cudaError_t e = cudaMemcpyAsync(M->p, params, bytes, cudaMemcpyHostToDevice, M->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(M->m, 0, bytes, M->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(M->v, 0, bytes, M->stream);
  if (e == cudaSuccess) e = refresh_bf16(M);
  if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
  M->step = 0;
  return check(e, "rpt_mlp_set_params");
}

int rpt_mlp_set_compute(rpt_mlp* mlp, int32_t value_format) {
  if (!mlp || (value_format != RPT_F32 && value_format != RPT_BF16)) {
    set_error("rpt_mlp_set_compute: need a network and RPT_F32 or RPT_BF16");
    return RPT_EINVAL;
  }
  reinterpret_cast<Mlp*>(mlp)->bf16 = value_format == RPT_BF16 ? 1 : 0;
  return RPT_OK;
}

int rpt_mlp_predict(rpt_mlp* mlp, const float* X, int32_t n, float* Y) {
  if (!mlp || !X || !Y || n < 1) {
    set_error("rpt_mlp_predict: bad argument");
    return RPT_EINVAL;
  }
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  cudaSetDevice(M->device);
  cudaError_t e = ensure_cap(M, n);
  const int L = (int)M->dims.size() - 1;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(M->act[0], X, sizeof(float) * (size_t)n * M->dims[0], cudaMemcpyHostToDevice, M->stream);
  if (e == cudaSuccess) {
    forward(M, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Y, M->act[L], sizeof(float) * (size_t)n * M->dims[L], cudaMemcpyDeviceToHost, M->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
  return check(e, "rpt_mlp_predict");
}

int rpt_mlp_infer(rpt_mlp* mlp, const float* features, float* z0_out) {
  if (!mlp || !features || !z0_out) {
    set_error("rpt_mlp_infer: bad argument");
    return RPT_EINVAL;
  }
  return rpt_mlp_predict(mlp, features, 1, z0_out);
}

int rpt_mlp_loss_grad(rpt_mlp* mlp, const float* X, const float* Y, int32_t n, double* loss, float* grad) {
  if (!mlp || !X || !Y || n < 1) {
    set_error("rpt_mlp_loss_grad: bad argument");
    return RPT_EINVAL;
  }
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  cudaSetDevice(M->device);
  const int L = (int)M->dims.size() - 1;
  cudaError_t e = ensure_cap(M, n);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(M->act[0], X, sizeof(float) * (size_t)n * M->dims[0], cudaMemcpyHostToDevice, M->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(M->y, Y, sizeof(float) * (size_t)n * M->dims[L], cudaMemcpyHostToDevice, M->stream);
  if (e == cudaSuccess) {
    forward(M, n);
    backward(M, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, M->loss, sizeof(double), cudaMemcpyDeviceToHost, M->stream);
  if (e == cudaSuccess && grad)
    e = cudaMemcpyAsync(grad, M->g, sizeof(float) * (size_t)M->nparam, cudaMemcpyDeviceToHost, M->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
  return check(e, "rpt_mlp_loss_grad");
}

int rpt_mlp_train(rpt_mlp* mlp, const float* X, const float* Y, int32_t n, const rpt_mlp_train_params* tp,
                  double* final_loss) {
  if (!mlp || !X || !Y || !tp || n < 1 || tp->epochs < 0 || tp->batch < 1 || !(tp->lr > 0.0)) {
    set_error("rpt_mlp_train: bad argument");
    return RPT_EINVAL;
  }
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  cudaSetDevice(M->device);
  const int L = (int)M->dims.size() - 1;
  const int nin = M->dims[0], nout = M->dims[L];
  const int B = std::min<int>(tp->batch, n);
  cudaError_t e = ensure_cap(M, B);
  if (e == cudaSuccess && n > M->nall) {
    cudaFree(M->xall);
    cudaFree(M->yall);
    M->xall = M->yall = nullptr;
    M->nall = 0;
    e = cudaMalloc(&M->xall, sizeof(float) * (size_t)n * nin);
    if (e == cudaSuccess) e = cudaMalloc(&M->yall, sizeof(float) * (size_t)n * nout);
    if (e == cudaSuccess) M->nall = n;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(M->xall, X, sizeof(float) * (size_t)n * nin, cudaMemcpyHostToDevice, M->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(M->yall, Y, sizeof(float) * (size_t)n * nout, cudaMemcpyHostToDevice, M->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rpt_mlp_train");
  std::mt19937_64 gen(tp->seed);
  std::vector<int> perm(n), ibuf;
  for (int i = 0; i < n; ++i) perm[i] = i;
  // one index upload per epoch (all batches of the epoch)
  int* d_perm = nullptr;
  if ((e = cudaMalloc(&d_perm, sizeof(int) * (size_t)n))) return cuda_fail(e, "rpt_mlp_train");
  double last = 0.0;
  const float b1 = (float)tp->beta1, b2 = (float)tp->beta2;
  for (int ep = 0; ep < tp->epochs && e == cudaSuccess; ++ep) {
    std::shuffle(perm.begin(), perm.end(), gen);
    e = cudaMemcpyAsync(d_perm, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, M->stream);
    for (int b0 = 0; b0 + B <= n && e == cudaSuccess; b0 += B) {   // full batches only
      k_gather_rows<<<blocks_for((int64_t)B * nin), 256, 0, M->stream>>>(B, nin, d_perm + b0, M->xall, M->act[0]);
      k_gather_rows<<<blocks_for((int64_t)B * nout), 256, 0, M->stream>>>(B, nout, d_perm + b0, M->yall, M->y);
      forward(M, B);
      backward(M, B);
      M->step += 1;
      const double bc1 = 1.0 - std::pow(tp->beta1, (double)M->step);
      const double bc2 = 1.0 - std::pow(tp->beta2, (double)M->step);
      const float lr_t = (float)(tp->lr * std::sqrt(bc2) / bc1);
      k_adam<<<blocks_for(M->nparam), 256, 0, M->stream>>>(M->nparam, M->p, M->g, M->m, M->v, lr_t, b1, b2,
                                                           (float)tp->eps, (float)tp->weight_decay);
      e = cudaGetLastError();
      if (e == cudaSuccess && M->bf16) e = refresh_bf16(M);
    }
    // stream ordering keeps the host-side permutation valid: wait before the next shuffle
    if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
  }
  if (e == cudaSuccess) e = cudaMemcpy(&last, M->loss, sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d_perm);
  if (e != cudaSuccess) return cuda_fail(e, "rpt_mlp_train");
  if (final_loss) *final_loss = last;
  return RPT_OK;
}

int rpt_admm_bb_solve_learned(rpt_plan* plan, rpt_mlp* mlp, const float* features, const double* zscale,
                              const rpt_admm_params* params, double* x_out, rpt_solve_info* info,
                              int32_t* used_warm_start) {
  if (!plan || !mlp || !features || !zscale || !x_out) {
    set_error("rpt_admm_bb_solve_learned: null argument");
    return RPT_EINVAL;
  }
  rpt_plan_stats st;
  int rc = rpt_plan_query(plan, &st);
  if (rc != RPT_OK) return rc;
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  if (M->dims.back() != st.n) {
    set_error("rpt_admm_bb_solve_learned: network output width != plan spots");
    return RPT_EINVAL;
  }
  std::vector<float> pred((size_t)st.n);
  if ((rc = rpt_mlp_predict(mlp, features, 1, pred.data())) != RPT_OK) return rc;
  std::vector<double> z0((size_t)st.n);
  for (int j = 0; j < st.n; ++j) z0[j] = (double)pred[j] * zscale[j];   // the solver projects z0 onto [lb, ub]
  if (used_warm_start) *used_warm_start = 1;
  rc = rpt_admm_bb_solve(plan, params, z0.data(), nullptr, x_out, info);
  if (rc == RPT_OK) return rc;
  if (rc != RPT_NOT_CONVERGED && rc != RPT_DIVERGED) return rc;
  // fallback: the cold-start method
  if (used_warm_start) *used_warm_start = 0;
  rpt_solve_info warm{};
  if (info) warm = *info;
  rc = rpt_admm_bb_solve(plan, params, nullptr, nullptr, x_out, info);
  if (info) {
    info->iterations += warm.iterations;
    info->inner += warm.inner;
    info->row_passes += warm.row_passes;
    info->kernels += warm.kernels;
    info->seconds += warm.seconds;
  }
  return rc;
}

}  // extern "C"
