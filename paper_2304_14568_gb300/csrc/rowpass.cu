// Fused scenario row pass: the sparse products A_s v and A_s^T r of the
// x-subproblem (App. A, normal equations; Eq. 4 for the gradient) in ONE read
// of every stored entry.
//
// For a run of rows of scenario s, with v_s staged in shared memory:
//     t_i   = a_{s,i}^T v_s                       (gather from shared memory)
//     coef  = c_s w_i t_i            (kNormal)   -> acc += coef * a_{s,i}
//           = c_s w_i (t_i - p_i)    (kResid)    -> acc += coef * a_{s,i},
//                                                   obj += c_s w_i (t_i - p_i)^2
// so acc = sum_i c_s w_i a_i a_i^T v = A~_s^T A~_s v with A~_s = diag(sqrt(c_s w)) A_s
// (App. A) without ever forming A~_s.  The scatter goes to a per-CTA
// shared-memory accumulator of n floats (shared-memory atomics); each work
// unit then writes its accumulator as one partial, and the partials of a
// scenario are summed in a fixed order by the consumer kernel.
//
// Two implementations of the same pass:
//  * k_rowpass_tma (default): a persistent CTA per SM streams its slice of the
//    matrix through an S-stage shared-memory ring.  One producer lane issues
//    bulk asynchronous copies (cp.async.bulk, completion counted on an
//    mbarrier) of row-aligned chunks: the row records, the values and the
//    indices.  Fifteen consumer warps take rows of a resident chunk from a
//    shared counter, one warp per row, and release the stage through a second
//    mbarrier.  Every wait is bounded; a wait that runs out sets the plan's
//    error word and the kernel drains its copies and returns.
//  * k_rowpass (register path): nnz-balanced row blocks, one CTA each; warps
//    load row entries straight into registers with a one-row prefetch.
#include "common.cuh"

namespace rpt {
namespace {

template <typename VT> __device__ __forceinline__ float to_f(VT x);
template <> __device__ __forceinline__ float to_f<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <> __device__ __forceinline__ float to_f<__nv_fp8_e4m3>(__nv_fp8_e4m3 x) { return float(x); }

template <typename VT> __device__ __forceinline__ const VT* vals(const DevPlan& P);
template <> __device__ __forceinline__ const float* vals<float>(const DevPlan& P) { return P.val32; }
template <> __device__ __forceinline__ const __nv_bfloat16* vals<__nv_bfloat16>(const DevPlan& P) { return P.valbf; }
template <> __device__ __forceinline__ const __nv_fp8_e4m3* vals<__nv_fp8_e4m3>(const DevPlan& P) { return P.val8; }

template <typename IT> __device__ __forceinline__ const IT* cols(const DevPlan& P);
template <> __device__ __forceinline__ const int32_t* cols<int32_t>(const DevPlan& P) { return P.col32; }
template <> __device__ __forceinline__ const uint16_t* cols<uint16_t>(const DevPlan& P) { return P.col16; }

__host__ __device__ __forceinline__ size_t round128(size_t x) { return (x + 127) & ~(size_t)127; }

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy primitives (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase with the given parity to complete: gives up after
// one second of device time (try_wait itself may suspend the thread for a while,
// so the bound is on time, not on the number of tries).
constexpr unsigned long long kWaitLimitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
}
// Bulk copy global -> shared; completion is counted in bytes on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void named_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Stage v_s (scaled by the column scales of quantised values) into sv, zero acc.
template <bool kScatter>
__device__ __forceinline__ void stage_vector(const DevPlan& P, const float* __restrict__ vin, int v_stride,
                                             int s, float* sv, float* acc, int t0, int nt) {
  const float4* v4 = reinterpret_cast<const float4*>(vin + (size_t)s * v_stride);
  const float4* cs4 =
      P.colscale ? reinterpret_cast<const float4*>(P.colscale + (size_t)s * P.n_pad) : nullptr;
  float4* sv4 = reinterpret_cast<float4*>(sv);
  float4* acc4 = reinterpret_cast<float4*>(acc);
  for (int k = t0; k < P.n_pad / 4; k += nt) {
    float4 x = v4[k];
    if (cs4) {
      const float4 q = cs4[k];
      x.x *= q.x; x.y *= q.y; x.z *= q.z; x.w *= q.w;
    }
    sv4[k] = x;
    if (kScatter) acc4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

template <bool kScatter>
__device__ __forceinline__ void flush_acc(const DevPlan& P, int s, const float* acc, float* __restrict__ out,
                                          int t0, int nt) {
  if (!kScatter) return;
  float4* out4 = reinterpret_cast<float4*>(out);
  const float4* acc4 = reinterpret_cast<const float4*>(acc);
  const float4* cs4 =
      P.colscale ? reinterpret_cast<const float4*>(P.colscale + (size_t)s * P.n_pad) : nullptr;
  for (int k = t0; k < P.n_pad / 4; k += nt) {
    float4 x = acc4[k];
    if (cs4) {
      const float4 q = cs4[k];
      x.x *= q.x; x.y *= q.y; x.z *= q.z; x.w *= q.w;
    }
    out4[k] = x;
  }
}

// ---------------------------------------------------------------------------
// TMA-ring row pass
// ---------------------------------------------------------------------------
constexpr int kHdr = 512;   // mbarriers (2 x 8), row counters (8), per-warp objective (16 doubles)

template <int MODE, typename VT, typename IT>
__global__ void __launch_bounds__(kTmaThreads, 1)
k_rowpass_tma(DevPlan P, const float* __restrict__ vin, int v_stride, const int* __restrict__ active,
              float* __restrict__ partial, double* __restrict__ objp, float* __restrict__ dose) {
  constexpr bool kScatter = (MODE == kNormal || MODE == kResid);
  constexpr int NCW = kTmaThreads / 32 - 1;     // consumer warps
  constexpr int KR = 8;                         // entries per lane kept in registers
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + 8;
  int* rowctr = reinterpret_cast<int*>(smem + 128);
  double* wobj = reinterpret_cast<double*>(smem + 256);
  float* sv = reinterpret_cast<float*>(smem + kHdr);
  float* acc = sv + P.n_pad;
  const int S = P.stages;
  const size_t rec_bytes = round128((size_t)(P.rmax + 1) * 16);
  const size_t val_bytes = round128((size_t)P.cmax * sizeof(VT));
  const size_t col_bytes = round128((size_t)P.cmax * sizeof(IT));
  const size_t stage_bytes = rec_bytes + val_bytes + col_bytes;
  unsigned char* stage0 = smem + round128(kHdr + (size_t)P.n_pad * 4 * (kScatter ? 2 : 1));

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_u32(&full[i]), 1);
      mbar_init(smem_u32(&empty[i]), NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int seg0 = P.cta_seg[blockIdx.x], seg1 = P.cta_seg[blockIdx.x + 1];

  if (warp == 0) {
    // ---------------- producer ----------------
    if (lane == 0) {
      const VT* gval = vals<VT>(P);
      const IT* gcol = cols<IT>(P);
      int gk = 0;
      bool ok = true;
      for (int sg = seg0; sg < seg1 && ok; ++sg) {
        const int4 seg = P.segs[sg];
        if (active != nullptr && active[seg.x] == 0) continue;
        const int4* rec = P.rowrec + (size_t)seg.x * (P.m_act + 1);
        for (int c = seg.y; c < seg.z; ++c, ++gk) {
          const int st = gk % S;
          if (gk >= S && !mbar_wait(smem_u32(&empty[st]), (uint32_t)((gk / S) - 1) & 1u)) {
            ok = false;
            break;
          }
          const ChunkDesc ch = P.chunks[c];
          unsigned char* sp = stage0 + (size_t)st * stage_bytes;
          const uint32_t rb = (uint32_t)(ch.n_rows + 1) * 16u;
          const uint32_t vb = (uint32_t)ch.n_ent * (uint32_t)sizeof(VT);
          const uint32_t cb = (uint32_t)ch.n_ent * (uint32_t)sizeof(IT);
          rowctr[st] = 0;
          const uint32_t fb = smem_u32(&full[st]);
          mbar_arrive_expect_tx(fb, rb + vb + cb);
          bulk_g2s(smem_u32(sp), rec + ch.row_begin, rb, fb);
          bulk_g2s(smem_u32(sp + rec_bytes), gval + ch.g_al, vb, fb);
          bulk_g2s(smem_u32(sp + rec_bytes + val_bytes), gcol + ch.g_al, cb, fb);
        }
      }
      if (!ok) atomicExch(P.err, 1);
      // drain: the last use of every stage has completed before the CTA exits
      for (int q = (gk > S ? gk - S : 0); q < gk; ++q)
        if (!mbar_wait(smem_u32(&full[q % S]), (uint32_t)(q / S) & 1u)) atomicExch(P.err, 2);
    }
  } else {
    // ---------------- consumers ----------------
    const int cw = warp - 1;
    const int ct = tid - 32;
    int gk = 0;
    bool ok = true;
    for (int sg = seg0; sg < seg1; ++sg) {
      const int4 seg = P.segs[sg];
      const int s = seg.x;
      if (active != nullptr && active[s] == 0) continue;
      named_sync(1, NCW * 32);                     // previous segment fully flushed
      stage_vector<kScatter>(P, vin, v_stride, s, sv, acc, ct, NCW * 32);
      named_sync(1, NCW * 32);
      const long long base = P.nnz_base[s];
      double obj = 0.0;
      for (int c = seg.y; c < seg.z; ++c, ++gk) {
        const int st = gk % S;
        if (ok && !mbar_wait(smem_u32(&full[st]), (uint32_t)(gk / S) & 1u)) {
          ok = false;
          if (lane == 0) atomicExch(P.err, 3);
        }
        if (ok) {
          const ChunkDesc ch = P.chunks[c];
          const unsigned char* sp = stage0 + (size_t)st * stage_bytes;
          const int4* rec = reinterpret_cast<const int4*>(sp);
          const VT* val = reinterpret_cast<const VT*>(sp + rec_bytes);
          const IT* col = reinterpret_cast<const IT*>(sp + rec_bytes + val_bytes);
          const long long off = base - ch.g_al;
          for (;;) {
            int r = 0;
            if (lane == 0) r = atomicAdd(&rowctr[st], 1);
            r = __shfl_sync(0xffffffffu, r, 0);
            if (r >= ch.n_rows) break;
            const int4 ra = rec[r];
            const int lo = (int)(ra.x + off);
            const int hi = (int)(rec[r + 1].x + off);
            float vr[KR];
            int cr[KR];
            float t = 0.f;
#pragma unroll
            for (int k = 0; k < KR; ++k) {
              const int idx = lo + lane + 32 * k;
              if (idx < hi) {
                vr[k] = to_f<VT>(val[idx]);
                cr[k] = (int)col[idx];
                t = fmaf(vr[k], sv[cr[k]], t);
              } else {
                vr[k] = 0.f;
                cr[k] = 0;
              }
            }
            for (int idx = lo + 32 * KR + lane; idx < hi; idx += 32)
              t = fmaf(to_f<VT>(val[idx]), sv[(int)col[idx]], t);
            t = warp_sum(t);
            const float wc = __int_as_float(ra.y);
            float coef;
            if (MODE == kNormal) {
              coef = wc * t;
            } else {
              const float rr = t - __int_as_float(ra.z);
              coef = wc * rr;
              if (lane == 0) {
                obj += (double)(coef * rr);
                if (MODE == kDose) dose[(size_t)s * P.m_act + ch.row_begin + r] = t;
              }
            }
            if (kScatter) {
#pragma unroll
              for (int k = 0; k < KR; ++k)
                if (lo + lane + 32 * k < hi) atomicAdd(&acc[cr[k]], coef * vr[k]);
              for (int idx = lo + 32 * KR + lane; idx < hi; idx += 32)
                atomicAdd(&acc[(int)col[idx]], coef * to_f<VT>(val[idx]));
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&empty[st]));
      }
      if (lane == 0) wobj[cw] = obj;
      named_sync(1, NCW * 32);
      flush_acc<kScatter>(P, s, acc, partial + (size_t)seg.w * P.n_pad, ct, NCW * 32);
      if (MODE != kNormal && ct == 0) {
        double tsum = 0.0;
        for (int k = 0; k < NCW; ++k) tsum += wobj[k];
        objp[seg.w] = tsum;
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// register-path row pass
// ---------------------------------------------------------------------------
template <int KR, typename VT, typename IT>
struct RowRegs {
  float v[KR];
  int c[KR];
  __device__ __forceinline__ void load(const VT* __restrict__ val, const IT* __restrict__ col,
                                       int a, int b, int lane) {
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const int idx = a + lane + 32 * k;
      if (idx < b) {
        v[k] = to_f<VT>(val[idx]);
        c[k] = (int)col[idx];
      } else {
        v[k] = 0.f;
        c[k] = 0;
      }
    }
  }
};

template <int MODE, typename VT, typename IT, int KR>
__global__ void __launch_bounds__(kRowThreads, 2)
k_rowpass(DevPlan P, const float* __restrict__ vin, int v_stride, const int* __restrict__ active,
          float* __restrict__ partial, double* __restrict__ objp, float* __restrict__ dose) {
  constexpr bool kScatter = (MODE == kNormal || MODE == kResid);
  constexpr bool kObjective = (MODE != kNormal);
  extern __shared__ float4 smem4[];
  float* sv = reinterpret_cast<float*>(smem4);
  float* acc = sv + P.n_pad;
  __shared__ int next_row;
  __shared__ double wobj[kRowThreads / 32];

  const int4 blk = P.blocks[blockIdx.x];
  const int s = blk.x;
  if (active != nullptr && active[s] == 0) return;   // uniform over the CTA
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  stage_vector<kScatter>(P, vin, v_stride, s, sv, acc, tid, kRowThreads);
  if (tid == 0) next_row = blk.y;
  __syncthreads();

  const int32_t* rp = P.row_ptr + (size_t)s * (P.m_act + 1);
  const VT* __restrict__ val = vals<VT>(P) + P.nnz_base[s];
  const IT* __restrict__ col = cols<IT>(P) + P.nnz_base[s];
  const float cs = P.cs[s];
  double obj = 0.0;

  for (;;) {
    int r0 = 0;
    if (lane == 0) r0 = atomicAdd(&next_row, 32);
    r0 = __shfl_sync(0xffffffffu, r0, 0);
    if (r0 >= blk.z) break;
    const int nr = min(32, blk.z - r0);
    int ra = 0, rb = 0;
    float wl = 0.f, pl = 0.f;
    if (lane < nr) {
      ra = rp[r0 + lane];
      rb = rp[r0 + lane + 1];
      wl = P.w[r0 + lane] * cs;
      if (kObjective) pl = P.p[r0 + lane];
    }
    RowRegs<KR, VT, IT> cur, nxt;
    int a = __shfl_sync(0xffffffffu, ra, 0);
    int b = __shfl_sync(0xffffffffu, rb, 0);
    cur.load(val, col, a, b, lane);
    for (int q = 0; q < nr; ++q) {
      int an = 0, bn = 0;
      if (q + 1 < nr) {   // prefetch the next row while this one is processed
        an = __shfl_sync(0xffffffffu, ra, q + 1);
        bn = __shfl_sync(0xffffffffu, rb, q + 1);
        nxt.load(val, col, an, bn, lane);
      }
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < KR; ++k) t = fmaf(cur.v[k], sv[cur.c[k]], t);
      // rest of a long row: batches of 32*KR independent loads
      for (int base = a + 32 * KR; base < b; base += 32 * KR) {
        RowRegs<KR, VT, IT> tl;
        tl.load(val, col, base, b, lane);
#pragma unroll
        for (int k = 0; k < KR; ++k) t = fmaf(tl.v[k], sv[tl.c[k]], t);
      }
      t = warp_sum(t);
      const float wc = __shfl_sync(0xffffffffu, wl, q);
      float coef = 0.f;
      if (MODE == kNormal) {
        coef = wc * t;
      } else {
        const float r = t - __shfl_sync(0xffffffffu, pl, q);
        coef = wc * r;
        if (lane == 0) {
          obj += (double)(coef * r);
          if (MODE == kDose) dose[(size_t)s * P.m_act + r0 + q] = t;
        }
      }
      if (kScatter && b > a) {
#pragma unroll
        for (int k = 0; k < KR; ++k)
          if (a + lane + 32 * k < b) atomicAdd(&acc[cur.c[k]], coef * cur.v[k]);
        for (int idx = a + 32 * KR + lane; idx < b; idx += 32)
          atomicAdd(&acc[(int)col[idx]], coef * to_f<VT>(val[idx]));
      }
      if (q + 1 < nr) {
        cur = nxt;
        a = an;
        b = bn;
      }
    }
  }

  if (kObjective && lane == 0) wobj[wid] = obj;
  __syncthreads();
  flush_acc<kScatter>(P, s, acc, partial + (size_t)blockIdx.x * P.n_pad, tid, kRowThreads);
  if (kObjective && tid == 0) {
    double t = 0.0;
    for (int k = 0; k < kRowThreads / 32; ++k) t += wobj[k];
    objp[blockIdx.x] = t;
  }
}

constexpr int kKR = 4;

template <int MODE>
void* pick(const DevPlan& P) {
  if (P.path == 1) {
    if (P.index_width == 16) {
      switch (P.value_format) {
        case 1: return (void*)k_rowpass_tma<MODE, __nv_bfloat16, uint16_t>;
        case 2: return (void*)k_rowpass_tma<MODE, __nv_fp8_e4m3, uint16_t>;
        default: return (void*)k_rowpass_tma<MODE, float, uint16_t>;
      }
    }
    switch (P.value_format) {
      case 1: return (void*)k_rowpass_tma<MODE, __nv_bfloat16, int32_t>;
      case 2: return (void*)k_rowpass_tma<MODE, __nv_fp8_e4m3, int32_t>;
      default: return (void*)k_rowpass_tma<MODE, float, int32_t>;
    }
  }
  if (P.index_width == 16) {
    switch (P.value_format) {
      case 1: return (void*)k_rowpass<MODE, __nv_bfloat16, uint16_t, kKR>;
      case 2: return (void*)k_rowpass<MODE, __nv_fp8_e4m3, uint16_t, kKR>;
      default: return (void*)k_rowpass<MODE, float, uint16_t, kKR>;
    }
  }
  switch (P.value_format) {
    case 1: return (void*)k_rowpass<MODE, __nv_bfloat16, int32_t, kKR>;
    case 2: return (void*)k_rowpass<MODE, __nv_fp8_e4m3, int32_t, kKR>;
    default: return (void*)k_rowpass<MODE, float, int32_t, kKR>;
  }
}

}  // namespace

size_t tma_smem_bytes(int n_pad, int cmax, int rmax, int stages, int value_bytes, int index_bytes,
                      bool scatter) {
  const size_t stage = round128((size_t)(rmax + 1) * 16) + round128((size_t)cmax * value_bytes) +
                       round128((size_t)cmax * index_bytes);
  return round128(kHdr + (size_t)n_pad * 4 * (scatter ? 2 : 1)) + (size_t)stages * stage;
}

void* rowpass_kernel(const DevPlan& P, int mode) {
  switch (mode) {
    case kNormal: return pick<kNormal>(P);
    case kResid: return pick<kResid>(P);
    case kObj: return pick<kObj>(P);
    default: return pick<kDose>(P);
  }
}

size_t rowpass_smem(const DevPlan& P, int mode) {
  const bool scatter = (mode == kNormal || mode == kResid);
  if (P.path == 1) {
    const int vb = P.value_format == 0 ? 4 : (P.value_format == 1 ? 2 : 1);
    const int ib = P.index_width == 16 ? 2 : 4;
    return tma_smem_bytes(P.n_pad, P.cmax, P.rmax, P.stages, vb, ib, scatter);
  }
  return (size_t)P.n_pad * sizeof(float) * (scatter ? 2 : 1);
}

int rowpass_threads(const DevPlan& P) { return P.path == 1 ? kTmaThreads : kRowThreads; }

// The dynamic shared-memory cap is a per-function, process-wide attribute, so
// it is raised to the device's opt-in maximum (never lowered): plans with
// different stage sizes can then coexist.
cudaError_t rowpass_prepare(const DevPlan& P) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  for (int mode = 0; mode < 4; ++mode) {
    void* fn = rowpass_kernel(P, mode);
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
    const int cap = optin - (int)fa.sharedSizeBytes;   // static shared memory counts against the cap
    if (rowpass_smem(P, mode) > (size_t)cap) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace rpt
