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
//    indices; it publishes each chunk's descriptor in shared memory and
//    prefetches the next one.  The other 31 warps consume: they split the rows of a
//    resident chunk statically in groups of lanes (one group per row), and
//    release the stage through a second mbarrier.  Every wait is bounded; a wait that runs out sets the plan's
//    error word and the kernel drains its copies and returns.
//  * k_rowpass (register path): nnz-balanced row blocks, one CTA each; warps
//    load row entries straight into registers with a one-row prefetch.
//  * k_rowpass_stream (rowstream.cu): persistent CTAs whose warps claim chunks
//    on their own and stream the entries straight into registers.
#include "rowcommon.cuh"

namespace rpt {
namespace {


// ---------------------------------------------------------------------------
// mbarrier / bulk-copy primitives (inline PTX)
// ---------------------------------------------------------------------------
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

// One group of G lanes processes one row (G in {1, 2, ..., 32}); a warp covers
// 32/G rows at once.  Lane sl of the group takes entries sl, sl + G, ... so that
// the lanes of one instruction touch consecutive entries (consecutive spot
// columns fall in different shared-memory banks for the gather and the scatter).
// Each lane keeps up to KR of its row's entries in registers between the dot and
// the scatter; longer rows (only with G = 32) re-read the rest.  Padding entries
// have value 0: they add nothing to the dot and the scatter skips them.
template <int MODE, typename VT, typename IT, int KR>
__device__ __forceinline__ void process_rows(const int4* __restrict__ rec, int r, bool valid, int G, int sl,
                                             const VT* __restrict__ val, const IT* __restrict__ col,
                                             long long off, const float* sv, float* acc, double& obj,
                                             float* __restrict__ dose, size_t dose_base) {
  constexpr bool kScatter = (MODE == kNormal || MODE == kResid);
  int4 ra = make_int4(0, 0, 0, 0);
  int lo = 0, hi = 0;
  if (valid) {
    ra = rec[r];
    lo = (int)(ra.x + off);
    hi = (int)(rec[r + 1].x + off);
  }
  float vr[KR];
  int cr[KR];
  float t = 0.f;
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const int idx = lo + sl + G * k;
    if (idx < hi) {
      vr[k] = to_f<VT>(val[idx]);
      cr[k] = (int)col[idx];
      t = fmaf(vr[k], sv[cr[k]], t);
    } else {
      vr[k] = 0.f;
      cr[k] = 0;
    }
  }
  for (int idx = lo + G * KR + sl; idx < hi; idx += G) t = fmaf(to_f<VT>(val[idx]), sv[(int)col[idx]], t);
  for (int o = G >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  const float wc = __int_as_float(ra.y);
  float coef;
  if (MODE == kNormal) {
    coef = wc * t;
  } else {
    const float rr = t - __int_as_float(ra.z);
    coef = wc * rr;
    if (valid && sl == 0) {
      obj += (double)(coef * rr);
      if (MODE == kDose) dose[dose_base + ra.w] = t;
    }
  }
  if (kScatter) {
#pragma unroll
    for (int k = 0; k < KR; ++k)
      if (vr[k] != 0.f) atomicAdd(&acc[cr[k]], coef * vr[k]);
    for (int idx = lo + G * KR + sl; idx < hi; idx += G) {
      const float a = to_f<VT>(val[idx]);
      if (a != 0.f) atomicAdd(&acc[(int)col[idx]], coef * a);
    }
  }
}

// ---------------------------------------------------------------------------
// TMA-ring row pass
// ---------------------------------------------------------------------------
constexpr int kHdr = 1024;  // mbarriers (2 x 8 x 8 B), chunk descriptors (8 x 32 B), per-warp objective (up to 64 doubles)
constexpr int kBatch = 4;   // chunks per queue pull

template <int MODE, typename VT, typename IT>
__global__ void __launch_bounds__(kTmaThreads, 1)
k_rowpass_tma(DevPlan P, const float* __restrict__ vin, int v_stride, const int* __restrict__ active,
              float* __restrict__ partial, double* __restrict__ objp, float* __restrict__ dose) {
  constexpr bool kScatter = (MODE == kNormal || MODE == kResid);
  constexpr int NCW = kTmaThreads / 32 - 1;     // consumer warps (wobj below holds up to 64)
  constexpr int KR = 8;                         // entries per lane kept in registers
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + 8;
  ChunkDesc* sdesc = reinterpret_cast<ChunkDesc*>(smem + 128);   // one per stage
  double* wobj = reinterpret_cast<double*>(smem + 512);
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

  if (warp == 0) {
    // ---------------- producer (one lane) ----------------
    if (lane == 0) {
      const VT* gval = vals<VT>(P);
      const IT* gcol = cols<IT>(P);
      int st = 0, ph = 0, issued = 0;
      bool ok = true;
      // walk the scenarios starting at this CTA's home scenario, taking chunks
      // from each scenario's queue until all queues are empty
      const int home = (int)(((long long)blockIdx.x * P.N) / gridDim.x);
      for (int k = 0; k < P.N && ok && !P.inject_timeout; ++k) {
        const int sc = (home + k) % P.N;
        if (active != nullptr && active[sc] == 0) continue;
        const int c0 = P.scen_chunk[sc], c1 = P.scen_chunk[sc + 1];
        // chunks are pulled in batches of kBatch; the next batch is requested when
        // a batch starts and each descriptor is fetched one chunk ahead, so the
        // queue and descriptor latencies overlap the stage waits
        int cb = c0 + kBatch * atomicAdd(&P.qnext[sc], 1);
        ChunkDesc nxt{};
        if (cb < c1) nxt = P.chunks[cb];
        while (cb < c1 && ok) {
          const int cbn = c0 + kBatch * atomicAdd(&P.qnext[sc], 1);
          const int ce = min(cb + kBatch, c1);
          for (int c = cb; c < ce; ++c) {
          const ChunkDesc ch = nxt;
          const int nn = (c + 1 < ce) ? c + 1 : cbn;
          if (nn < c1) nxt = P.chunks[nn];
          // stage st is free once its previous use (phase ph ^ 1) was released
          if (issued >= S && !mbar_wait(smem_u32(&empty[st]), (uint32_t)(ph ^ 1))) {
            ok = false;
            break;
          }
          unsigned char* sp = stage0 + (size_t)st * stage_bytes;
          const uint32_t rb = (uint32_t)(ch.n_rows + 1) * 16u;
          const uint32_t vb = (uint32_t)ch.n_ent * (uint32_t)sizeof(VT);
          const uint32_t cb = (uint32_t)ch.n_ent * (uint32_t)sizeof(IT);
          const int4* rec = P.rowrec + P.rec_base[sc];
          sdesc[st] = ch;
          const uint32_t fb = smem_u32(&full[st]);
          mbar_arrive_expect_tx(fb, rb + vb + cb);
          bulk_g2s(smem_u32(sp), rec + ch.row_begin, rb, fb);
          bulk_g2s(smem_u32(sp + rec_bytes), gval + ch.g_al, vb, fb);
          bulk_g2s(smem_u32(sp + rec_bytes + val_bytes), gcol + ch.g_al, cb, fb);
          ++issued;
          if (++st == S) {
            st = 0;
            ph ^= 1;
          }
          }
          cb = cbn;
        }
      }
      // end-of-work marker in the next stage (none when a timeout is injected)
      if (P.inject_timeout) {
        ok = true;
      } else if (ok && (issued < S || mbar_wait(smem_u32(&empty[st]), (uint32_t)(ph ^ 1)))) {
        ChunkDesc endm{};
        endm.n_rows = -1;
        sdesc[st] = endm;
        mbar_arrive(smem_u32(&full[st]));
        ++issued;
        if (++st == S) {
          st = 0;
          ph ^= 1;
        }
      } else {
        ok = false;
      }
      if (!ok) atomicExch(P.err, 1);
      // drain: the last use of every stage has completed before the CTA exits
      for (int q = 0; q < S && q < issued; ++q) {
        if (--st < 0) {
          st = S - 1;
          ph ^= 1;
        }
        if (!mbar_wait(smem_u32(&full[st]), (uint32_t)ph)) atomicExch(P.err, 2);
      }
    }
  } else {
    // ---------------- consumers ----------------
    const int cw = warp - 1;
    const int ct = tid - 32;
    int st = 0, ph = 0;
    int s = -1;                 // scenario whose vector is staged
    long long base = 0;
    double obj = 0.0;
    for (;;) {
      if (!mbar_wait(smem_u32(&full[st]), (uint32_t)ph)) {
        if (lane == 0) atomicExch(P.err, 3);
        break;
      }
      const ChunkDesc ch = sdesc[st];
      if (ch.n_rows >= 0 && ch.s != s) {
        // scenario switch: publish the finished scenario's slot, stage the next vector
        if (s >= 0) {
          obj = warp_sum_d(obj);
          if (lane == 0) wobj[cw] = obj;
          obj = 0.0;
          named_sync(1, NCW * 32);
          const int slot = blockIdx.x * P.N + s;
          flush_acc<kScatter>(P, s, acc, partial + (size_t)slot * P.n_pad, ct, NCW * 32);
          if (ct == 0) {
            if (MODE != kNormal) {
              double tsum = 0.0;
              for (int k = 0; k < NCW; ++k) tsum += wobj[k];
              objp[slot] = tsum;
            }
            P.visited[(size_t)s * P.grid + blockIdx.x] = 1;
          }
          named_sync(1, NCW * 32);
        }
        s = ch.s;
        base = P.nnz_base[s];
        stage_vector<kScatter>(P, vin, v_stride, s, sv, acc, ct, NCW * 32);
        named_sync(1, NCW * 32);
      }
      if (ch.n_rows < 0) break;   // end of work (every consumer warp sees it)
      const unsigned char* sp = stage0 + (size_t)st * stage_bytes;
      const int4* rec = reinterpret_cast<const int4*>(sp);
      const VT* val = reinterpret_cast<const VT*>(sp + rec_bytes);
      const IT* col = reinterpret_cast<const IT*>(sp + rec_bytes + val_bytes);
      const long long off = base - ch.g_al;
      const int G = ch.group;                // lanes per row
      const int rpw = 32 / G;                // rows per warp step
      const int sl = lane & (G - 1), sub = lane / G;
      const size_t dose_base = (size_t)s * P.m_act;
      for (int r0 = cw * rpw; r0 < ch.n_rows; r0 += NCW * rpw) {
        const int r = r0 + sub;
        process_rows<MODE, VT, IT, KR>(rec, r, r < ch.n_rows, G, sl, val, col, off, sv, acc, obj,
                                              dose, dose_base);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[st]));
      if (++st == S) {
        st = 0;
        ph ^= 1;
      }
    }
    if (s >= 0) {
      obj = warp_sum_d(obj);
      if (lane == 0) wobj[cw] = obj;
      named_sync(1, NCW * 32);
      const int slot = blockIdx.x * P.N + s;
      flush_acc<kScatter>(P, s, acc, partial + (size_t)slot * P.n_pad, ct, NCW * 32);
      if (ct == 0) {
        if (MODE != kNormal) {
          double tsum = 0.0;
          for (int k = 0; k < NCW; ++k) tsum += wobj[k];
          objp[slot] = tsum;
        }
        P.visited[(size_t)s * P.grid + blockIdx.x] = 1;
      }
    }
  }
  finish_pass<MODE != kNormal>(P);
}

// ---------------------------------------------------------------------------
// register-path row pass
// ---------------------------------------------------------------------------
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

  const int4 blk = P.blocks[blockIdx.x];      // (s, first row, end row, lanes per row)
  const int s = blk.x;
  const bool run = (active == nullptr || active[s] != 0);   // uniform over the CTA
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (run) {
    stage_vector<kScatter>(P, vin, v_stride, s, sv, acc, tid, kRowThreads);
    if (tid == 0) next_row = blk.y;
    __syncthreads();
    const int4* __restrict__ rec = P.rowrec + P.rec_base[s];
    const VT* __restrict__ val = vals<VT>(P) + P.nnz_base[s];
    const IT* __restrict__ col = cols<IT>(P) + P.nnz_base[s];
    const int G = blk.w, rpw = 32 / G;
    const int sl = lane & (G - 1), sub = lane / G;
    const size_t dose_base = (size_t)s * P.m_act;
    double obj = 0.0;
    for (;;) {
      int r0 = 0;
      if (lane == 0) r0 = atomicAdd(&next_row, rpw);
      r0 = __shfl_sync(0xffffffffu, r0, 0);
      if (r0 >= blk.z) break;
      const int r = r0 + sub;
      process_rows<MODE, VT, IT, KR>(rec, r, r < blk.z, G, sl, val, col, 0, sv, acc, obj, dose,
                                            dose_base);
    }
    if (kObjective) {
      obj = warp_sum_d(obj);
      if (lane == 0) wobj[wid] = obj;
    }
    __syncthreads();
    flush_acc<kScatter>(P, s, acc, partial + (size_t)blockIdx.x * P.n_pad, tid, kRowThreads);
    if (kObjective && tid == 0) {
      double t = 0.0;
      for (int k = 0; k < kRowThreads / 32; ++k) t += wobj[k];
      objp[blockIdx.x] = t;
    }
  }
  finish_pass<kObjective>(P);
}

constexpr int kKR = 8;

template <int MODE>
void* pick(const DevPlan& P) {
  if (P.path == 2) return stream_rowpass_kernel(P, MODE);
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
  if (P.path == 2) return stream_smem_bytes(P.n_pad, P.rmax, scatter);
  return (size_t)P.n_pad * sizeof(float) * (scatter ? 2 : 1);
}

int rowpass_threads(const DevPlan& P) {
  return P.path == 1 ? kTmaThreads : (P.path == 2 ? kStrThreads : kRowThreads);
}

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
