// Streaming row pass (path 2): the same fused scenario pass as rowpass.cu
// (acc_s = sum_i c_s w_i a_i (a_i^T v_s [- p_i]), App. A normal equations and
// Eq. 4), organised so that shared memory carries as little as possible.
//
// A persistent CTA per SM holds one scenario's v_s and accumulator in shared
// memory at a time.  Each of its warps is an independent consumer: it claims
// row-aligned chunks of that scenario from the scenario's queue and streams each
// row's entries from global memory straight into registers, one row step ahead
// of the step it computes.  Shared memory then sees only the gather from v_s,
// the scatter into acc and the chunk's row records (copied in with cp.async
// while the previous chunk is processed).  When a chunk is claimed, one chunk
// ahead, its entries are prefetched into L2 (cp.async.bulk.prefetch), so the
// register loads hit L2.  When the scenario's queue is empty the CTA flushes its
// accumulator to the (CTA, scenario) partial slot and moves on to the next
// scenario with work left; the CTA that finishes last publishes the slot lists.
//
// Rows are stored padded with zero entries to a multiple of 4 (16-byte aligned
// starts), so a lane loads 4 consecutive entries ("a quad") with one vector load.
// All rows of a chunk share one length class, which fixes the lanes per row G
// and the quads each lane keeps in registers, Q, at compile time (padded length):
//   class 0: len <= 32  (G 8,  Q 1)       class 3: len <= 256 (G 32, Q 2)
//   class 1: len <= 64  (G 16, Q 1)       class 4: longer     (G 32, Q 4, one
//   class 2: len <= 128 (G 32, Q 1)                buffer; quads past 4 re-read)
// Padding entries (value 0) add nothing to the dot and are skipped by the scatter.
// Nothing here waits on another CTA or on a flag: the only waits are
// cp.async.wait_all (this thread's own copies) and CTA barriers.
#include "rowcommon.cuh"

namespace rpt {
namespace {

constexpr int kStrWarps = kStrThreads / 32;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Hint: fetch [p, p + bytes) into L2 (p 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

struct WChunk {                 // a claimed chunk, uniform over the warp (n_rows < 0: none)
  long long g_al;
  int row_begin, n_rows, n_ent, cls;
};

template <int Q>
struct StepBuf {                // one row step of one lane: Q quads
  float v[Q][4];
  int c[Q][4];
  int nq;                       // quads of the row held by this lane (> Q: rest re-read)
  int lo;                       // first entry of the row (offset in the scenario, multiple of 4)
  float wc, pp;                 // c_s w_i, p_i
  int kept;                     // kept-row index
  bool valid;
};

struct WarpStream {
  const DevPlan* P;
  int sc, c0, c1;
  int4* rs;                     // this warp's two record slots, (rmax + 1) records each
  int slot;                     // slot holding cur's records
  WChunk cur, nx;               // chunk being loaded; next chunk (records in flight to slot ^ 1)
  int q_pend;                   // lane 0: claimed queue position of the chunk after nx (-1: none)
  int lane;
};

__device__ __forceinline__ WChunk load_chunk(const DevPlan& P, int c, int c1) {
  WChunk w;
  if (c < c1) {
    const ChunkDesc ch = P.chunks[c];
    w.g_al = ch.g_al;
    w.row_begin = ch.row_begin;
    w.n_rows = ch.n_rows;
    w.n_ent = ch.n_ent;
    w.cls = ch.pad;
  } else {
    w.g_al = 0;
    w.row_begin = 0;
    w.n_rows = -1;
    w.n_ent = 0;
    w.cls = -1;
  }
  return w;
}

// Start fetching chunk w: its n_rows + 1 records to `dst` (cp.async, 16 bytes a
// lane), its entries into L2 (bulk prefetch of the 16-entry aligned span).
template <typename VT, typename IT>
__device__ __forceinline__ void fetch_chunk(const WarpStream& W, const WChunk& w, int4* dst) {
  if (w.n_rows < 0) return;
  const int4* src = W.P->rowrec + W.P->rec_base[W.sc] + w.row_begin;
  for (int k = W.lane; k <= w.n_rows; k += 32) cp_async16(smem_u32(dst + k), src + k);
  if (W.lane == 0) {
    prefetch_l2(vals<VT>(*W.P) + w.g_al, (uint32_t)w.n_ent * (uint32_t)sizeof(VT));
    prefetch_l2(cols<IT>(*W.P) + w.g_al, (uint32_t)w.n_ent * (uint32_t)sizeof(IT));
  }
}

// Lane 0 takes the next position of the scenario's queue (other lanes: 0).
__device__ __forceinline__ int claim(const WarpStream& W) {
  return W.lane == 0 ? atomicAdd(&W.P->qnext[W.sc], 1) : 0;
}

// Make nx the current chunk; start fetching the chunk after it (claimed one
// chunk ago) and claim the next queue position.
template <typename VT, typename IT>
__device__ __forceinline__ void advance(WarpStream& W) {
  cp_async_wait_all();          // nx's records have landed (this lane's copies) ...
  __syncwarp();                 // ... and every lane's
  W.cur = W.nx;
  W.slot ^= 1;
  const int q = __shfl_sync(0xffffffffu, W.q_pend, 0);
  W.nx = load_chunk(*W.P, q < 0 ? W.c1 : W.c0 + q, W.c1);
  fetch_chunk<VT, IT>(W, W.nx, W.rs + (size_t)(W.slot ^ 1) * (W.P->rmax + 1));
  W.q_pend = W.nx.n_rows >= 0 ? claim(W) : -1;
}

// Load row r of the current chunk (records in `rs`) into b: lane sl of the row's
// group holds quads sl, sl + G, ... (the first Q of them).
template <typename VT, typename IT, int G, int Q>
__device__ __forceinline__ void load_step(StepBuf<Q>& b, const int4* rs, int r, int n_rows, int sl,
                                          const VT* __restrict__ gv, const IT* __restrict__ gc) {
  b.valid = r < n_rows;
  if (b.valid) {
    const int4 ra = rs[r];
    const int hi = rs[r + 1].x;
    b.lo = ra.x;
    b.wc = __int_as_float(ra.y);
    b.pp = __int_as_float(ra.z);
    b.kept = ra.w;
    b.nq = (((hi - ra.x) >> 2) - sl + G - 1) / G;
  } else {
    b.lo = 0;
    b.wc = 0.f;
    b.pp = 0.f;
    b.kept = 0;
    b.nq = 0;
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    if (q < b.nq) {
      const int e = b.lo + 4 * (sl + q * G);
      quad_v<true, VT>(gv + e, b.v[q]);
      quad_c<true, IT>(gc + e, b.c[q]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        b.v[q][k] = 0.f;
        b.c[q][k] = 0;
      }
    }
  }
}

// Dot with v_s, reduce over the row's G lanes, then scatter (or objective/dose).
template <int MODE, typename VT, typename IT, int G, int Q, bool kLong>
__device__ __forceinline__ void compute_step(const StepBuf<Q>& b, int sl, const VT* __restrict__ gv,
                                             const IT* __restrict__ gc, const float* sv, float* acc,
                                             double& obj, float* __restrict__ dose, size_t dose_base) {
  constexpr bool kScatter = (MODE == kNormal || MODE == kResid);
  float t0 = 0.f, t1 = 0.f;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    t0 = fmaf(b.v[q][0], sv[b.c[q][0]], t0);
    t1 = fmaf(b.v[q][1], sv[b.c[q][1]], t1);
    t0 = fmaf(b.v[q][2], sv[b.c[q][2]], t0);
    t1 = fmaf(b.v[q][3], sv[b.c[q][3]], t1);
  }
  if (kLong)
    for (int q = Q; q < b.nq; ++q) {
      float v[4];
      int c[4];
      const int e = b.lo + 4 * (sl + q * G);
      quad_v<true, VT>(gv + e, v);
      quad_c<true, IT>(gc + e, c);
#pragma unroll
      for (int k = 0; k < 4; ++k) t0 = fmaf(v[k], sv[c[k]], t0);
    }
  float t = t0 + t1;
#pragma unroll
  for (int o = G >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  float coef;
  if (MODE == kNormal) {
    coef = b.wc * t;
  } else {
    const float rr = t - b.pp;
    coef = b.wc * rr;
    if (b.valid && sl == 0) {
      obj += (double)(coef * rr);
      if (MODE == kDose) dose[dose_base + b.kept] = t;
    }
  }
  if (kScatter) {
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (b.v[q][k] != 0.f) atomicAdd(&acc[b.c[q][k]], coef * b.v[q][k]);
    if (kLong)
      for (int q = Q; q < b.nq; ++q) {
        float v[4];
        int c[4];
        const int e = b.lo + 4 * (sl + q * G);
        quad_v<true, VT>(gv + e, v);
        quad_c<true, IT>(gc + e, c);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (v[k] != 0.f) atomicAdd(&acc[c[k]], coef * v[k]);
      }
  }
}

// One pipelined step: find the step after the one in `a` (moving on to the next
// chunk when it has the same class), load it into `b`, then compute `a`.
// Returns false when no further step of this class follows.
template <int MODE, typename VT, typename IT, int G, int Q, bool kLong, int CLS>
__device__ __forceinline__ bool stream_step(WarpStream& W, StepBuf<Q>& a, StepBuf<Q>& b, int& r, int sl,
                                           int sub, const VT* gv, const IT* gc, const float* sv, float* acc,
                                           double& obj, float* dose, size_t dose_base) {
  constexpr int rpw = 32 / G;
  int rn = r + rpw;
  bool more = true;
  if (rn >= W.cur.n_rows) {
    if (W.nx.n_rows >= 0 && W.nx.cls == CLS) {
      advance<VT, IT>(W);
      rn = 0;
    } else {
      more = false;
    }
  }
  if (more)
    load_step<VT, IT, G, Q>(b, W.rs + (size_t)W.slot * (W.P->rmax + 1), rn + sub, W.cur.n_rows, sl, gv, gc);
  compute_step<MODE, VT, IT, G, Q, kLong>(a, sl, gv, gc, sv, acc, obj, dose, dose_base);
  r = rn;
  return more;
}

// Process the current chunk and every following chunk of the same class; on
// return the current chunk is the first one of another class (or none).
// kPipe: two register buffers (load one step ahead); otherwise one.
template <int MODE, typename VT, typename IT, int G, int Q, bool kLong, bool kPipe, int CLS>
__device__ __forceinline__ void stream_class(WarpStream& W, const VT* gv, const IT* gc, const float* sv,
                                             float* acc, double& obj, float* dose, size_t dose_base) {
  constexpr int rpw = 32 / G;
  const int sl = W.lane & (G - 1), sub = W.lane / G;
  int r = 0;
  if (kPipe) {
    StepBuf<Q> A, B;
    load_step<VT, IT, G, Q>(A, W.rs + (size_t)W.slot * (W.P->rmax + 1), sub, W.cur.n_rows, sl, gv, gc);
    for (;;) {
      if (!stream_step<MODE, VT, IT, G, Q, kLong, CLS>(W, A, B, r, sl, sub, gv, gc, sv, acc, obj, dose,
                                                         dose_base))
        break;
      if (!stream_step<MODE, VT, IT, G, Q, kLong, CLS>(W, B, A, r, sl, sub, gv, gc, sv, acc, obj, dose,
                                                         dose_base))
        break;
    }
  } else {
    StepBuf<Q> A;
    for (;;) {
      load_step<VT, IT, G, Q>(A, W.rs + (size_t)W.slot * (W.P->rmax + 1), r + sub, W.cur.n_rows, sl, gv, gc);
      compute_step<MODE, VT, IT, G, Q, kLong>(A, sl, gv, gc, sv, acc, obj, dose, dose_base);
      r += rpw;
      if (r >= W.cur.n_rows) {
        if (W.nx.n_rows >= 0 && W.nx.cls == CLS) {
          advance<VT, IT>(W);
          r = 0;
        } else {
          break;
        }
      }
    }
  }
  if (W.nx.n_rows >= 0) advance<VT, IT>(W);
  else W.cur.n_rows = -1;
}

template <int MODE, typename VT, typename IT>
__global__ void __launch_bounds__(kStrThreads, 1)
k_rowpass_stream(DevPlan P, const float* __restrict__ vin, int v_stride, const int* __restrict__ active,
                 float* __restrict__ partial, double* __restrict__ objp, float* __restrict__ dose) {
  constexpr bool kScatter = (MODE == kNormal || MODE == kResid);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double wobj[kStrWarps];
  __shared__ int s_go, s_did;
  float* sv = reinterpret_cast<float*>(smem);
  float* acc = sv + P.n_pad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int4* recs = reinterpret_cast<int4*>(smem + round128((size_t)P.n_pad * 4 * (kScatter ? 2 : 1)));

  WarpStream W;
  W.P = &P;
  W.lane = lane;
  W.rs = recs + (size_t)warp * 2 * (P.rmax + 1);
  const int home = (int)(((long long)blockIdx.x * P.N) / gridDim.x);
  for (int k = 0; k < P.N; ++k) {
    const int sc = (home + k) % P.N;
    if (active != nullptr && active[sc] == 0) continue;
    const int c0 = P.scen_chunk[sc], c1 = P.scen_chunk[sc + 1];
    if (tid == 0) {
      s_go = *reinterpret_cast<volatile int*>(&P.qnext[sc]) < c1 - c0;
      s_did = 0;
    }
    __syncthreads();
    const bool go = s_go;
    __syncthreads();
    if (!go) continue;
    stage_vector<kScatter>(P, vin, v_stride, sc, sv, acc, tid, kStrThreads);
    __syncthreads();

    // this warp's first two chunks
    W.sc = sc;
    W.c0 = c0;
    W.c1 = c1;
    W.slot = 0;
    int q = __shfl_sync(0xffffffffu, claim(W), 0);
    W.cur = load_chunk(P, c0 + q, c1);
    double obj = 0.0;
    if (W.cur.n_rows >= 0) {
      if (lane == 0) s_did = 1;
      fetch_chunk<VT, IT>(W, W.cur, W.rs);
      q = __shfl_sync(0xffffffffu, claim(W), 0);
      W.nx = load_chunk(P, c0 + q, c1);
      fetch_chunk<VT, IT>(W, W.nx, W.rs + (P.rmax + 1));
      W.q_pend = W.nx.n_rows >= 0 ? claim(W) : -1;
      cp_async_wait_all();
      __syncwarp();
      const VT* gv = vals<VT>(P) + P.nnz_base[sc];
      const IT* gc = cols<IT>(P) + P.nnz_base[sc];
      const size_t dose_base = (size_t)sc * P.m_act;
      while (W.cur.n_rows >= 0) {
        switch (W.cur.cls) {
          case 0: stream_class<MODE, VT, IT, 8, 1, false, true, 0>(W, gv, gc, sv, acc, obj, dose, dose_base); break;
          case 1: stream_class<MODE, VT, IT, 16, 1, false, true, 1>(W, gv, gc, sv, acc, obj, dose, dose_base); break;
          case 2: stream_class<MODE, VT, IT, 32, 1, false, true, 2>(W, gv, gc, sv, acc, obj, dose, dose_base); break;
          case 3: stream_class<MODE, VT, IT, 32, 2, false, true, 3>(W, gv, gc, sv, acc, obj, dose, dose_base); break;
          default: stream_class<MODE, VT, IT, 32, 4, true, false, 4>(W, gv, gc, sv, acc, obj, dose, dose_base); break;
        }
      }
    }
    obj = warp_sum_d(obj);
    if (lane == 0) wobj[warp] = obj;
    __syncthreads();
    if (s_did) {
      const int slot = blockIdx.x * P.N + sc;
      flush_acc<kScatter>(P, sc, acc, partial + (size_t)slot * P.n_pad, tid, kStrThreads);
      if (tid == 0) {
        if (MODE != kNormal) {
          double tsum = 0.0;
          for (int w = 0; w < kStrWarps; ++w) tsum += wobj[w];
          objp[slot] = tsum;
        }
        P.visited[(size_t)sc * P.grid + blockIdx.x] = 1;
      }
    }
    __syncthreads();
  }
  finish_pass<MODE != kNormal>(P);
}

template <int MODE>
void* pick(const DevPlan& P) {
  if (P.index_width == 16) {
    switch (P.value_format) {
      case 1: return (void*)k_rowpass_stream<MODE, __nv_bfloat16, uint16_t>;
      case 2: return (void*)k_rowpass_stream<MODE, __nv_fp8_e4m3, uint16_t>;
      default: return (void*)k_rowpass_stream<MODE, float, uint16_t>;
    }
  }
  switch (P.value_format) {
    case 1: return (void*)k_rowpass_stream<MODE, __nv_bfloat16, int32_t>;
    case 2: return (void*)k_rowpass_stream<MODE, __nv_fp8_e4m3, int32_t>;
    default: return (void*)k_rowpass_stream<MODE, float, int32_t>;
  }
}

}  // namespace

void* stream_rowpass_kernel(const DevPlan& P, int mode) {
  switch (mode) {
    case kNormal: return pick<kNormal>(P);
    case kResid: return pick<kResid>(P);
    case kObj: return pick<kObj>(P);
    default: return pick<kDose>(P);
  }
}

size_t stream_smem_bytes(int n_pad, int rmax, bool scatter) {
  return round128((size_t)n_pad * 4 * (scatter ? 2 : 1)) + (size_t)kStrWarps * 2 * (rmax + 1) * 16;
}

}  // namespace rpt
