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
// Implementations of the same pass:
//  * k_rowpass_tma<..., BUN = true> (bundled ring, the default where it pays):
//    the ring below over row bundles (4 rows sharing one index per block column)
//    with an exact 64-bit fixed-point accumulator, see process_bundle.
//  * k_rowpass_tma (ring): a persistent CTA per SM streams its slice of the
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
// try_wait with a suspend-time hint: a waiting thread sleeps until the phase
// completes or about 0.1 ms pass, instead of spinning and taking issue slots
// from the warps that work.
constexpr uint32_t kSuspendHintNs = 100000;
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendHintNs)
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

// Round y (a float32 of magnitude below 2^62) to the nearest integer, halves away
// from zero, with integer operations on its bits: y = m 2^e with m the 24-bit
// significand, so the result is m << e, or (m + 2^(-e-1)) >> -e when e < 0.  (A
// float-to-64-bit-integer conversion instruction runs on the FP64 pipe, which is
// narrow on this GPU.)  Zero and subnormal inputs give 0.
__device__ __forceinline__ long long fixed_round(float y) {
  const unsigned b = __float_as_uint(y);
  const int e = (int)((b >> 23) & 0xffu) - 150;
  if (e < -24) return 0;                              // |y| < 0.5
  const long long m = (long long)((b & 0x7fffffu) | 0x800000u);
  const long long q = e >= 0 ? (m << e) : ((m + (1ll << (-e - 1))) >> (-e));
  return (b >> 31) ? -q : q;
}

// One group of G lanes (G in {8, 16, 32}) processes one row bundle (layout.h):
// lane sl takes block columns sl, sl + G, ...; each block column holds the
// values of the bundle's 4 rows at one spot column.  Dot products t_r of the 4
// rows in float32 (fixed order), reduced over the G lanes by a transposing
// butterfly: after it, lane sl holds the whole sum of row rho = sl / (G/4).  The
// scatter adds sum_r coef_r a_{r,c} per block column to the 64-bit fixed-point
// accumulator (scale fscale = 2^F): integer sums are exact, so the result does
// not depend on the order of the atomics.  Block columns whose four values are
// zero (none are stored) or whose scaled contribution rounds to 0 add nothing.
template <int MODE, typename VT, typename IT, int KR, bool FIX>
__device__ __forceinline__ void process_bundle(const int4* __restrict__ rec, int b, bool valid, int G, int sl,
                                               const VT* __restrict__ val, const IT* __restrict__ col,
                                               long long off, const float* sv, float* accf,
                                               float fscale, double& obj, float* __restrict__ dose,
                                               size_t dose_base) {
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(accf);
  constexpr bool kScatter = (MODE == kNormal || MODE == kResid);
  constexpr unsigned kFull = 0xffffffffu;
  int lo = 0, hi = 0;
  if (valid) {
    lo = (int)(rec[4 * b].x + off);
    hi = (int)(rec[4 * b + 4].x + off);
  }
  float a[KR][4];
  int c[KR];
  float t[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const int idx = lo + sl + G * k;
    if (idx < hi) {
      quad_v<false, VT>(val + 4 * (size_t)idx, a[k]);
      c[k] = (int)col[idx];
      const float v = sv[c[k]];
#pragma unroll
      for (int r = 0; r < 4; ++r) t[r] = fmaf(a[k][r], v, t[r]);
    } else {
#pragma unroll
      for (int r = 0; r < 4; ++r) a[k][r] = 0.f;
      c[k] = 0;
    }
  }
  for (int idx = lo + G * KR + sl; idx < hi; idx += G) {
    float q[4];
    quad_v<false, VT>(val + 4 * (size_t)idx, q);
    const float v = sv[(int)col[idx]];
#pragma unroll
    for (int r = 0; r < 4; ++r) t[r] = fmaf(q[r], v, t[r]);
  }
  // transposing butterfly: halves exchange rows {0,1} / {2,3}, quarters one row
  const int h = G >> 1, qd = G >> 2;
  const bool up = (sl & h) != 0, up2 = (sl & qd) != 0;
  const float k0 = up ? t[2] : t[0], k1 = up ? t[3] : t[1];
  const float g0 = up ? t[0] : t[2], g1 = up ? t[1] : t[3];
  const float u0 = k0 + __shfl_xor_sync(kFull, g0, h);
  const float u1 = k1 + __shfl_xor_sync(kFull, g1, h);
  float tw = (up2 ? u1 : u0) + __shfl_xor_sync(kFull, up2 ? u0 : u1, qd);
  for (int o = qd >> 1; o > 0; o >>= 1) tw += __shfl_xor_sync(kFull, tw, o);
  const int rho = sl >> (__ffs(qd) - 1);         // the row whose whole dot this lane holds (qd a power of 2)
  float wc = 0.f, pr = 0.f;
  int kept = -1;
  if (valid) {
    wc = __int_as_float(reinterpret_cast<const int*>(&rec[4 * b + 1])[rho]);
    pr = __int_as_float(reinterpret_cast<const int*>(&rec[4 * b + 2])[rho]);
    kept = reinterpret_cast<const int*>(&rec[4 * b + 3])[rho];
  }
  float own;
  if (MODE == kNormal) {
    own = wc * tw;
  } else {
    const float rr = tw - pr;
    own = wc * rr;
    if (valid && (sl & (qd - 1)) == 0) {
      obj += (double)(own * rr);
      if (MODE == kDose && kept >= 0) dose[dose_base + kept] = tw;
    }
  }
  if (kScatter) {
    const int g0l = (threadIdx.x & 31) - sl;     // first lane of the group
    float coef[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) coef[r] = __shfl_sync(kFull, own, g0l + r * qd);
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const float sc = coef[0] * a[k][0] + coef[1] * a[k][1] + coef[2] * a[k][2] + coef[3] * a[k][3];
      if (FIX) {
        const long long qv = fixed_round(sc * fscale);
        if (qv != 0) atomicAdd(&acc[c[k]], (unsigned long long)qv);
      } else if (sc != 0.f) {
        atomicAdd(&accf[c[k]], sc);
      }
    }
    for (int idx = lo + G * KR + sl; idx < hi; idx += G) {
      float q[4];
      quad_v<false, VT>(val + 4 * (size_t)idx, q);
      const float sc = coef[0] * q[0] + coef[1] * q[1] + coef[2] * q[2] + coef[3] * q[3];
      if (FIX) {
        const long long qv = fixed_round(sc * fscale);
        if (qv != 0) atomicAdd(&acc[(int)col[idx]], (unsigned long long)qv);
      } else if (sc != 0.f) {
        atomicAdd(&accf[(int)col[idx]], sc);
      }
    }
  }
}

// Scale exponent F of the fixed-point accumulation: 2^F * bound <= 2^60, so
// that no sum of up to 2^2 times the bound (float32 rounding of the products
// included) can overflow 63 bits; kFexpNaN marks a non-finite vector.
__device__ __forceinline__ int fixed_exp(float vmax, double k, double pterm) {
  if (!isfinite(vmax)) return kFexpNaN;
  const double bound = k * (double)vmax + pterm;
  if (!(bound > 0.0)) return 0;
  int e;
  frexp(bound, &e);                              // bound < 2^e
  return max(-126, min(126, 60 - e));
}

// ---------------------------------------------------------------------------
// TMA-ring row pass
// ---------------------------------------------------------------------------
constexpr int kHdr = 1024;  // mbarriers (2 x 8 x 8 B), chunk descriptors (8 x 32 B), per-warp objective (up to 64 doubles)
constexpr int kBatch = 4;   // chunks per queue pull

// BUN = false: rows of the CSR layout (path 1), float accumulator.  BUN = true:
// row bundles (path 3), records of 4 int4 per bundle, 4 values per block column,
// 64-bit fixed-point accumulator (see process_bundle); the staged vector's
// maximum magnitude sets the scale of each scenario.
// NT threads per CTA (one producer warp, NT / 32 - 1 consumer warps); the
// bundled path trades warps for registers: 1024 threads keep 6 block columns
// per lane in registers, 768 keep 8 and 640 keep 10 (so fewer block columns of
// wide bundles are read twice).
template <int MODE, typename VT, typename IT, bool BUN, bool FIX, int NT = kTmaThreads>
__global__ void __launch_bounds__(NT, 1)
k_rowpass_tma(DevPlan P, const float* __restrict__ vin, int v_stride, const int* __restrict__ active,
              float* __restrict__ partial, double* __restrict__ objp, float* __restrict__ dose) {
  constexpr bool kScatter = (MODE == kNormal || MODE == kResid);
  constexpr int NCW = NT / 32 - 1;              // consumer warps (wobj below holds up to 64)
  constexpr int KR = BUN ? (NT >= 1024 ? kBundleKeep : (NT >= 768 ? 8 : 10)) : 8;   // block columns (entries)
                                                // per lane kept in registers
  constexpr int RPU = BUN ? 4 : 1;              // int4 records per row (bundle)
  constexpr int VPE = BUN ? 4 : 1;              // values per stored entry (block column)
  constexpr bool FX = BUN && FIX;                // 64-bit fixed-point accumulator
  constexpr int ACCB = FX ? 8 : 4;              // accumulator bytes per column
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + 8;
  ChunkDesc* sdesc = reinterpret_cast<ChunkDesc*>(smem + 128);   // one per stage
  double* wobj = reinterpret_cast<double*>(smem + 512);
  float* wmax = reinterpret_cast<float*>(smem + 512 + 8 * NCW);  // per-warp max |v| (bundled path)
  float* sv = reinterpret_cast<float*>(smem + kHdr);
  float* acc = sv + P.n_pad;
  unsigned long long* acc64 = reinterpret_cast<unsigned long long*>(acc);
  const int S = P.stages;
  const size_t rec_bytes = round128((size_t)(P.rmax * RPU + 1) * 16);
  const size_t val_bytes = round128((size_t)P.cmax * VPE * sizeof(VT));
  const size_t col_bytes = round128((size_t)P.cmax * sizeof(IT));
  const size_t stage_bytes = rec_bytes + val_bytes + col_bytes;
  unsigned char* stage0 = smem + round128(kHdr + (size_t)P.n_pad * (4 + (kScatter ? ACCB : 0)));

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
          const uint32_t rb = (uint32_t)(ch.n_rows * RPU + 1) * 16u;
          const uint32_t vb = (uint32_t)ch.n_ent * (uint32_t)(VPE * sizeof(VT));
          const uint32_t cb = (uint32_t)ch.n_ent * (uint32_t)sizeof(IT);
          const int4* rec = P.rowrec + P.rec_base[sc];
          sdesc[st] = ch;
          const uint32_t fb = smem_u32(&full[st]);
          mbar_arrive_expect_tx(fb, rb + vb + cb);
          bulk_g2s(smem_u32(sp), rec + (size_t)ch.row_begin * RPU, rb, fb);
          bulk_g2s(smem_u32(sp + rec_bytes), gval + ch.g_al * VPE, vb, fb);
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
    float fscale = 0.f;         // bundled path: 2^F of the staged scenario
    int fexp = 0;
    // work units (one row or bundle group of a warp) are dealt round-robin over the
    // consumer warps across consecutive chunks: a chunk with fewer units than
    // warps leaves the rest free for the next chunk instead of idle.  Every warp
    // sees the same chunk sequence, so all agree on the rotation.
    int rot = 0;
    auto publish = [&]() {
      obj = warp_sum_d(obj);
      if (lane == 0) wobj[cw] = obj;
      obj = 0.0;
      named_sync(1, NCW * 32);
      const int slot = blockIdx.x * P.N + s;
      if (FX) {
        if (kScatter) {
          unsigned long long* out = reinterpret_cast<unsigned long long*>(partial) + (size_t)slot * P.n_pad;
          for (int k = ct; k < P.n_pad; k += NCW * 32) out[k] = acc64[k];
        }
      } else {
        flush_acc<kScatter>(P, s, acc, partial + (size_t)slot * P.n_pad, ct, NCW * 32);
      }
      if (ct == 0) {
        if (MODE != kNormal) {
          double tsum = 0.0;
          for (int k = 0; k < NCW; ++k) tsum += wobj[k];
          objp[slot] = tsum;
        }
        if (FX && kScatter) P.fexp[s] = fexp;
        P.visited[(size_t)s * P.grid + blockIdx.x] = 1;
      }
    };
    for (;;) {
      if (!mbar_wait(smem_u32(&full[st]), (uint32_t)ph)) {
        if (lane == 0) atomicExch(P.err, 3);
        break;
      }
      const ChunkDesc ch = sdesc[st];
      if (ch.n_rows >= 0 && ch.s != s) {
        // scenario switch: publish the finished scenario's slot, stage the next vector
        if (s >= 0) {
          publish();
          named_sync(1, NCW * 32);
        }
        s = ch.s;
        base = P.nnz_base[s];
        if (FX) {
          float vm = stage_vector_max<kScatter>(P, vin, v_stride, s, sv, acc64, ct, NCW * 32);
          vm = warp_max(vm);
          if (lane == 0) wmax[cw] = vm;
          named_sync(1, NCW * 32);
          float vmax = 0.f;   // +inf if the vector is not finite
          for (int k = 0; k < NCW; ++k) vmax = fmaxf(vmax, wmax[k]);
          fexp = kScatter ? fixed_exp(vmax, P.kbound[2 * s], MODE == kResid ? P.kbound[2 * s + 1] : 0.0) : 0;
          fscale = (fexp == kFexpNaN) ? 0.f : __int_as_float((fexp + 127) << 23);
        } else {
          stage_vector<kScatter>(P, vin, v_stride, s, sv, acc, ct, NCW * 32);
          named_sync(1, NCW * 32);
        }
      }
      if (ch.n_rows < 0) break;   // end of work (every consumer warp sees it)
      const unsigned char* sp = stage0 + (size_t)st * stage_bytes;
      const int4* rec = reinterpret_cast<const int4*>(sp);
      const VT* val = reinterpret_cast<const VT*>(sp + rec_bytes);
      const IT* col = reinterpret_cast<const IT*>(sp + rec_bytes + val_bytes);
      const long long off = base - ch.g_al;
      const int G = ch.group;                // lanes per row (bundle)
      const int lg = __ffs(G) - 1;           // G is a power of two: shifts, not divisions
      const int rpw = 32 >> lg;              // rows (bundles) per warp step
      const int sl = lane & (G - 1), sub = lane >> lg;
      const size_t dose_base = (size_t)s * P.m_act;
      const int units = (ch.n_rows + rpw - 1) >> (5 - lg);
      int u0 = cw - rot;
      if (u0 < 0) u0 += NCW;
      rot = (rot + units) % NCW;
      for (int u = u0; u < units; u += NCW) {
        const int r = u * rpw + sub;
        if (BUN)
          process_bundle<MODE, VT, IT, KR, FIX>(rec, r, r < ch.n_rows, G, sl, val, col, off, sv, acc, fscale,
                                                obj, dose, dose_base);
        else
          process_rows<MODE, VT, IT, KR>(rec, r, r < ch.n_rows, G, sl, val, col, off, sv, acc, obj, dose,
                                         dose_base);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty[st]));
      if (++st == S) {
        st = 0;
        ph ^= 1;
      }
    }
    if (s >= 0) publish();
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
    const int G = blk.w, lg = __ffs(G) - 1, rpw = 32 >> lg;   // G a power of two
    const int sl = lane & (G - 1), sub = lane >> lg;
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

template <int MODE, bool BUN, bool FIX, int NT = kTmaThreads>
void* pick_ring(const DevPlan& P) {
  if (P.index_width == 16) {
    switch (P.value_format) {
      case 1: return (void*)k_rowpass_tma<MODE, __nv_bfloat16, uint16_t, BUN, FIX, NT>;
      case 2: return (void*)k_rowpass_tma<MODE, __nv_fp8_e4m3, uint16_t, BUN, FIX, NT>;
      default: return (void*)k_rowpass_tma<MODE, float, uint16_t, BUN, FIX, NT>;
    }
  }
  switch (P.value_format) {
    case 1: return (void*)k_rowpass_tma<MODE, __nv_bfloat16, int32_t, BUN, FIX, NT>;
    case 2: return (void*)k_rowpass_tma<MODE, __nv_fp8_e4m3, int32_t, BUN, FIX, NT>;
    default: return (void*)k_rowpass_tma<MODE, float, int32_t, BUN, FIX, NT>;
  }
}

template <int MODE, bool FIX>
void* pick_bundled(const DevPlan& P) {
  if (P.ring_threads == 768) return pick_ring<MODE, true, FIX, 768>(P);
  if (P.ring_threads == 640) return pick_ring<MODE, true, FIX, 640>(P);
  return pick_ring<MODE, true, FIX, kTmaThreads>(P);
}

template <int MODE>
void* pick(const DevPlan& P) {
  if (P.path == 3) return P.acc64 ? pick_bundled<MODE, true>(P) : pick_bundled<MODE, false>(P);
  if (P.path == 2) return stream_rowpass_kernel(P, MODE);
  if (P.path == 1) return pick_ring<MODE, false, false>(P);
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

namespace {

// Bounds of the fixed-point accumulation (bundled layout), one warp per bundle of
// scenario s, on the stored values q (codes of quantised formats):
//   Kc[c] += sum_r c_s w_r |q_rc| ||q_r||_1,   Pc[c] += sum_r c_s w_r |q_rc| p_r
// so that |acc_c| <= Kc[c] max|v_s| (+ Pc[c] with the prescription term).
template <typename VT, typename IT>
__global__ void k_bun_bound(DevPlan P, int s, double* __restrict__ Kc, double* __restrict__ Pc) {
  const int lane = threadIdx.x & 31;
  const int4* rec = P.rowrec + P.rec_base[s];
  const int nb = (P.rec_base[s + 1] - P.rec_base[s]) / 4 - 1;
  const VT* val = vals<VT>(P) + 4 * P.nnz_base[s];
  const IT* col = cols<IT>(P) + P.nnz_base[s];
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += nw) {
    const int lo = rec[4 * b].x, hi = rec[4 * b + 4].x;
    float wc[4], pr[4];
    for (int r = 0; r < 4; ++r) {
      wc[r] = __int_as_float(reinterpret_cast<const int*>(&rec[4 * b + 1])[r]);
      pr[r] = __int_as_float(reinterpret_cast<const int*>(&rec[4 * b + 2])[r]);
    }
    double l1[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = lo + lane; k < hi; k += 32) {
      float q[4];
      quad_v<true, VT>(val + 4 * (size_t)k, q);
      for (int r = 0; r < 4; ++r) l1[r] += fabs((double)q[r]);
    }
    for (int r = 0; r < 4; ++r) l1[r] = warp_sum_d(l1[r]);
    for (int k = lo + lane; k < hi; k += 32) {
      float q[4];
      quad_v<true, VT>(val + 4 * (size_t)k, q);
      double kc = 0.0, pc = 0.0;
      for (int r = 0; r < 4; ++r) {
        const double aw = (double)wc[r] * fabs((double)q[r]);
        kc += aw * l1[r];
        pc += aw * (double)pr[r];
      }
      const int c = (int)col[k];
      if (kc != 0.0) atomicAdd(&Kc[c], kc);
      if (pc != 0.0) atomicAdd(&Pc[c], pc);
    }
  }
}

// out[0] = max Kc, out[1] = max Pc (one block).
__global__ void k_bound_max(const double* __restrict__ Kc, const double* __restrict__ Pc, int n, double* out) {
  __shared__ double sk[32], sp[32];
  double mk = 0.0, mp = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    mk = fmax(mk, Kc[j]);
    mp = fmax(mp, Pc[j]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mk = fmax(mk, __shfl_xor_sync(0xffffffffu, mk, o));
    mp = fmax(mp, __shfl_xor_sync(0xffffffffu, mp, o));
  }
  if ((threadIdx.x & 31) == 0) {
    sk[threadIdx.x >> 5] = mk;
    sp[threadIdx.x >> 5] = mp;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mk = fmax(mk, sk[w]);
      mp = fmax(mp, sp[w]);
    }
    out[0] = mk;
    out[1] = mp;
  }
}

template <typename VT, typename IT>
cudaError_t bundle_bounds_t(const DevPlan& P, double* kc, double* pc, double* kbound, cudaStream_t st) {
  for (int s = 0; s < P.N; ++s) {
    cudaError_t e = cudaMemsetAsync(kc, 0, sizeof(double) * P.n_pad, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(pc, 0, sizeof(double) * P.n_pad, st);
    if (e != cudaSuccess) return e;
    k_bun_bound<VT, IT><<<P.grid, 256, 0, st>>>(P, s, kc, pc);
    k_bound_max<<<1, 1024, 0, st>>>(kc, pc, P.n, kbound + 2 * s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---- reweighting (rpt_plan_set_weights) ------------------------------------
// Row records of scenario s for new weights: c_s w_k and p_k of every listed row
// (kept index k), as float32 bits like plan creation writes them.
__global__ void k_reweight_rows(DevPlan P, int s, double cs, const double* __restrict__ wk,
                                const double* __restrict__ pk) {
  int4* rec = const_cast<int4*>(P.rowrec) + P.rec_base[s];
  const int span = P.rec_base[s + 1] - P.rec_base[s];
  const int stride = gridDim.x * blockDim.x;
  if (P.path == 3) {
    const int nb = span / 4 - 1;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += stride)
      for (int r = 0; r < 4; ++r) {
        const int k = reinterpret_cast<const int*>(&rec[4 * b + 3])[r];
        if (k < 0) continue;
        reinterpret_cast<int*>(&rec[4 * b + 1])[r] = __float_as_int((float)(cs * wk[k]));
        reinterpret_cast<int*>(&rec[4 * b + 2])[r] = __float_as_int((float)pk[k]);
      }
  } else {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < span - 1; q += stride) {
      const int k = rec[q].w;
      rec[q].y = __float_as_int((float)(cs * wk[k]));
      rec[q].z = __float_as_int((float)pk[k]);
    }
  }
}

// Jacobi diagonal of scenario s, sum_i c_s w_i a_ij^2, as exact 64-bit fixed-point
// sums (scale 2^F given by the caller from a bound), one warp per row or bundle;
// a = the stored value (dequantised).
template <typename VT, typename IT>
__global__ void k_reweight_diag(DevPlan P, int s, double cs, const double* __restrict__ wk, double scale,
                                unsigned long long* __restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const int4* rec = P.rowrec + P.rec_base[s];
  const int span = P.rec_base[s + 1] - P.rec_base[s];
  const long long base = P.nnz_base[s];
  const float* csc = P.colscale ? P.colscale + (size_t)s * P.n_pad : nullptr;
  const int nw = gridDim.x * (blockDim.x >> 5);
  const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (P.path == 3) {
    const VT* val = vals<VT>(P) + 4 * base;
    const IT* col = cols<IT>(P) + base;
    for (int b = wid; b < span / 4 - 1; b += nw) {
      double wd[4];
      for (int r = 0; r < 4; ++r) {
        const int k = reinterpret_cast<const int*>(&rec[4 * b + 3])[r];
        wd[r] = k >= 0 ? cs * wk[k] : 0.0;
      }
      for (int e = rec[4 * b].x + lane; e < rec[4 * b + 4].x; e += 32) {
        float q[4];
        quad_v<true, VT>(val + 4 * (size_t)e, q);
        const int c = (int)col[e];
        const double sc = csc ? (double)csc[c] : 1.0;
        double v = 0.0;
        for (int r = 0; r < 4; ++r) v += wd[r] * ((double)q[r] * sc) * ((double)q[r] * sc);
        const long long iv = __double2ll_rn(v * scale);
        if (iv) atomicAdd(&acc[c], (unsigned long long)iv);
      }
    }
  } else {
    const VT* val = vals<VT>(P) + base;
    const IT* col = cols<IT>(P) + base;
    for (int q = wid; q < span - 1; q += nw) {
      const double wd = cs * wk[rec[q].w];
      for (int e = rec[q].x + lane; e < rec[q + 1].x; e += 32) {
        const int c = (int)col[e];
        const double a = (double)to_f<VT>(val[e]) * (csc ? (double)csc[c] : 1.0);
        const long long iv = __double2ll_rn(wd * a * a * scale);
        if (iv) atomicAdd(&acc[c], (unsigned long long)iv);
      }
    }
  }
}

template <typename VT, typename IT>
cudaError_t reweight_t(const DevPlan& P, int s, double cs, const double* wk, const double* pk, double scale,
                       unsigned long long* acc, cudaStream_t st) {
  k_reweight_rows<<<P.grid, 256, 0, st>>>(P, s, cs, wk, pk);
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * P.n_pad, st);
  if (e != cudaSuccess) return e;
  k_reweight_diag<VT, IT><<<P.grid, 256, 0, st>>>(P, s, cs, wk, scale, acc);
  return cudaGetLastError();
}

}  // namespace

cudaError_t plan_reweight(const DevPlan& P, int s, double cs, const double* wk, const double* pk, double scale,
                          unsigned long long* acc, cudaStream_t st) {
  if (P.index_width == 16) {
    switch (P.value_format) {
      case 1: return reweight_t<__nv_bfloat16, uint16_t>(P, s, cs, wk, pk, scale, acc, st);
      case 2: return reweight_t<__nv_fp8_e4m3, uint16_t>(P, s, cs, wk, pk, scale, acc, st);
      default: return reweight_t<float, uint16_t>(P, s, cs, wk, pk, scale, acc, st);
    }
  }
  switch (P.value_format) {
    case 1: return reweight_t<__nv_bfloat16, int32_t>(P, s, cs, wk, pk, scale, acc, st);
    case 2: return reweight_t<__nv_fp8_e4m3, int32_t>(P, s, cs, wk, pk, scale, acc, st);
    default: return reweight_t<float, int32_t>(P, s, cs, wk, pk, scale, acc, st);
  }
}

cudaError_t bundle_bounds(const DevPlan& P, double* kc, double* pc, double* kbound, cudaStream_t st) {
  if (P.index_width == 16) {
    switch (P.value_format) {
      case 1: return bundle_bounds_t<__nv_bfloat16, uint16_t>(P, kc, pc, kbound, st);
      case 2: return bundle_bounds_t<__nv_fp8_e4m3, uint16_t>(P, kc, pc, kbound, st);
      default: return bundle_bounds_t<float, uint16_t>(P, kc, pc, kbound, st);
    }
  }
  switch (P.value_format) {
    case 1: return bundle_bounds_t<__nv_bfloat16, int32_t>(P, kc, pc, kbound, st);
    case 2: return bundle_bounds_t<__nv_fp8_e4m3, int32_t>(P, kc, pc, kbound, st);
    default: return bundle_bounds_t<float, int32_t>(P, kc, pc, kbound, st);
  }
}

size_t tma_smem_bytes(int n_pad, int cmax, int rmax, int stages, int value_bytes, int index_bytes,
                      bool scatter, bool bundled, bool fixed) {
  const int rpu = bundled ? 4 : 1, vpe = bundled ? 4 : 1, accb = (bundled && fixed) ? 8 : 4;
  const size_t stage = round128((size_t)(rmax * rpu + 1) * 16) + round128((size_t)cmax * vpe * value_bytes) +
                       round128((size_t)cmax * index_bytes);
  return round128(kHdr + (size_t)n_pad * (4 + (scatter ? accb : 0))) + (size_t)stages * stage;
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
  if (P.path == 1 || P.path == 3) {
    const int vb = P.value_format == 0 ? 4 : (P.value_format == 1 ? 2 : 1);
    const int ib = P.index_width == 16 ? 2 : 4;
    return tma_smem_bytes(P.n_pad, P.cmax, P.rmax, P.stages, vb, ib, scatter, P.path == 3, P.acc64 != 0);
  }
  if (P.path == 2) return stream_smem_bytes(P.n_pad, P.rmax, scatter);
  return (size_t)P.n_pad * sizeof(float) * (scatter ? 2 : 1);
}

int rowpass_threads(const DevPlan& P) {
  if (P.path == 3) return (P.ring_threads == 768 || P.ring_threads == 640) ? P.ring_threads : kTmaThreads;
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
