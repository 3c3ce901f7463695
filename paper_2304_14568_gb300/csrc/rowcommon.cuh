// Device helpers shared by the row-pass translation units (rowpass.cu: ring and
// register paths; rowstream.cu: streaming path).
#pragma once
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

// ---- 4 consecutive entries ("a quad") of the padded layout ------------------
// Every stored row starts on a multiple of 4 entries, so a quad is one aligned
// vector load: 16 bytes of float or int32, 8 of bf16 or uint16, 4 of fp8.
// kG: read-only global load (ld.global.nc); otherwise a plain load (shared memory).
template <bool kG, typename T>
__device__ __forceinline__ T ldv(const T* p) {
  if constexpr (kG) return __ldg(p);
  else return *p;
}
template <bool kG, typename VT> __device__ __forceinline__ void quad_v(const VT* p, float (&o)[4]);
template <bool kG, typename IT> __device__ __forceinline__ void quad_c(const IT* p, int (&o)[4]);
template <> __device__ __forceinline__ void quad_v<true, float>(const float* p, float (&o)[4]) {
  const float4 x = ldv<true>(reinterpret_cast<const float4*>(p));
  o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
}
template <> __device__ __forceinline__ void quad_v<false, float>(const float* p, float (&o)[4]) {
  const float4 x = ldv<false>(reinterpret_cast<const float4*>(p));
  o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
}
template <bool kG>
__device__ __forceinline__ void quad_bf16(const __nv_bfloat16* p, float (&o)[4]) {
  const uint2 x = ldv<kG>(reinterpret_cast<const uint2*>(p));   // bf16 -> f32 is exact: the high half
  o[0] = __uint_as_float(x.x << 16); o[1] = __uint_as_float(x.x & 0xffff0000u);
  o[2] = __uint_as_float(x.y << 16); o[3] = __uint_as_float(x.y & 0xffff0000u);
}
template <> __device__ __forceinline__ void quad_v<true, __nv_bfloat16>(const __nv_bfloat16* p, float (&o)[4]) {
  quad_bf16<true>(p, o);
}
template <> __device__ __forceinline__ void quad_v<false, __nv_bfloat16>(const __nv_bfloat16* p, float (&o)[4]) {
  quad_bf16<false>(p, o);
}
template <bool kG>
__device__ __forceinline__ void quad_fp8(const __nv_fp8_e4m3* p, float (&o)[4]) {
  const unsigned x = ldv<kG>(reinterpret_cast<const unsigned*>(p));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __nv_fp8_e4m3 q;
    q.__x = (__nv_fp8_storage_t)((x >> (8 * k)) & 0xffu);
    o[k] = float(q);
  }
}
template <> __device__ __forceinline__ void quad_v<true, __nv_fp8_e4m3>(const __nv_fp8_e4m3* p, float (&o)[4]) {
  quad_fp8<true>(p, o);
}
template <> __device__ __forceinline__ void quad_v<false, __nv_fp8_e4m3>(const __nv_fp8_e4m3* p, float (&o)[4]) {
  quad_fp8<false>(p, o);
}
template <bool kG>
__device__ __forceinline__ void quad_i32(const int32_t* p, int (&o)[4]) {
  const int4 x = ldv<kG>(reinterpret_cast<const int4*>(p));
  o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
}
template <bool kG>
__device__ __forceinline__ void quad_u16(const uint16_t* p, int (&o)[4]) {
  const uint2 x = ldv<kG>(reinterpret_cast<const uint2*>(p));
  o[0] = (int)(x.x & 0xffffu); o[1] = (int)(x.x >> 16); o[2] = (int)(x.y & 0xffffu); o[3] = (int)(x.y >> 16);
}
template <> __device__ __forceinline__ void quad_c<true, int32_t>(const int32_t* p, int (&o)[4]) { quad_i32<true>(p, o); }
template <> __device__ __forceinline__ void quad_c<false, int32_t>(const int32_t* p, int (&o)[4]) { quad_i32<false>(p, o); }
template <> __device__ __forceinline__ void quad_c<true, uint16_t>(const uint16_t* p, int (&o)[4]) { quad_u16<true>(p, o); }
template <> __device__ __forceinline__ void quad_c<false, uint16_t>(const uint16_t* p, int (&o)[4]) { quad_u16<false>(p, o); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
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

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Bundled path: stage v_s (scaled like stage_vector), zero the 64-bit
// accumulator, and return this thread's max |staged value| (+inf or NaN if the
// vector is not finite, so that the caller sees it).
template <bool kScatter>
__device__ __forceinline__ float stage_vector_max(const DevPlan& P, const float* __restrict__ vin, int v_stride,
                                                  int s, float* sv, unsigned long long* acc, int t0, int nt) {
  const float4* v4 = reinterpret_cast<const float4*>(vin + (size_t)s * v_stride);
  const float4* cs4 =
      P.colscale ? reinterpret_cast<const float4*>(P.colscale + (size_t)s * P.n_pad) : nullptr;
  float4* sv4 = reinterpret_cast<float4*>(sv);
  float m = 0.f;
  bool bad = false;
  for (int k = t0; k < P.n_pad / 4; k += nt) {
    float4 x = v4[k];
    if (cs4) {
      const float4 q = cs4[k];
      x.x *= q.x; x.y *= q.y; x.z *= q.z; x.w *= q.w;
    }
    sv4[k] = x;
    m = fmaxf(m, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
    bad |= !(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(x.w));
  }
  if (kScatter) {
    ulonglong2* a2 = reinterpret_cast<ulonglong2*>(acc);
    for (int k = t0; k < P.n_pad / 2; k += nt) a2[k] = make_ulonglong2(0ull, 0ull);
  }
  return bad ? __int_as_float(0x7f800000) : m;
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

// The CTA that finishes last publishes the pass's bookkeeping: per scenario,
// the ordered list of partial slots that were written (paths 1 and 2; static
// for path 0) and the objective summed in slot order; it also resets the chunk
// queues and the finishing counter for the next pass.  Every CTA must call it.
template <bool kObjective>
__device__ __forceinline__ void finish_pass(const DevPlan& P) {
  __shared__ bool last_cta;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last_cta = (atomicAdd(P.done_ctr, 1u) + 1u == gridDim.x);
  }
  __syncthreads();
  if (!last_cta) return;
  __threadfence();
  // one warp per scenario; lane l takes the l-th contiguous range of slots, so the
  // slot list comes out in increasing order and the objective is summed in a
  // fixed order for a given set of slots
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  constexpr unsigned kFull = 0xffffffffu;
  for (int s = threadIdx.x >> 5; s < P.N; s += nw) {
    double o = 0.0;
    if (P.path >= 1) {
      const int per = (P.grid + 31) / 32;
      const int cb = min(lane * per, P.grid), ce = min(cb + per, P.grid);
      const unsigned char* vis = P.visited + (size_t)s * P.grid;
      int cnt = 0;
      for (int c = cb; c < ce; ++c)
        if (__ldcg(vis + c)) {
          ++cnt;
          if (kObjective) o += __ldcg(&P.objp[c * P.N + s]);
        }
      int incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
      }
      int pos = incl - cnt;
      for (int c = cb; c < ce; ++c)
        if (__ldcg(vis + c)) {
          P.slot_list[(size_t)s * P.slot_cap + pos++] = c * P.N + s;
          P.visited[(size_t)s * P.grid + c] = 0;
        }
      const int total = __shfl_sync(kFull, incl, 31);
      if (lane == 0) {
        P.slot_count[s] = total;
        P.qnext[s] = 0;
      }
    } else if (kObjective) {
      const int cnt = P.slot_count[s];
      const int per = (cnt + 31) / 32;
      const int kb = min(lane * per, cnt), ke = min(kb + per, cnt);
      for (int k = kb; k < ke; ++k) o += __ldcg(&P.objp[P.slot_list[(size_t)s * P.slot_cap + k]]);
    }
    if (kObjective) {
      o = warp_sum_d(o);
      if (lane == 0) P.objs[s] = o;
    }
  }
  if (threadIdx.x == 0) *P.done_ctr = 0u;
}

}  // namespace
}  // namespace rpt
