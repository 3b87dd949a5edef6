// Correction passes of the high-precision path (mixed-precision iterative
// refinement around the exact Q1.63 passes).
//
// For a base estimate X (Q1.63) the remaining error e = pi - X solves
// e = r + (1-alpha) e P, the same contraction as Eq. 7 with r in place of
// alpha e_s: r = alpha r_push when X is the reserve of a push state (then
// pi = X + sum_v r_push(v) pi_v), r = X' - X when X' is one exact pass from X.
// These passes solve it with FP32 arithmetic, the gathered z_e = (1-alpha) e/d
// stored in FP32 (half the bytes of a Q1.63 gather) or BF16 (a quarter; its
// rounding stalls the iteration near 1e-2 of the cycle's start, so it serves
// the first part of a cycle).  The result is folded into X, and an exact pass
// measures ||X' - X||_1, which certifies the stop exactly as before: the
// precision of these passes decides how fast the bound falls, never whether
// it holds.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "f32_lanes.cuh"
#include "sweep_kernel.cuh"

namespace ppr {

typedef __nv_bfloat16 bf16;

struct RefArgs {
  int32_t n_items;
  const int4* items;  // work list for RLay<KT, T>::L lanes per row
  const int32_t* in_rp;
  const int32_t* in_ci;
  const int32_t* deg;
  const void* ze_in;   // (1-alpha) e / d, FP32 or BF16 [n][KT]
  void* ze_out;        // same type as ze_in
  const float* rf;     // r of the cycle
  float* e_out;        // e of this pass (NULL: not written)
  float one_minus_alpha;
  float relax;         // in-place passes: z_e <- z_e + relax (z_e' - z_e); 1 = plain
  const int32_t* npieces;
  float* heavy_acc;
  unsigned int* heavy_cnt;
  double* resid;       // [KT] sums of |e_new - e_old| (NULL: not measured)
  int light_first = 1; // in-place passes: deal the work list from its light end
};

// a lane loads 16 B of a node's tile row (V values of T); L lanes cover the row
template <int KT, typename T>
struct RLay {
  static constexpr int VMAX = 16 / (int)sizeof(T);
  static constexpr int V = KT < VMAX ? KT : VMAX;
  static constexpr int L = KT / V;
  static constexpr int EPW = 32 / L;
};

constexpr int kBf16FastBlocks = 5;

// gathers in flight per lane and blocks per SM (measured on R-MAT scale 20):
// FP32 rows: wide rows keep more gathers per warp, narrow ones more warps;
// BF16 rows carry 8 columns per lane, whose sums need 64 registers
template <int KT, typename T, bool MEAS>
struct RefTune {
  static constexpr bool kBf16 = sizeof(T) == 2;
  static constexpr int UNR = kBf16 ? 8 : (RLay<KT, T>::L >= 8 ? 8 : 4);
  // passes without the residual sums need fewer registers
  static constexpr int MIN_BLOCKS = kBf16 ? (MEAS ? 4 : kBf16FastBlocks) : (RLay<KT, T>::L >= 8 ? 6 : 8);
};

// raw 16-byte (or narrower) row piece of V values of T, converted to FP32 when summed
template <typename T, int V>
struct Raw;
template <>
struct Raw<float, 4> { typedef float4 type; };
template <>
struct Raw<float, 2> { typedef float2 type; };
template <>
struct Raw<float, 1> { typedef float type; };
template <>
struct Raw<bf16, 8> { typedef uint4 type; };
template <>
struct Raw<bf16, 4> { typedef uint2 type; };
template <>
struct Raw<bf16, 2> { typedef unsigned int type; };
template <>
struct Raw<bf16, 1> { typedef unsigned short type; };

// Loads of z_e.  An in-place pass (every unmeasured pass) writes the buffer
// it gathers from, so its loads go through L2 (ld.global.cg, coherent across
// SMs); the read-only path (ld.global.nc) serves only buffers that no thread
// writes during the kernel (the measured pass reads one buffer and writes the
// other).
template <typename T, int V, bool COH = false>
__device__ __forceinline__ typename Raw<T, V>::type ld_raw(const T* p) {
  const auto* q = reinterpret_cast<const typename Raw<T, V>::type*>(p);
  if constexpr (COH) return __ldcg(q);
  else return __ldg(q);
}
template <typename T, int V>
__device__ __forceinline__ typename Raw<T, V>::type zero_raw() {
  typename Raw<T, V>::type z{};
  return z;
}

// BF16 -> FP32 is exact: the 16 stored bits are the high half of the float
__device__ __forceinline__ float bf_lo(unsigned w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(unsigned w) { return __uint_as_float(w & 0xffff0000u); }

// a0 += lo(w), a1 += hi(w) for two BF16 values packed in w, each widened
// exactly and added with one rounding (round to nearest), like
// a0 += bf_lo(w), a1 += bf_hi(w), but as one mixed-precision add per value
// (add.f32.bf16) instead of a shift or mask followed by an FP32 add: the
// widening had made the ALU pipe the busiest one of the BF16 pass
__device__ __forceinline__ void add_bf2(float& a0, float& a1, unsigned w) {
  asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
      "add.rn.f32.bf16 %0, lo, %0;\n\tadd.rn.f32.bf16 %1, hi, %1;\n\t}"
      : "+f"(a0), "+f"(a1)
      : "r"(w));
}

template <typename T, int V>
__device__ __forceinline__ void add_raw(float (&acc)[V], const typename Raw<T, V>::type& t) {
  if constexpr (std::is_same<T, float>::value) {
    if constexpr (V == 4) { acc[0] += t.x; acc[1] += t.y; acc[2] += t.z; acc[3] += t.w; }
    else if constexpr (V == 2) { acc[0] += t.x; acc[1] += t.y; }
    else { acc[0] += t; }
  } else {
    if constexpr (V == 8) {
      add_bf2(acc[0], acc[1], t.x);
      add_bf2(acc[2], acc[3], t.y);
      add_bf2(acc[4], acc[5], t.z);
      add_bf2(acc[6], acc[7], t.w);
    } else if constexpr (V == 4) {
      add_bf2(acc[0], acc[1], t.x);
      add_bf2(acc[2], acc[3], t.y);
    } else if constexpr (V == 2) {
      add_bf2(acc[0], acc[1], t);
    } else {
      acc[0] += bf_lo((unsigned)t);
    }
  }
}

template <typename T, int V, bool COH>
__device__ __forceinline__ void ld_row(const T* p, float (&v)[V]) {
#pragma unroll
  for (int q = 0; q < V; ++q) v[q] = 0.f;
  add_raw<T, V>(v, ld_raw<T, V, COH>(p));
}

// FP32 row piece of V values (V up to 8)
template <int V>
__device__ __forceinline__ void ld_f32(const float* p, float (&v)[V]) {
  if constexpr (V == 8) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
    ldf<V>(p, v);
  }
}

template <int V>
__device__ __forceinline__ void st_f32(float* p, const float (&v)[V]) {
  if constexpr (V == 8) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
  } else if constexpr (V == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (V == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
    p[0] = v[0];
  }
}

__device__ __forceinline__ unsigned pack_bf2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
  return *reinterpret_cast<const unsigned*>(&h);
}

template <typename T, int V>
__device__ __forceinline__ void st_row(T* p, const float (&v)[V]) {
  if constexpr (std::is_same<T, float>::value) {
    st_f32<V>(p, v);
  } else if constexpr (V == 8) {
    *reinterpret_cast<uint4*>(p) = make_uint4(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]), pack_bf2(v[4], v[5]),
                                              pack_bf2(v[6], v[7]));
  } else if constexpr (V == 4) {
    *reinterpret_cast<uint2*>(p) = make_uint2(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]));
  } else if constexpr (V == 2) {
    *reinterpret_cast<unsigned*>(p) = pack_bf2(v[0], v[1]);
  } else {
    *reinterpret_cast<bf16*>(p) = __float2bfloat16_rn(v[0]);
  }
}

// row operands of the epilogue, r of the row (read-only for the whole pass)
// and d.  BF16 passes load them before the row's gathers so that their
// latency overlaps them; FP32 passes, short of registers, load them after
// (measured both ways on R-MAT scale 20: each choice is the faster one)
template <int V>
struct RowPre {
  float r[V];
  float d;
};

template <typename T>
constexpr bool kPrefetchRow = sizeof(T) == 2;

template <int KT, typename T>
__device__ __forceinline__ RowPre<RLay<KT, T>::V> refine_prefetch(const RefArgs& a, int u, int slot) {
  constexpr int V = RLay<KT, T>::V;
  RowPre<V> p{};
  if constexpr (kPrefetchRow<T>) {
    ld_f32<V>(a.rf + (size_t)u * KT + slot * V, p.r);
    p.d = (float)__ldg(&a.deg[u]);
  }
  return p;
}

// finish row u: e = r + sum, ze = e (1-alpha) / d
template <int KT, typename T, bool MEAS>
__device__ __forceinline__ void refine_epilogue(const RefArgs& a, int u, int slot,
                                                const RowPre<RLay<KT, T>::V>& pre,
                                                const float (&acc)[RLay<KT, T>::V],
                                                float (&res)[RLay<KT, T>::V]) {
  constexpr int V = RLay<KT, T>::V;
  const size_t base = (size_t)u * KT + slot * V;
  float r[V];
  float d;
  if constexpr (kPrefetchRow<T>) {
#pragma unroll
    for (int q = 0; q < V; ++q) r[q] = pre.r[q];
    d = pre.d;
  } else {
    ld_f32<V>(a.rf + base, r);
    d = (float)__ldg(&a.deg[u]);
  }
  const float share = a.one_minus_alpha / d;
  float e[V], zn[V];
#pragma unroll
  for (int q = 0; q < V; ++q) {
    e[q] = r[q] + acc[q];
    zn[q] = e[q] * share;
  }
  if (a.relax != 1.f) {
    // over-relaxed in-place pass (ze_in == ze_out): this row's own old value
    float zo[V];
    ld_row<T, V, !MEAS>(static_cast<const T*>(a.ze_in) + base, zo);
#pragma unroll
    for (int q = 0; q < V; ++q) zn[q] = zo[q] + a.relax * (zn[q] - zo[q]);
  }
  if (MEAS) {
    float zo[V];
    ld_row<T, V, false>(static_cast<const T*>(a.ze_in) + base, zo);
    const float inv = d / a.one_minus_alpha;
#pragma unroll
    for (int q = 0; q < V; ++q) res[q] += fabsf(zn[q] - zo[q]) * inv;
  }
  st_row<T, V>(static_cast<T*>(a.ze_out) + base, zn);
  if (a.e_out) st_f32<V>(a.e_out + base, e);
}

template <int KT, typename T, bool COH>
__device__ __forceinline__ void refine_gather_warp(const RefArgs& a, int e_begin, int e_end, int lane, int slot,
                                                   float (&acc)[RLay<KT, T>::V]) {
  constexpr int V = RLay<KT, T>::V, L = RLay<KT, T>::L, EPW = RLay<KT, T>::EPW, UNR = RefTune<KT, T, false>::UNR;
  const T* z = static_cast<const T*>(a.ze_in);
  for (int base = e_begin; base < e_end; base += EPW * UNR) {
    int v[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) {
      const int e = base + q * EPW + lane / L;
      v[q] = e < e_end ? __ldg(&a.in_ci[e]) : -1;
    }
    typename Raw<T, V>::type t[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q)
      t[q] = v[q] >= 0 ? ld_raw<T, V, COH>(z + (size_t)v[q] * KT + slot * V) : zero_raw<T, V>();
#pragma unroll
    for (int q = 0; q < UNR; ++q) add_raw<T, V>(acc, t[q]);
  }
}

// One work item of a pass (see build_plan): a piece of a split row, a run of
// medium rows (a warp per row) or a run of light rows (L lanes per row).
template <int KT, typename T, bool MEAS>
__device__ __forceinline__ void refine_item(const RefArgs& a, const int4 w, int lane, int slot,
                                            float (&res)[RLay<KT, T>::V]) {
  constexpr int V = RLay<KT, T>::V, L = RLay<KT, T>::L;
  const T* z = static_cast<const T*>(a.ze_in);
  if (w.x == 0) {
    // piece of a split row; the last piece to arrive finishes the row
    const int u = w.y;
    float acc[V] = {};
    refine_gather_warp<KT, T, !MEAS>(a, w.z, w.w, lane, slot, acc);
#pragma unroll
    for (int off = L; off < 32; off <<= 1)
#pragma unroll
      for (int q = 0; q < V; ++q) acc[q] += __shfl_xor_sync(kFull, acc[q], off);
    if (lane < L)
#pragma unroll
      for (int q = 0; q < V; ++q) atomicAdd(&a.heavy_acc[(size_t)u * KT + slot * V + q], acc[q]);
    __threadfence();
    unsigned ticket = 0;
    if (lane == 0) ticket = atomicAdd(&a.heavy_cnt[u], 1u);
    ticket = __shfl_sync(kFull, ticket, 0);
    if (ticket == (unsigned)a.npieces[u] - 1u) {
      __threadfence();
      if (lane < L) {
        float tot[V];
#pragma unroll
        for (int q = 0; q < V; ++q) tot[q] = atomicExch(&a.heavy_acc[(size_t)u * KT + slot * V + q], 0.f);
        refine_epilogue<KT, T, MEAS>(a, u, slot, refine_prefetch<KT, T>(a, u, slot), tot, res);
      }
      if (lane == 0) atomicExch(&a.heavy_cnt[u], 0u);
    }
  } else if (w.x == 1) {
    for (int u = w.y; u < w.z; ++u) {
      const auto pre = refine_prefetch<KT, T>(a, u, slot);
      float acc[V] = {};
      refine_gather_warp<KT, T, !MEAS>(a, __ldg(&a.in_rp[u]), __ldg(&a.in_rp[u + 1]), lane, slot, acc);
#pragma unroll
      for (int off = L; off < 32; off <<= 1)
#pragma unroll
        for (int q = 0; q < V; ++q) acc[q] += __shfl_xor_sync(kFull, acc[q], off);
      if (lane < L) refine_epilogue<KT, T, MEAS>(a, u, slot, pre, acc, res);
    }
  } else {
    for (int u = w.y + lane / L; u < w.z; u += 32 / L) {
      const auto pre = refine_prefetch<KT, T>(a, u, slot);
      const int e1 = __ldg(&a.in_rp[u + 1]);
      float acc[V] = {};
#pragma unroll RefTune<KT, T, MEAS>::UNR
      for (int e = __ldg(&a.in_rp[u]); e < e1; ++e)
        add_raw<T, V>(acc, ld_raw<T, V, !MEAS>(z + (size_t)__ldg(&a.in_ci[e]) * KT + slot * V));
      refine_epilogue<KT, T, MEAS>(a, u, slot, pre, acc, res);
    }
  }
}

// per-column sums |e' - e| of a block into resid: warp w's partial sums are
// in sred[w][0..KT), then one atomic per column
template <int KT>
__device__ __forceinline__ void refine_resid_block(float (&sred)[8][KT], double* resid) {
  __syncthreads();
  if (threadIdx.x < KT) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += (double)sred[w][threadIdx.x];
    atomicAdd(&resid[threadIdx.x], sum);
  }
}

// MEAS: the measured (synchronous) pass of a batch, which also sums |e' - e|.
// An in-place pass (asynchronous updates) with a.light_first deals the work
// list from its light end: the light rows (at most 16 in-edges, 90 % of the
// rows of an R-MAT graph, 12 % of its edges) are updated first, and the rows
// with many in-edges, which hold 88 % of the edges, then gather their fresh
// values in the same pass.  Dealt from the heavy end instead, those gathers
// read the light rows' values of the previous pass: R-MAT scale 22 took 46.7
// instead of 38.8 passes per 64-source tile, scale 20 39.5 instead of 37.8
// (and alternating the two directions 57.5).
template <int KT, typename T, bool MEAS>
__global__ void __launch_bounds__(256, (RefTune<KT, T, MEAS>::MIN_BLOCKS)) refine_pass_kernel(RefArgs a) {
  constexpr int V = RLay<KT, T>::V, L = RLay<KT, T>::L;
  const int lane = threadIdx.x & 31;
  const int slot = lane % L;
  float res[V];
#pragma unroll
  for (int q = 0; q < V; ++q) res[q] = 0.f;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < a.n_items; it += nwarps)
    refine_item<KT, T, MEAS>(a, __ldg(&a.items[(MEAS || !a.light_first) ? it : a.n_items - 1 - it]), lane, slot, res);
  if constexpr (MEAS) {
    __shared__ float sred[8][KT];
#pragma unroll
    for (int off = L; off < 32; off <<= 1)
#pragma unroll
      for (int q = 0; q < V; ++q) res[q] += __shfl_xor_sync(kFull, res[q], off);
    const int warp = threadIdx.x >> 5;
    if (lane < L)
#pragma unroll
      for (int q = 0; q < V; ++q) sred[warp][lane * V + q] = res[q];
    refine_resid_block<KT>(sred, a.resid);
  }
}

// z_e of the BF16 passes into FP32 (exact) for the FP32 passes that follow
__global__ void bf16_to_f32_kernel(int64_t count, const bf16* __restrict__ in, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __bfloat162float(in[i]);
}

template <typename T>
__device__ __forceinline__ void st_one(T* p, float v) {
  if constexpr (std::is_same<T, float>::value) *p = v;
  else *p = __float2bfloat16_rn(v);
}

// The setup and fold kernels below stream n x KT cells.  With KT >= 4 a
// thread takes 4 cells of one node per step, as 16-byte loads and stores:
// one 8-byte load per thread and step kept too few bytes in flight to cover
// the DRAM latency (the setup ran at 0.41 of the copy bandwidth).
template <int KT>
struct Ew {
  static constexpr int G = KT >= 4 ? 4 : 1;  // cells per thread and step
};

__device__ __forceinline__ void ld4(const u64* p, u64 (&v)[4]) {
  const ulonglong2 a = reinterpret_cast<const ulonglong2*>(p)[0];
  const ulonglong2 b = reinterpret_cast<const ulonglong2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

__device__ __forceinline__ void st4(u64* p, const u64 (&v)[4]) {
  reinterpret_cast<ulonglong2*>(p)[0] = make_ulonglong2(v[0], v[1]);
  reinterpret_cast<ulonglong2*>(p)[1] = make_ulonglong2(v[2], v[3]);
}

__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

__device__ __forceinline__ void st4(bf16* p, const float (&v)[4]) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]), hi = __floats2bfloat162_rn(v[2], v[3]);
  uint2 w;
  w.x = *reinterpret_cast<unsigned int*>(&lo);
  w.y = *reinterpret_cast<unsigned int*>(&hi);
  *reinterpret_cast<uint2*>(p) = w;
}

// r of a push state: rf = alpha r_push (FP32, the fixed-point r_push rounded
// to FP32, then times alpha), first correction e1 = rf
template <int KT, typename T>
__global__ void refine_setup_push_kernel(int64_t n, const u64* __restrict__ r_push, double alpha,
                                         const int32_t* __restrict__ deg, float one_minus_alpha, float* __restrict__ rf,
                                         T* __restrict__ ze) {
  constexpr int G = Ew<KT>::G;
  const int64_t groups = n * KT / G;
  const float af = (float)alpha;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = g * G;
    const float s = one_minus_alpha / (float)deg[i / KT];
    if constexpr (G == 4) {
      u64 r[4];
      ld4(r_push + i, r);
      float v[4], z[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        v[q] = u64_to_f32<-63>(r[q]) * af;
        z[q] = v[q] * s;
      }
      st4(rf + i, v);
      st4(ze + i, z);
    } else {
      const float v = u64_to_f32<-63>(r_push[i]) * af;
      rf[i] = v;
      st_one<T>(ze + i, v * s);
    }
  }
}

// r of X after one exact pass X': rf = X' - X (exact signed difference, then FP32)
template <int KT, typename T>
__global__ void refine_setup_resid_kernel(int64_t n, const u64* __restrict__ x_new, const u64* __restrict__ x,
                                          const int32_t* __restrict__ deg, float one_minus_alpha,
                                          float* __restrict__ rf, T* __restrict__ ze) {
  constexpr int G = Ew<KT>::G;
  const int64_t groups = n * KT / G;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = g * G;
    const float s = one_minus_alpha / (float)deg[i / KT];
    u64 a[G], b[G];
    if constexpr (G == 4) {
      ld4(x_new + i, a);
      ld4(x + i, b);
    } else {
      a[0] = x_new[i];
      b[0] = x[i];
    }
    float v[G], z[G];
#pragma unroll
    for (int q = 0; q < G; ++q) {
      v[q] = sfix_to_f32((long long)(a[q] - b[q]));
      z[q] = v[q] * s;
    }
    if constexpr (G == 4) {
      st4(rf + i, v);
      st4(ze + i, z);
    } else {
      rf[i] = v[0];
      st_one<T>(ze + i, z[0]);
    }
  }
}

// X += e (rounded to Q1.63, kept >= 0); z = (1-alpha) X / d for the exact pass
template <int KT>
__global__ void refine_fold_kernel(int64_t n, const float* __restrict__ e, u64* __restrict__ x,
                                   const uint64_t* __restrict__ omega, u64* __restrict__ z) {
  constexpr int G = Ew<KT>::G;
  const int64_t groups = n * KT / G;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = g * G;
    const uint64_t om = omega[i / KT];
    float ev[G];
    u64 xv[G], zv[G];
    if constexpr (G == 4) {
      const float4 e4 = reinterpret_cast<const float4*>(e + i)[0];
      ev[0] = e4.x; ev[1] = e4.y; ev[2] = e4.z; ev[3] = e4.w;
      ld4(x + i, xv);
    } else {
      ev[0] = e[i];
      xv[0] = x[i];
    }
#pragma unroll
    for (int q = 0; q < G; ++q) {
      const long long s = (long long)xv[q] + f32_to_sfix(ev[q]);
      xv[q] = s > 0 ? (u64)s : 0ull;
      zv[q] = mulhi_round(xv[q], om);
    }
    if constexpr (G == 4) {
      st4(x + i, xv);
      st4(z + i, zv);
    } else {
      x[i] = xv[0];
      z[i] = zv[0];
    }
  }
}

// z = (1-alpha) x / d
template <int KT>
__global__ void z_of_x_kernel(int64_t n, const u64* __restrict__ x, const uint64_t* __restrict__ omega,
                              u64* __restrict__ z) {
  const int64_t total = n * KT;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = mulhi_round(x[i], omega[i / KT]);
}

}  // namespace ppr
