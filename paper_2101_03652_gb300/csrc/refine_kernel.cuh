// FP32 correction passes of the high-precision path (mixed-precision
// iterative refinement around the exact Q1.63 passes).
//
// For a base estimate X (Q1.63) the remaining error e = pi - X solves
// e = r + (1-alpha) e P, the same contraction as Eq. 7 with r in place of
// alpha e_s: r = alpha r_push when X is the reserve of a push state (then
// pi = X + sum_v r_push(v) pi_v), r = X' - X when X' is one exact pass from X.
// These passes solve it in FP32 (half the bytes of a Q1.63 gather), the result
// is folded into X, and an exact pass measures ||X' - X||_1, which certifies
// the stop exactly as before: the precision of the FP32 passes decides how
// fast the bound falls, never whether it holds.
#pragma once

#include "f32_lanes.cuh"
#include "sweep_kernel.cuh"

namespace ppr {

struct RefArgs {
  int32_t n_items;
  const int4* items;  // work list for Lay32<KT>::L lanes per row
  const int32_t* in_rp;
  const int32_t* in_ci;
  const int32_t* deg;
  const float* ze_in;  // (1-alpha) e / d
  float* ze_out;
  const float* rf;     // r of the cycle
  float* e_out;        // e of this pass (NULL: not written)
  float one_minus_alpha;
  const int32_t* npieces;
  float* heavy_acc;
  unsigned int* heavy_cnt;
  double* resid;       // [KT] sums of |e_new - e_old| (NULL: not measured)
};

// gathers in flight per lane and blocks per SM: wide tiles keep more gathers
// per warp; narrow ones more warps (measured on R-MAT scale 20)
template <int KT>
struct RefTune {
  static constexpr int UNR = KT >= 32 ? 8 : 4;
  static constexpr int MIN_BLOCKS = KT >= 32 ? 6 : 8;
};

template <int V>
__device__ __forceinline__ void stf(float* p, const float (&v)[V]) {
  if constexpr (V == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (V == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
    p[0] = v[0];
  }
}

// finish row u: e = r + sum, ze = e (1-alpha) / d
template <int KT>
__device__ __forceinline__ void refine_epilogue(const RefArgs& a, int u, int slot, const float (&acc)[Lay32<KT>::V],
                                                float (&res)[Lay32<KT>::V]) {
  constexpr int V = Lay32<KT>::V;
  const float d = (float)__ldg(&a.deg[u]);
  const float share = a.one_minus_alpha / d;
  const size_t base = (size_t)u * KT + slot * V;
  float r[V], e[V], zn[V];
  ldf<V>(a.rf + base, r);  // read-only for the whole pass
#pragma unroll
  for (int q = 0; q < V; ++q) {
    e[q] = r[q] + acc[q];
    zn[q] = e[q] * share;
  }
  if (a.resid) {
    float zo[V];
    ldf<V>(a.ze_in + base, zo);
    const float inv = d / a.one_minus_alpha;
#pragma unroll
    for (int q = 0; q < V; ++q) res[q] += fabsf(zn[q] - zo[q]) * inv;
  }
  stf<V>(a.ze_out + base, zn);
  if (a.e_out) stf<V>(a.e_out + base, e);
}

template <int KT>
__device__ __forceinline__ void refine_gather_warp(const RefArgs& a, int e_begin, int e_end, int lane, int slot,
                                                   float (&acc)[Lay32<KT>::V]) {
  constexpr int V = Lay32<KT>::V, L = Lay32<KT>::L, EPW = Lay32<KT>::EPW, UNR = RefTune<KT>::UNR;
  for (int base = e_begin; base < e_end; base += EPW * UNR) {
    int v[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) {
      const int e = base + q * EPW + lane / L;
      v[q] = e < e_end ? __ldg(&a.in_ci[e]) : -1;
    }
    float t[UNR][V];
#pragma unroll
    for (int q = 0; q < UNR; ++q) {
      if (v[q] >= 0) {
        ldf<V>(a.ze_in + (size_t)v[q] * KT + slot * V, t[q]);
      } else {
#pragma unroll
        for (int w = 0; w < V; ++w) t[q][w] = 0.f;
      }
    }
#pragma unroll
    for (int q = 0; q < UNR; ++q)
#pragma unroll
      for (int w = 0; w < V; ++w) acc[w] += t[q][w];
  }
}

template <int KT>
__global__ void __launch_bounds__(256, RefTune<KT>::MIN_BLOCKS) refine_pass_kernel(RefArgs a) {
  constexpr int V = Lay32<KT>::V, L = Lay32<KT>::L;
  const int lane = threadIdx.x & 31;
  const int slot = lane % L;
  float res[V];
#pragma unroll
  for (int q = 0; q < V; ++q) res[q] = 0.f;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < a.n_items; it += nwarps) {
    const int4 w = __ldg(&a.items[it]);
    if (w.x == 0) {
      // piece of a split row; the last piece to arrive finishes the row
      const int u = w.y;
      float acc[V] = {};
      refine_gather_warp<KT>(a, w.z, w.w, lane, slot, acc);
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
          refine_epilogue<KT>(a, u, slot, tot, res);
        }
        if (lane == 0) atomicExch(&a.heavy_cnt[u], 0u);
      }
    } else if (w.x == 1) {
      for (int u = w.y; u < w.z; ++u) {
        float acc[V] = {};
        refine_gather_warp<KT>(a, __ldg(&a.in_rp[u]), __ldg(&a.in_rp[u + 1]), lane, slot, acc);
#pragma unroll
        for (int off = L; off < 32; off <<= 1)
#pragma unroll
          for (int q = 0; q < V; ++q) acc[q] += __shfl_xor_sync(kFull, acc[q], off);
        if (lane < L) refine_epilogue<KT>(a, u, slot, acc, res);
      }
    } else {
      for (int u = w.y + lane / L; u < w.z; u += 32 / L) {
        const int e1 = __ldg(&a.in_rp[u + 1]);
        float acc[V] = {};
#pragma unroll RefTune<KT>::UNR
        for (int e = __ldg(&a.in_rp[u]); e < e1; ++e) {
          float t[V];
          ldf<V>(a.ze_in + (size_t)__ldg(&a.in_ci[e]) * KT + slot * V, t);
#pragma unroll
          for (int q = 0; q < V; ++q) acc[q] += t[q];
        }
        refine_epilogue<KT>(a, u, slot, acc, res);
      }
    }
  }
  if (!a.resid) return;
  __shared__ float sred[8][KT];
#pragma unroll
  for (int off = L; off < 32; off <<= 1)
#pragma unroll
    for (int q = 0; q < V; ++q) res[q] += __shfl_xor_sync(kFull, res[q], off);
  const int warp = threadIdx.x >> 5;
  if (lane < L)
#pragma unroll
    for (int q = 0; q < V; ++q) sred[warp][lane * V + q] = res[q];
  __syncthreads();
  if (threadIdx.x < KT) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += (double)sred[w][threadIdx.x];
    atomicAdd(&a.resid[threadIdx.x], sum);
  }
}

// r of a push state: rf = alpha r_push (FP32), first correction e1 = rf
template <int KT>
__global__ void refine_setup_push_kernel(int64_t n, const u64* __restrict__ r_push, double alpha,
                                         const int32_t* __restrict__ deg, float one_minus_alpha, float* __restrict__ rf,
                                         float* __restrict__ ze) {
  const int64_t total = n * KT;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = (float)((double)r_push[i] * (alpha / kFixOne));
    rf[i] = v;
    ze[i] = v * (one_minus_alpha / (float)deg[i / KT]);
  }
}

// r of X after one exact pass X': rf = X' - X (exact signed difference, then FP32)
template <int KT>
__global__ void refine_setup_resid_kernel(int64_t n, const u64* __restrict__ x_new, const u64* __restrict__ x,
                                          const int32_t* __restrict__ deg, float one_minus_alpha,
                                          float* __restrict__ rf, float* __restrict__ ze) {
  const int64_t total = n * KT;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const long long dlt = (long long)(x_new[i] - x[i]);
    const float v = (float)((double)dlt * (1.0 / kFixOne));
    rf[i] = v;
    ze[i] = v * (one_minus_alpha / (float)deg[i / KT]);
  }
}

// X += e (rounded to Q1.63, kept >= 0); z = (1-alpha) X / d for the exact pass
template <int KT>
__global__ void refine_fold_kernel(int64_t n, const float* __restrict__ e, u64* __restrict__ x,
                                   const uint64_t* __restrict__ omega, u64* __restrict__ z) {
  const int64_t total = n * KT;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const long long dlt = llrint((double)e[i] * kFixOne);
    const long long xv = (long long)x[i] + dlt;
    const u64 xn = xv > 0 ? (u64)xv : 0ull;
    x[i] = xn;
    z[i] = mulhi_round(xn, omega[i / KT]);
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
