// The pull sweep of the high-precision path (one pass of SimFwdPush in
// estimate form, Sec. 4.1 Eq. 7 with Lemma 1): for every in-CSR row u,
// x'(u) = alpha [u = s] + sum over in-neighbours v of z(v), z = (1-alpha) x / d,
// for a tile of KT sources at once.  Values are Q1.63 fixed point.
#pragma once

#include <cuda_bf16.h>

#include "fixconv.cuh"
#include "ppr_internal.cuh"

namespace ppr {

typedef unsigned long long u64;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ u64 mulhi_round(u64 x, u64 w) {
  u64 hi = __umul64hi(x, w);
  u64 lo = x * w;
  return hi + (lo >> 63);
}

// ------------------------------------------------------------ sweep phase
struct SweepArgs {
  int32_t n_items;   // work items of this pass (items over rows without in-edges come last and
                     // are left out once those rows hold their constant value in both buffers)
  const int4* items; // {kind, a, b, c}: kind 0 = piece [b, c) of split row a; 1 = rows [a, b)
                     // one warp per row; 2 = rows [a, b) with L lanes per row
  const int32_t* in_rp;
  const int32_t* in_ci;
  const uint64_t* omega;
  const float* invw;
  const u64* z_in;
  u64* z_out;        // NULL: z of this pass not stored (a measuring pass)
  u64* x_out;        // optional: the estimate x of this pass
  int32_t src[64];   // tile's sources (new ids), -1 for unused columns
  u64 alpha_raw;     // alpha in Q1.63
  double* resid;     // [KT] sums of |x_new - x_old| in raw units (this pass); NULL: not needed
  const int32_t* heavy_npieces;
  u64* heavy_acc;
  unsigned int* heavy_cnt;
  // measuring pass that also sets up the next refinement cycle (x_base not
  // NULL): r = x' - x_base exactly, its l1 norm into resid, r as FP32 into
  // rf_next and r (1-alpha)/d into ze_next (FP32, or BF16 when ze_bf16);
  // neither z_out nor x_out is written
  const u64* x_base = nullptr;
  float* rf_next = nullptr;
  void* ze_next = nullptr;
  int ze_bf16 = 0;
};

constexpr int kItemPeriods = 16;  // target cost of one work item (see build_plan)
constexpr int kLightMax = 16;     // rows with at most this many in-edges use lane groups
constexpr int kUnr = 4;           // gathers each lane issues before consuming them

template <int KT>
struct Lay {
  static constexpr int V = KT >= 2 ? 2 : 1;  // uint64 per lane load (16 B when 2)
  static constexpr int L = KT / V;           // lanes covering one row of the tile
  static constexpr int EPW = 32 / L;         // edges a warp gathers per step
};

// COH: the buffer is written during the kernel (an in-place pass), so the
// load goes through L2 (ld.global.cg) instead of the read-only path
template <int V, bool COH = false>
__device__ __forceinline__ void ld_vec(const u64* p, u64 (&v)[V]) {
  if constexpr (V == 2) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
    ulonglong2 t = COH ? __ldcg(q) : __ldg(q);
    v[0] = t.x;
    v[1] = t.y;
  } else {
    v[0] = COH ? __ldcg(p) : __ldg(p);
  }
}
template <int V>
__device__ __forceinline__ void st_vec(u64* p, const u64 (&v)[V]) {
  if constexpr (V == 2) {
    *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(v[0], v[1]);
  } else {
    p[0] = v[0];
  }
}

// finish row u for the V columns of `slot`: x = sum + alpha [u == s], z = x w
template <int KT, bool COH>
__device__ __forceinline__ void row_epilogue(const SweepArgs& a, int u, int slot, const u64 (&acc)[Lay<KT>::V],
                                             float (&res)[Lay<KT>::V]) {
  constexpr int V = Lay<KT>::V;
  const float iw = __ldg(&a.invw[u]);
  if (a.x_base) {
    const size_t base = (size_t)u * KT + slot * V;
    u64 xo[V];
    ld_vec<V>(a.x_base + base, xo);
    const float share = 1.f / iw;
#pragma unroll
    for (int q = 0; q < V; ++q) {
      const u64 xn = acc[q] + (u == a.src[slot * V + q] ? a.alpha_raw : 0ull);
      const long long d = (long long)(xn - xo[q]);
      res[q] += u64_to_f32<0>(d < 0 ? 0ull - (u64)d : (u64)d);
      const float rv = sfix_to_f32(d);
      a.rf_next[base + q] = rv;
      if (a.ze_bf16)
        static_cast<__nv_bfloat16*>(a.ze_next)[base + q] = __float2bfloat16_rn(rv * share);
      else
        static_cast<float*>(a.ze_next)[base + q] = rv * share;
    }
    return;
  }
  const u64 om = __ldg(&a.omega[u]);
  u64 zn[V], xn[V];
#pragma unroll
  for (int q = 0; q < V; ++q) {
    const int c = slot * V + q;
    xn[q] = acc[q] + (u == a.src[c] ? a.alpha_raw : 0ull);
    zn[q] = mulhi_round(xn[q], om);
  }
  if (a.resid) {
    u64 zo[V];
    ld_vec<V, COH>(a.z_in + (size_t)u * KT + slot * V, zo);
#pragma unroll
    for (int q = 0; q < V; ++q) res[q] += u64_to_f32<0>(zn[q] > zo[q] ? zn[q] - zo[q] : zo[q] - zn[q]) * iw;
  }
  if (a.z_out) st_vec<V>(a.z_out + (size_t)u * KT + slot * V, zn);
  if (a.x_out) st_vec<V>(a.x_out + (size_t)u * KT + slot * V, xn);
}

// Sum z over in-edges [e_begin, e_end) of one row; the warp's lanes cover
// EPW edges per step (L lanes per edge) and UNR steps are issued before any
// is consumed, so each lane keeps UNR independent gathers in flight.  The
// loop bound is warp-uniform; lanes past the end are predicated off.
template <int KT, int UNR, bool COH>
__device__ __forceinline__ void gather_warp(const SweepArgs& a, int e_begin, int e_end, int lane, int slot,
                                            u64 (&acc)[Lay<KT>::V]) {
  constexpr int V = Lay<KT>::V, L = Lay<KT>::L, EPW = Lay<KT>::EPW;
  for (int base = e_begin; base < e_end; base += EPW * UNR) {
    int v[UNR];
#pragma unroll
    for (int q = 0; q < UNR; ++q) {
      const int e = base + q * EPW + lane / L;
      v[q] = e < e_end ? __ldg(&a.in_ci[e]) : -1;
    }
    u64 t[UNR][V];
#pragma unroll
    for (int q = 0; q < UNR; ++q) {
      if (v[q] >= 0) {
        ld_vec<V, COH>(a.z_in + (size_t)v[q] * KT + slot * V, t[q]);
      } else {
#pragma unroll
        for (int w = 0; w < V; ++w) t[q][w] = 0;
      }
    }
#pragma unroll
    for (int q = 0; q < UNR; ++q)
#pragma unroll
      for (int w = 0; w < V; ++w) acc[w] += t[q][w];
  }
}

// INPLACE: z_out == z_in (asynchronous pass), loads of z through L2
template <int KT, bool INPLACE>
__global__ void __launch_bounds__(256, 6) sweep_kernel(SweepArgs a) {
  constexpr int V = Lay<KT>::V, L = Lay<KT>::L;
  constexpr int UNR = kUnr;
  const int lane = threadIdx.x & 31;
  const int slot = lane % L;
  float res[V];
#pragma unroll
  for (int q = 0; q < V; ++q) res[q] = 0.f;

  // Items are about equally long and grouped by kind; dealing them to warps
  // round-robin gives every warp nearly the same amount and mix of work
  // without any atomic on the claim path.
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < a.n_items; it += nwarps) {
    const int4 w = __ldg(&a.items[it]);
    if (w.x == 0) {
      // piece of a split row: partial sums combined with integer atomics; the
      // last piece of the row to arrive finishes it
      const int u = w.y;
      u64 acc[V] = {};
      gather_warp<KT, UNR, INPLACE>(a, w.z, w.w, lane, slot, acc);
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
      if (ticket == (unsigned)a.heavy_npieces[u] - 1u) {
        __threadfence();
        if (lane < L) {
          u64 tot[V];
#pragma unroll
          for (int q = 0; q < V; ++q) tot[q] = atomicExch(&a.heavy_acc[(size_t)u * KT + slot * V + q], 0ull);
          row_epilogue<KT, INPLACE>(a, u, slot, tot, res);
        }
        if (lane == 0) atomicExch(&a.heavy_cnt[u], 0u);
      }
    } else if (w.x == 1) {
      // medium rows: one warp per row
      for (int u = w.y; u < w.z; ++u) {
        u64 acc[V] = {};
        gather_warp<KT, UNR, INPLACE>(a, __ldg(&a.in_rp[u]), __ldg(&a.in_rp[u + 1]), lane, slot, acc);
#pragma unroll
        for (int off = L; off < 32; off <<= 1)
#pragma unroll
          for (int q = 0; q < V; ++q) acc[q] += __shfl_xor_sync(kFull, acc[q], off);
        if (lane < L) row_epilogue<KT, INPLACE>(a, u, slot, acc, res);
      }
    } else {
      // light rows: L lanes per row, 32/L consecutive rows at a time (rows are
      // sorted by length, so rows sharing a warp have nearly equal length)
      for (int u = w.y + lane / L; u < w.z; u += 32 / L) {
        const int e1 = __ldg(&a.in_rp[u + 1]);
        u64 acc[V] = {};
#pragma unroll 4
        for (int e = __ldg(&a.in_rp[u]); e < e1; ++e) {
          u64 t[V];
          ld_vec<V, INPLACE>(a.z_in + (size_t)__ldg(&a.in_ci[e]) * KT + slot * V, t);
#pragma unroll
          for (int q = 0; q < V; ++q) acc[q] += t[q];
        }
        row_epilogue<KT, INPLACE>(a, u, slot, acc, res);
      }
    }
  }

  if (!a.resid) return;
  // per-column residual: lanes with equal slot, then warps, then one atomic per column
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

}  // namespace ppr
