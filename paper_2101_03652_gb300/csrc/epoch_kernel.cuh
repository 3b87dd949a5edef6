// Algorithm 3's dense epochs on the GPU: in epoch i only nodes with
// r(v) > d_v r'_max, r'_max = lambda^(i/epochNum) / m, push; a pass pushes every
// such node at once (synchronous), as a pull over the in-CSR.  State is the
// residue r and reserve pi_hat in Q1.63; y(v) = (1-alpha) r(v) / d_v for the
// nodes that push in the coming pass, 0 otherwise.
#pragma once

#include "sweep_kernel.cuh"

namespace ppr {

struct EpochArgs {
  int32_t n_items;
  const int4* items;  // the work list of the pull sweep (same layout)
  const int32_t* in_rp;
  const int32_t* in_ci;
  const int32_t* deg;
  const uint64_t* omega;  // (1-alpha)/d in Q0.64
  const u64* y_in;        // shares pushed in this pass
  u64* y_out;             // shares of the next pass (threshold of this epoch)
  u64* r;                 // residue (in place)
  u64* pi;                // reserve (in place)
  u64 alpha64;            // alpha in Q0.64
  u64 rmax_raw;           // r'_max in Q1.63
  const int32_t* npieces;
  u64* heavy_acc;
  unsigned int* heavy_cnt;
  u64* rsum;              // [KT] residue sums after the pass (exact)
  u64* active;            // [KT] nodes that will push in the next pass
};

// finish row u: a node that pushed in this pass moves alpha r to its reserve
// and keeps nothing; r' = kept + incoming; decide the next pass's push
template <int KT>
__device__ __forceinline__ void epoch_epilogue(const EpochArgs& a, int u, int slot, const u64 (&acc)[Lay<KT>::V],
                                               u64 (&rs)[Lay<KT>::V], u64 (&act)[Lay<KT>::V]) {
  constexpr int V = Lay<KT>::V;
  const u64 om = __ldg(&a.omega[u]);
  const u64 thr = (u64)__ldg(&a.deg[u]) * a.rmax_raw;
  const size_t base = (size_t)u * KT + slot * V;
  u64 yo[V], ro[V], pn[V], rn[V], yn[V];
  ld_vec<V>(a.y_in + base, yo);
  ld_vec<V>(a.r + base, ro);
  ld_vec<V>(a.pi + base, pn);
#pragma unroll
  for (int q = 0; q < V; ++q) {
    const bool pushed = yo[q] != 0;
    if (pushed) pn[q] += __umul64hi(ro[q], a.alpha64);
    rn[q] = (pushed ? 0ull : ro[q]) + acc[q];
    const bool on = rn[q] > thr;
    yn[q] = on ? mulhi_round(rn[q], om) : 0ull;
    rs[q] += rn[q];
    act[q] += on ? 1ull : 0ull;
  }
  st_vec<V>(a.pi + base, pn);
  st_vec<V>(a.r + base, rn);
  st_vec<V>(a.y_out + base, yn);
}

template <int KT>
__global__ void __launch_bounds__(256, 6) epoch_sweep_kernel(EpochArgs a) {
  constexpr int V = Lay<KT>::V, L = Lay<KT>::L, EPW = Lay<KT>::EPW;
  const int lane = threadIdx.x & 31;
  const int slot = lane % L;
  u64 rs[V], act[V];
#pragma unroll
  for (int q = 0; q < V; ++q) rs[q] = act[q] = 0;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < a.n_items; it += nwarps) {
    const int4 w = __ldg(&a.items[it]);
    auto gather = [&](int e0, int e1, u64 (&acc)[V]) {
      for (int e = e0 + lane / L; e < e1; e += EPW) {
        u64 t[V];
        ld_vec<V>(a.y_in + (size_t)__ldg(&a.in_ci[e]) * KT + slot * V, t);
#pragma unroll
        for (int q = 0; q < V; ++q) acc[q] += t[q];
      }
#pragma unroll
      for (int off = L; off < 32; off <<= 1)
#pragma unroll
        for (int q = 0; q < V; ++q) acc[q] += __shfl_xor_sync(kFull, acc[q], off);
    };
    if (w.x == 0) {
      const int u = w.y;
      u64 acc[V] = {};
      gather(w.z, w.w, acc);
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
          u64 tot[V];
#pragma unroll
          for (int q = 0; q < V; ++q) tot[q] = atomicExch(&a.heavy_acc[(size_t)u * KT + slot * V + q], 0ull);
          epoch_epilogue<KT>(a, u, slot, tot, rs, act);
        }
        if (lane == 0) atomicExch(&a.heavy_cnt[u], 0u);
      }
    } else if (w.x == 1) {
      for (int u = w.y; u < w.z; ++u) {
        u64 acc[V] = {};
        gather(__ldg(&a.in_rp[u]), __ldg(&a.in_rp[u + 1]), acc);
        if (lane < L) epoch_epilogue<KT>(a, u, slot, acc, rs, act);
      }
    } else {
      for (int u = w.y + lane / L; u < w.z; u += 32 / L) {
        const int e1 = __ldg(&a.in_rp[u + 1]);
        u64 acc[V] = {};
        for (int e = __ldg(&a.in_rp[u]); e < e1; ++e) {
          u64 t[V];
          ld_vec<V>(a.y_in + (size_t)__ldg(&a.in_ci[e]) * KT + slot * V, t);
#pragma unroll
          for (int q = 0; q < V; ++q) acc[q] += t[q];
        }
        epoch_epilogue<KT>(a, u, slot, acc, rs, act);
      }
    }
  }
  __shared__ u64 sr[8][KT], sa[8][KT];
#pragma unroll
  for (int off = L; off < 32; off <<= 1)
#pragma unroll
    for (int q = 0; q < V; ++q) {
      rs[q] += __shfl_xor_sync(kFull, rs[q], off);
      act[q] += __shfl_xor_sync(kFull, act[q], off);
    }
  const int warp = threadIdx.x >> 5;
  if (lane < L)
#pragma unroll
    for (int q = 0; q < V; ++q) {
      sr[warp][lane * V + q] = rs[q];
      sa[warp][lane * V + q] = act[q];
    }
  __syncthreads();
  if (threadIdx.x < KT) {
    u64 s1 = 0, s2 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s1 += sr[w][threadIdx.x];
      s2 += sa[w][threadIdx.x];
    }
    atomicAdd(&a.rsum[threadIdx.x], s1);
    if (s2) atomicAdd(&a.active[threadIdx.x], s2);
  }
}

// y = (1-alpha) r / d for nodes above the (new) threshold, else 0; counts them
template <int KT>
__global__ void epoch_activate_kernel(int64_t n, const int32_t* __restrict__ deg, const uint64_t* __restrict__ omega,
                                      const u64* __restrict__ r, u64 rmax_raw, u64* __restrict__ y,
                                      u64* __restrict__ active) {
  u64 cnt = 0;
  const int64_t total = n * KT;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = i / KT;
    const bool on = r[i] > (u64)deg[u] * rmax_raw;
    y[i] = on ? mulhi_round(r[i], omega[u]) : 0ull;
    cnt += on;
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) cnt += __shfl_xor_sync(kFull, cnt, off);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&active[0], cnt);
}

}  // namespace ppr
