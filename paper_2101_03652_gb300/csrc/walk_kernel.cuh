// SpeedPPR walks (Algorithm 4, step 4) and the Philox-4x32-10 generator they
// draw from.  Walk w of source column c starts at the node whose range of the
// exclusive prefix sum of W_v (ascending original id) holds w; at step t it
// reads Philox-4x32-10 with key (seed_lo, seed_hi) and counter
// (w_lo, w_hi, t/2, source index): words 2(t%2) and 2(t%2)+1 decide stopping
// (stop iff word < floor(alpha 2^32)) and the move (out-neighbour number
// (word * d) >> 32).  An endpoint u adds one to count(u) and r(v)/W_v to
// pi_hat(u).
#pragma once
#include <cstdint>

namespace ppr {

typedef unsigned long long u64;
constexpr unsigned kAllLanes = 0xffffffffu;

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with the round constants 0xD2511F53 and 0xCD9E8D57,
// the key bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

struct WalkArgs {
  int64_t n;
  const int32_t* out_rp;
  const int32_t* out_ci;
  const int32_t* deg;
  const int32_t* new_of_old;
  const int64_t* offs;   // [KT][n+1] exclusive prefix sums of W_v (original order)
  const float* r;
  unsigned int* counts;  // [n][KT]
  double* est;           // [n][KT]
  u64* steps;            // [KT] total moves
  int* status;           // set to 1 when a walk exceeds max_steps
  uint32_t key0, key1;
  uint32_t stop_below;   // floor(alpha * 2^32)
  int32_t max_steps;
  int32_t col0;          // source index of the tile's first column
};

// Each thread runs kWalksPerThread consecutive walk ids, so the start node
// advances monotonically (one binary search per thread) and a warp waits for
// the longest of its threads' walk *sums* rather than of single walks.  The
// walks are taken kWalkLanes at a time, stepped in lockstep, so that their
// random loads (row pointers, then the column index) are in flight together.
// A thread merges consecutive endpoints at the same node before its atomics.
constexpr int kWalksPerThread = 16;
constexpr int kWalkLanes = 2;

template <int KT>
__global__ void __launch_bounds__(256, 6) walk_kernel(WalkArgs a) {
  const int c = blockIdx.y;
  const int64_t* offs = a.offs + (size_t)c * (a.n + 1);
  const int64_t total = offs[a.n];
  const int64_t w_begin = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kWalksPerThread;
  u64 moves = 0;
  if (w_begin < total) {
    const int64_t w_end = min(w_begin + (int64_t)kWalksPerThread, total);
    int64_t lo = 0, hi = a.n - 1;  // last o with offs[o] <= w_begin
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (offs[mid] <= w_begin) lo = mid; else hi = mid - 1;
    }
    int64_t o = lo;
    int32_t pend_u = -1;
    unsigned pend_n = 0;
    double pend_est = 0.0;
    bool failed = false;
    for (int64_t w0 = w_begin; w0 < w_end; w0 += kWalkLanes) {
      int32_t cur[kWalkLanes];
      double inc[kWalkLanes];
      int32_t t[kWalkLanes];
      bool live[kWalkLanes];
      uint4 words[kWalkLanes];
#pragma unroll
      for (int j = 0; j < kWalkLanes; ++j) {
        const int64_t w = w0 + j;
        live[j] = w < w_end;
        t[j] = 0;
        cur[j] = 0;
        inc[j] = 0.0;
        words[j] = make_uint4(0, 0, 0, 0);
        if (live[j]) {
          while (offs[o + 1] <= w) ++o;
          const int32_t v = a.new_of_old[o];
          const double rv = (double)a.r[(size_t)v * KT + c];
          inc[j] = rv / (double)(offs[o + 1] - offs[o]);
          cur[j] = v;
        }
      }
      bool any = true;
      while (any) {
        any = false;
#pragma unroll
        for (int j = 0; j < kWalkLanes; ++j) {
          if (!live[j]) continue;
          const int64_t w = w0 + j;
          if ((t[j] & 1) == 0)
            words[j] = philox4x32_10(make_uint4((uint32_t)w, (uint32_t)((u64)w >> 32), (uint32_t)(t[j] >> 1),
                                                (uint32_t)(a.col0 + c)),
                                     a.key0, a.key1);
          const uint32_t stopw = (t[j] & 1) ? words[j].z : words[j].x;
          if (stopw < a.stop_below) { live[j] = false; t[j] = -t[j] - 1; continue; }  // stopped: t < 0
          if (t[j] >= a.max_steps) { live[j] = false; failed = true; t[j] = -t[j] - 1; continue; }
          any = true;
        }
        // the moves of the walks still running, their loads issued together
        int32_t e0[kWalkLanes], d[kWalkLanes];
#pragma unroll
        for (int j = 0; j < kWalkLanes; ++j)
          if (live[j]) {
            e0[j] = __ldg(&a.out_rp[cur[j]]);
            d[j] = __ldg(&a.out_rp[cur[j] + 1]) - e0[j];
          }
#pragma unroll
        for (int j = 0; j < kWalkLanes; ++j)
          if (live[j]) {
            const uint32_t movew = (t[j] & 1) ? words[j].w : words[j].y;
            cur[j] = __ldg(&a.out_ci[e0[j] + (int32_t)__umulhi(movew, (uint32_t)d[j])]);
            ++t[j];
          }
      }
      // endpoints in walk-id order
#pragma unroll
      for (int j = 0; j < kWalkLanes; ++j) {
        if (w0 + j >= w_end) continue;
        moves += (u64)(-t[j] - 1);
        if (cur[j] != pend_u) {
          if (pend_n) {
            atomicAdd(&a.counts[(size_t)pend_u * KT + c], pend_n);
            atomicAdd(&a.est[(size_t)pend_u * KT + c], pend_est);
          }
          pend_u = cur[j];
          pend_n = 0;
          pend_est = 0.0;
        }
        pend_n += 1;
        pend_est += inc[j];
      }
    }
    if (pend_n) {
      atomicAdd(&a.counts[(size_t)pend_u * KT + c], pend_n);
      atomicAdd(&a.est[(size_t)pend_u * KT + c], pend_est);
    }
    if (failed) atomicExch(a.status, 1);
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) moves += __shfl_xor_sync(kAllLanes, moves, off);
  if ((threadIdx.x & 31) == 0 && moves) atomicAdd(&a.steps[c], moves);
}

}  // namespace ppr
