// FP32 correction pass of a 64-source tile with TMA row gathers for the rows
// with many in-edges (the same pass as refine_pass_kernel<64, float>: for
// every row u, e(u) = r(u) + sum over in-neighbours v of z_e(v), z_e = (1-alpha)
// e / d, Sec. 4.1 Eq. 7 applied to the error of the current estimate).
//
// The in-CSR rows are sorted by in-degree, so rows [0, u_h) (more than
// kLightMax in-edges; about 88 % of the edges of an R-MAT graph) occupy the
// edge range [0, h_edges).  That range is cut into chunks of kTmaChunk edges,
// dealt round-robin to the "TMA warps" of the grid.  A TMA warp streams its
// chunks in stages of 32 edges: the 32 gathered rows (256 B each) land in one
// of its two shared-memory slots through eight four-row tile::gather4 copies,
// while it sums the other slot row by row and finishes every row whose last
// edge it passes (epilogue operands loaded a row ahead).  A row cut by a chunk
// boundary is finished by whichever of its pieces arrives last (partial sums
// by atomics, as for the split rows of the work list).  The other warps of the
// block ("LSU warps") process the light rows' work items with vector loads,
// concurrently.
//
// Selected by PPR_FLAG_TMA_GATHER.  Measured on GB300 it loses to the default
// pass: a gather-only probe moves R-MAT scale-22 rows at 15.7 TB/s with
// per-warp four-row gathers (about 16 TB/s even for rows resident in L2, where
// per-lane loads reach 20 TB/s), while refine_pass_kernel already moves the
// heavy rows at about 15.5 TB/s; with two warps of each block fixed to the
// heavy rows this pass takes 0.54 ms against 0.33 ms at R-MAT scale 20 and
// 2.2 ms against 1.5 ms at scale 22.
#pragma once

#include "refine_kernel.cuh"
#include "tma.cuh"

namespace ppr {

constexpr int kTmaRows = 32;                           // gathered rows per stage
constexpr int kTmaChunk = 1024;                        // edges per chunk
constexpr int kTmaStagesPerChunk = kTmaChunk / kTmaRows;
constexpr int kTmaIdxAhead = 3;                        // column indices loaded this many stages early
constexpr int kTmaSlotFloats = kTmaRows * 64;          // one slot: 32 rows of 64 FP32 values
constexpr int kTmaBlockWarps = 8;

// shared-memory bytes of a block with NT TMA warps: two slots and two
// mbarriers per warp, plus room to align the slots to 1 KB
constexpr size_t tma_smem_bytes(int nt) { return (size_t)nt * (2 * kTmaSlotFloats * 4 + 2 * 8) + 1024; }

struct TmaArgs {
  CUtensorMap map;            // ze_in as a 2-D FP32 tensor {64, n}, rows of 256 B, box {64, 1}
  int32_t h_edges;            // edges of rows [0, u_h)
  int32_t u_h;                // first row with at most kLightMax in-edges
  int32_t n_chunks;           // ceil(h_edges / kTmaChunk)
  int32_t item0;              // first work item of the light rows
  const int4* chunks;         // per chunk: {row holding its first edge, that row's first edge, its end, 0}
  const int32_t* split_slot;  // per row < u_h: slot of a row that meets two or more chunks, else -1
  const int32_t* split_np;    // per slot: chunks the row meets
  float* split_acc;           // per slot: 64 partial sums (zero between passes)
  unsigned int* split_cnt;    // per slot: pieces arrived (zero between passes)
  unsigned int* status;       // kTmaWaitTimeout when a wait ran out
};

// epilogue operands of a row, two columns per lane
struct TmaRowOps {
  float2 r;   // r of the cycle
  float2 zo;  // the row's z_e before this pass (relaxation, measured sums)
  float d;    // out-degree
};

template <bool MEAS>
__device__ __forceinline__ TmaRowOps tma_row_ops(const RefArgs& a, int u, int lane) {
  TmaRowOps o;
  const size_t base = (size_t)u * 64 + 2 * lane;
  o.r = __ldg(reinterpret_cast<const float2*>(a.rf + base));
  const float2* zp = reinterpret_cast<const float2*>(static_cast<const float*>(a.ze_in) + base);
  if (MEAS) o.zo = __ldg(zp);                   // read-only buffer in the measured pass
  else if (a.relax != 1.f) o.zo = __ldcg(zp);   // in place: through L2
  else o.zo = make_float2(0.f, 0.f);
  o.d = (float)__ldg(&a.deg[u]);
  return o;
}

template <bool MEAS>
__device__ __forceinline__ void tma_row_epilogue(const RefArgs& a, int u, int lane, float2 sum, const TmaRowOps& o,
                                                 float2& res) {
  const float share = a.one_minus_alpha / o.d;
  const float2 e = make_float2(o.r.x + sum.x, o.r.y + sum.y);
  float2 zn = make_float2(e.x * share, e.y * share);
  if (a.relax != 1.f) {
    zn.x = o.zo.x + a.relax * (zn.x - o.zo.x);
    zn.y = o.zo.y + a.relax * (zn.y - o.zo.y);
  }
  if (MEAS) {
    const float inv = o.d / a.one_minus_alpha;
    res.x += fabsf(zn.x - o.zo.x) * inv;
    res.y += fabsf(zn.y - o.zo.y) * inv;
  }
  const size_t base = (size_t)u * 64 + 2 * lane;
  *reinterpret_cast<float2*>(static_cast<float*>(a.ze_out) + base) = zn;
  if (a.e_out) *reinterpret_cast<float2*>(a.e_out + base) = e;
}

// partial sum of a row cut by chunk boundaries; the last piece finishes it
template <bool MEAS>
__device__ __forceinline__ void tma_split_add(const RefArgs& a, const TmaArgs& t, int u, int lane, float2 part,
                                              const TmaRowOps& o, float2& res) {
  const int sl = __ldg(&t.split_slot[u]);
  float* acc = t.split_acc + (size_t)sl * 64 + 2 * lane;
  atomicAdd(acc, part.x);
  atomicAdd(acc + 1, part.y);
  __threadfence();
  __syncwarp();
  unsigned ticket = 0;
  if (lane == 0) ticket = atomicAdd(&t.split_cnt[sl], 1u);
  ticket = __shfl_sync(kFull, ticket, 0);
  if (ticket == (unsigned)__ldg(&t.split_np[sl]) - 1u) {
    __threadfence();
    float2 tot;
    tot.x = atomicExch(acc, 0.f);
    tot.y = atomicExch(acc + 1, 0.f);
    tma_row_epilogue<MEAS>(a, u, lane, tot, o, res);
    if (lane == 0) atomicExch(&t.split_cnt[sl], 0u);
  }
}

// first edge of stage s of TMA warp tw (of ntw), or INT_MAX past its last chunk
__device__ __forceinline__ int tma_stage_e0(const TmaArgs& t, int tw, int ntw, int s) {
  const int c = tw + (s / kTmaStagesPerChunk) * ntw;
  if (c >= t.n_chunks) return 0x7fffffff;
  return c * kTmaChunk + (s % kTmaStagesPerChunk) * kTmaRows;
}

// The TMA warp's part of the pass.  Returns false when a wait ran out (the
// status word is then set and no copy of this warp is left in flight).
template <bool MEAS>
__device__ __forceinline__ bool refine_tma_rows(const RefArgs& a, const TmaArgs& t, float* slots, uint64_t* bars,
                                                int tw, int ntw, int lane, float2& res) {
  const int H = t.h_edges;
  if (lane == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init_fence();
  }
  __syncwarp();
  auto ld_idx = [&](int s) -> int {
    const int e0 = tma_stage_e0(t, tw, ntw, s);
    return (e0 < H && lane < H - e0) ? __ldg(&a.in_ci[e0 + lane]) : -1;
  };
  // stage s: its rows into slot s & 1 (eight gather4 copies; a short last
  // stage repeats its last row, which is then not summed)
  auto issue = [&](int s, int idx) {
    const int e0 = tma_stage_e0(t, tw, ntw, s);
    if (e0 >= H) return;
    const int cnt = min(kTmaRows, H - e0);
    const int sl = s & 1;
    __syncwarp();
    fence_proxy_async_smem();
    const int ng = (cnt + 3) >> 2;
    if (lane == 0) mbar_expect_tx(&bars[sl], (unsigned)(ng * 4 * 64 * 4));
    __syncwarp();
    int y[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int src = 4 * (lane & 7) + h;
      y[h] = __shfl_sync(kFull, idx, src < cnt ? src : cnt - 1);
    }
    if (lane < ng) tma_gather4(slots + (size_t)sl * kTmaSlotFloats + lane * 4 * 64, &t.map, 0, y[0], y[1], y[2], y[3],
                               &bars[sl]);
  };

  issue(0, ld_idx(0));
  int idx[kTmaIdxAhead];
#pragma unroll
  for (int j = 0; j < kTmaIdxAhead; ++j) idx[j] = ld_idx(1 + j);
  int4 ndesc = tw < t.n_chunks ? __ldg(&t.chunks[tw]) : make_int4(0, 0, 0, 0);
  int u = 0, rs = 0, re = 0, nre = 0, c_e0 = 0, c_e1 = 0;
  float2 acc = make_float2(0.f, 0.f);
  TmaRowOps ops{};
  bool ok = true;
  int s = 0;
  for (;; ++s) {
    const int e0 = tma_stage_e0(t, tw, ntw, s);
    if (e0 >= H) break;
    issue(s + 1, idx[0]);
#pragma unroll
    for (int j = 0; j + 1 < kTmaIdxAhead; ++j) idx[j] = idx[j + 1];
    idx[kTmaIdxAhead - 1] = ld_idx(s + 1 + kTmaIdxAhead);
    const int cnt = min(kTmaRows, H - e0);
    if (s % kTmaStagesPerChunk == 0) {
      // a new chunk: its first row (which may have begun in an earlier chunk)
      const int4 d = ndesc;
      const int cn = tw + (s / kTmaStagesPerChunk + 1) * ntw;
      ndesc = cn < t.n_chunks ? __ldg(&t.chunks[cn]) : make_int4(0, 0, 0, 0);
      u = d.x;
      rs = d.y;
      re = d.z;
      nre = u + 1 < t.u_h ? __ldg(&a.in_rp[u + 2]) : 0;
      c_e0 = e0;
      c_e1 = min(e0 + kTmaChunk, H);
      ops = tma_row_ops<MEAS>(a, u, lane);
      acc = make_float2(0.f, 0.f);
    }
    ok = mbar_wait(&bars[s & 1], (unsigned)((s >> 1) & 1));
    if (!__all_sync(kFull, ok)) {
      ok = false;
      break;
    }
    const float* src = slots + (size_t)(s & 1) * kTmaSlotFloats + 2 * lane;
    int r = 0;
    while (r < cnt) {
      const int stop = min(cnt, re - e0);
#pragma unroll 4
      for (; r < stop; ++r) {
        const float2 x = *reinterpret_cast<const float2*>(src + r * 64);
        acc.x += x.x;
        acc.y += x.y;
      }
      if (e0 + r != re) break;  // the stage ends inside row u
      {
        // row u ends here
        if (rs < c_e0) tma_split_add<MEAS>(a, t, u, lane, acc, ops, res);
        else tma_row_epilogue<MEAS>(a, u, lane, acc, ops, res);
        ++u;
        rs = re;
        re = nre;
        if (u < t.u_h) {
          nre = u + 1 < t.u_h ? __ldg(&a.in_rp[u + 2]) : 0;
          ops = tma_row_ops<MEAS>(a, u, lane);
        }
        acc = make_float2(0.f, 0.f);
      }
    }
    // the chunk's last stage: a row that continues into a later chunk hands
    // over its partial sum
    if (e0 + cnt == c_e1 && u < t.u_h && rs < c_e1 && re > c_e1) tma_split_add<MEAS>(a, t, u, lane, acc, ops, res);
  }
  if (!ok) {
    // copies already issued land before the block may exit
    for (int q = s; q <= s + 1; ++q)
      if (tma_stage_e0(t, tw, ntw, q) < H) mbar_wait(&bars[q & 1], (unsigned)((q >> 1) & 1));
    if (lane == 0) atomicOr(t.status, kTmaWaitTimeout);
  }
  return ok;
}

// NT TMA warps and 8 - NT LSU warps per block.  MEAS: the measured
// (synchronous) pass of a batch, which also sums |e' - e| per column.
template <bool MEAS, int NT>
__global__ void __launch_bounds__(256, 6) refine_tma_kernel(const __grid_constant__ RefArgs a,
                                                            const __grid_constant__ TmaArgs t) {
  constexpr int KT = 64, V = RLay<KT, float>::V, L = RLay<KT, float>::L;
  extern __shared__ __align__(1024) unsigned char tma_smem_raw[];
  // TMA destinations must be 128-byte aligned: align the slots explicitly
  unsigned char* tma_smem = tma_smem_raw + ((1024u - (smem_addr(tma_smem_raw) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2 res_t = make_float2(0.f, 0.f);
  float res_l[V];
#pragma unroll
  for (int q = 0; q < V; ++q) res_l[q] = 0.f;
  if (warp < NT) {
    float* slots = reinterpret_cast<float*>(tma_smem) + (size_t)warp * 2 * kTmaSlotFloats;
    uint64_t* bars = reinterpret_cast<uint64_t*>(tma_smem + (size_t)NT * 2 * kTmaSlotFloats * 4) + 2 * warp;
    refine_tma_rows<MEAS>(a, t, slots, bars, blockIdx.x * NT + warp, gridDim.x * NT, lane, res_t);
  } else {
    const int slot = lane % L;
    const int nlw = gridDim.x * (kTmaBlockWarps - NT);
    for (int it = t.item0 + blockIdx.x * (kTmaBlockWarps - NT) + (warp - NT); it < a.n_items; it += nlw)
      refine_item<KT, float, MEAS>(a, __ldg(&a.items[it]), lane, slot, res_l);
  }
  if (!MEAS) return;
  __shared__ float sred[kTmaBlockWarps][KT];
  if (warp < NT) {
    sred[warp][2 * lane] = res_t.x;
    sred[warp][2 * lane + 1] = res_t.y;
  } else {
#pragma unroll
    for (int off = L; off < 32; off <<= 1)
#pragma unroll
      for (int q = 0; q < V; ++q) res_l[q] += __shfl_xor_sync(kFull, res_l[q], off);
    if (lane < L)
#pragma unroll
      for (int q = 0; q < V; ++q) sred[warp][lane * V + q] = res_l[q];
  }
  refine_resid_block<KT>(sred, a.resid);
}

}  // namespace ppr
