// Approximate SSPPR on the GPU: SpeedPPR (Algorithm 4).
//
// Step 1: W from Eq. 8 (natural logarithm), mu = 1/n unless given.
// Steps 2-3: Algorithm 4 runs PowerPush to lambda = m/W and then refines until
// no node is active w.r.t. r_max = 1/W.  Both steps are Forward Push with
// different orders of push operations, and the refinement's end state (no
// active node) implies the first step's (sum r <= m r_max = m/W).  Here the
// pushes run as synchronous sweeps over the in-CSR: every node with
// r(v) > d_v / W pushes at once (Eq. 7 restricted to the active set, Sec. 4.1),
// until no node is active.  State is FP32, one column per source of a tile.
// Step 4: for each v with r(v) > 0, W_v = ceil(r(v) W) alpha-random walks start
// at v; a walk ending at u adds r(v)/W_v to pi_hat(u).
//
// Random numbers: walk ids are the exclusive prefix sum of W_v over
// ascending original node id.  Walk w at step t uses Philox-4x32-10 with key
// (seed_lo, seed_hi) and counter (w_lo, w_hi, t/2, source index); words 2(t%2)
// and 2(t%2)+1 decide stopping (stop iff word < floor(alpha 2^32)) and the
// move (out-neighbour number (word * d) >> 32 in the caller's row order).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ppr_internal.cuh"
#include "f32_lanes.cuh"
#include "walk_kernel.cuh"

namespace ppr {

// ----------------------------------------------------------- push sweeps
struct ApxArgs {
  int32_t n_items;
  const int4* items;  // same work list layout as the high-precision sweeps
  const int32_t* in_rp;
  const int32_t* in_ci;
  const int32_t* deg;
  const float* y_in;  // (1-alpha) r / d of nodes pushing in this sweep, else 0
  float* y_out;
  float* r;           // residue (includes the part pushed in the next sweep)
  float* pi;          // reserve
  float alpha, one_minus_alpha, rmax;
  const int32_t* npieces;
  float* heavy_acc;
  unsigned int* heavy_cnt;
  u64* active;        // [KT] nodes active after this sweep
  double* rsum;       // [KT] sum of residues after this sweep
};

// finish row u: r' = kept residue + incoming; decide the next push
template <int KT>
__device__ __forceinline__ void apx_epilogue(const ApxArgs& a, int u, int slot, const float (&acc)[Lay32<KT>::V],
                                             unsigned (&act)[Lay32<KT>::V], float (&rs)[Lay32<KT>::V]) {
  constexpr int V = Lay32<KT>::V;
  const int d = __ldg(&a.deg[u]);
  const float thr = (float)d * a.rmax;
  const float share = a.one_minus_alpha / (float)d;
  const size_t base = (size_t)u * KT + slot * V;
#pragma unroll
  for (int q = 0; q < V; ++q) {
    const float keep = a.y_in[base + q] > 0.f ? 0.f : a.r[base + q];
    const float rn = keep + acc[q];
    const bool on = rn > thr;
    a.r[base + q] = rn;
    a.y_out[base + q] = on ? rn * share : 0.f;
    if (on) a.pi[base + q] += a.alpha * rn;
    act[q] += on ? 1u : 0u;
    rs[q] += rn;
  }
}

template <int KT>
__device__ __forceinline__ void apx_gather_warp(const ApxArgs& a, int e_begin, int e_end, int lane, int slot,
                                                float (&acc)[Lay32<KT>::V]) {
  constexpr int V = Lay32<KT>::V, L = Lay32<KT>::L, EPW = Lay32<KT>::EPW, UNR = 4;
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
        ldf<V>(a.y_in + (size_t)v[q] * KT + slot * V, t[q]);
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
__global__ void __launch_bounds__(256, 6) apx_sweep_kernel(ApxArgs a) {
  constexpr int V = Lay32<KT>::V, L = Lay32<KT>::L;
  const int lane = threadIdx.x & 31;
  const int slot = lane % L;
  unsigned act[V];
  float rs[V];
#pragma unroll
  for (int q = 0; q < V; ++q) { act[q] = 0; rs[q] = 0.f; }
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < a.n_items; it += nwarps) {
    const int4 w = __ldg(&a.items[it]);
    if (w.x == 0) {
      const int u = w.y;
      float acc[V] = {};
      apx_gather_warp<KT>(a, w.z, w.w, lane, slot, acc);
#pragma unroll
      for (int off = L; off < 32; off <<= 1)
#pragma unroll
        for (int q = 0; q < V; ++q) acc[q] += __shfl_xor_sync(kAllLanes, acc[q], off);
      if (lane < L)
#pragma unroll
        for (int q = 0; q < V; ++q) atomicAdd(&a.heavy_acc[(size_t)u * KT + slot * V + q], acc[q]);
      __threadfence();
      unsigned ticket = 0;
      if (lane == 0) ticket = atomicAdd(&a.heavy_cnt[u], 1u);
      ticket = __shfl_sync(kAllLanes, ticket, 0);
      if (ticket == (unsigned)a.npieces[u] - 1u) {
        __threadfence();
        if (lane < L) {
          float tot[V];
#pragma unroll
          for (int q = 0; q < V; ++q) tot[q] = atomicExch(&a.heavy_acc[(size_t)u * KT + slot * V + q], 0.f);
          apx_epilogue<KT>(a, u, slot, tot, act, rs);
        }
        if (lane == 0) atomicExch(&a.heavy_cnt[u], 0u);
      }
    } else if (w.x == 1) {
      for (int u = w.y; u < w.z; ++u) {
        float acc[V] = {};
        apx_gather_warp<KT>(a, __ldg(&a.in_rp[u]), __ldg(&a.in_rp[u + 1]), lane, slot, acc);
#pragma unroll
        for (int off = L; off < 32; off <<= 1)
#pragma unroll
          for (int q = 0; q < V; ++q) acc[q] += __shfl_xor_sync(kAllLanes, acc[q], off);
        if (lane < L) apx_epilogue<KT>(a, u, slot, acc, act, rs);
      }
    } else {
      for (int u = w.y + lane / L; u < w.z; u += 32 / L) {
        const int e1 = __ldg(&a.in_rp[u + 1]);
        float acc[V] = {};
#pragma unroll 4
        for (int e = __ldg(&a.in_rp[u]); e < e1; ++e) {
          float t[V];
          ldf<V>(a.y_in + (size_t)__ldg(&a.in_ci[e]) * KT + slot * V, t);
#pragma unroll
          for (int q = 0; q < V; ++q) acc[q] += t[q];
        }
        apx_epilogue<KT>(a, u, slot, acc, act, rs);
      }
    }
  }
  __shared__ unsigned sact[8][KT];
  __shared__ float srs[8][KT];
#pragma unroll
  for (int off = L; off < 32; off <<= 1)
#pragma unroll
    for (int q = 0; q < V; ++q) {
      act[q] += __shfl_xor_sync(kAllLanes, act[q], off);
      rs[q] += __shfl_xor_sync(kAllLanes, rs[q], off);
    }
  const int warp = threadIdx.x >> 5;
  if (lane < L)
#pragma unroll
    for (int q = 0; q < V; ++q) {
      sact[warp][lane * V + q] = act[q];
      srs[warp][lane * V + q] = rs[q];
    }
  __syncthreads();
  if (threadIdx.x < KT) {
    u64 ca = 0;
    double cs = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ca += sact[w][threadIdx.x];
      cs += (double)srs[w][threadIdx.x];
    }
    if (ca) atomicAdd(&a.active[threadIdx.x], ca);
    atomicAdd(&a.rsum[threadIdx.x], cs);
  }
}

// r = e_s, and s pushes in the first sweep
template <int KT>
__global__ void apx_init_kernel(const int32_t* __restrict__ src_new, int ncols, const int32_t* __restrict__ deg,
                                float alpha, float* r, float* y, float* pi) {
  const int c = threadIdx.x;
  if (c < ncols) {
    const int32_t s = src_new[c];
    const size_t i = (size_t)s * KT + c;
    r[i] = 1.f;
    y[i] = (1.f - alpha) / (float)deg[s];
    pi[i] = alpha;
  }
}

// ------------------------------------------------------------ walk phase
// cnt[c][o] = ceil(r(new(o)) * W) for r > 0 (IEEE double multiply, then ceil)
template <int KT>
__global__ void walk_count_kernel(int64_t n, const int32_t* __restrict__ new_of_old, const float* __restrict__ r,
                                  double W, int ncols, int64_t* __restrict__ cnt) {
  const int c = blockIdx.y;
  if (c >= ncols) return;
  int64_t* col = cnt + (size_t)c * (n + 1);
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    const float rv = r[(size_t)new_of_old[o] * KT + c];
    col[o] = rv > 0.f ? (int64_t)ceil(__dmul_rn((double)rv, W)) : 0;
  }
}

// exclusive prefix sum of each column of cnt (n values, then the total at [n])
constexpr int kScanItems = 8;
constexpr int kScanBlock = 256 * kScanItems;

__global__ void scan_block_kernel(int64_t n, int64_t* __restrict__ cnt, int64_t* __restrict__ block_sums,
                                  int64_t nblocks) {
  const int c = blockIdx.y;
  int64_t* col = cnt + (size_t)c * (n + 1);
  const int64_t b0 = (int64_t)blockIdx.x * kScanBlock;
  int64_t v[kScanItems];
  int64_t sum = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t o = b0 + threadIdx.x * kScanItems + i;
    v[i] = o < n ? col[o] : 0;
    sum += v[i];
  }
  // block-wide exclusive scan of the per-thread sums
  __shared__ int64_t warp_sums[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t incl = sum;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    int64_t t = __shfl_up_sync(kAllLanes, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  int64_t wbase = 0;
  for (int w = 0; w < warp; ++w) wbase += warp_sums[w];
  int64_t run = wbase + incl - sum;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t o = b0 + threadIdx.x * kScanItems + i;
    if (o < n) col[o] = run;
    run += v[i];
  }
  if (threadIdx.x == 255) block_sums[(size_t)c * nblocks + blockIdx.x] = wbase + incl;
}

__global__ void scan_sums_kernel(int64_t n, int64_t* __restrict__ cnt, int64_t* __restrict__ block_sums,
                                 int64_t nblocks) {
  // one block per column: sequential chunks of 256 block sums
  const int c = blockIdx.x;
  int64_t* bs = block_sums + (size_t)c * nblocks;
  __shared__ int64_t carry_s;
  __shared__ int64_t warp_sums[8];
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t b0 = 0; b0 < nblocks; b0 += 256) {
    const int64_t b = b0 + threadIdx.x;
    const int64_t v = b < nblocks ? bs[b] : 0;
    int64_t incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      int64_t t = __shfl_up_sync(kAllLanes, incl, off);
      if (lane >= off) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    int64_t wbase = 0, total = 0;
    for (int w = 0; w < 8; ++w) {
      if (w < warp) wbase += warp_sums[w];
      total += warp_sums[w];
    }
    const int64_t carry = carry_s;
    if (b < nblocks) bs[b] = carry + wbase + incl - v;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + total;
    __syncthreads();
  }
  if (threadIdx.x == 0) cnt[(size_t)c * (n + 1) + n] = carry_s;
}

__global__ void scan_add_kernel(int64_t n, int64_t* __restrict__ cnt, const int64_t* __restrict__ block_sums,
                                int64_t nblocks) {
  const int c = blockIdx.y;
  int64_t* col = cnt + (size_t)c * (n + 1);
  const int64_t add = block_sums[(size_t)c * nblocks + blockIdx.x];
  const int64_t b0 = (int64_t)blockIdx.x * kScanBlock;
  for (int i = threadIdx.x; i < kScanBlock; i += blockDim.x) {
    const int64_t o = b0 + i;
    if (o < n) col[o] += add;
  }
}


// out_pi = reserve + walk estimates; optional residue and counts (original ids)
template <int KT>
__global__ void apx_finish_kernel(int64_t n, const int32_t* __restrict__ new_of_old, const float* __restrict__ pi,
                                  const double* __restrict__ est, const float* __restrict__ r,
                                  const unsigned* __restrict__ counts, int ncols, int64_t col0,
                                  double* __restrict__ out_pi, double* __restrict__ out_r,
                                  uint32_t* __restrict__ out_counts) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    const size_t u = (size_t)new_of_old[o] * KT;
    for (int c = 0; c < ncols; ++c) {
      const size_t dst = (size_t)(col0 + c) * n + o;
      out_pi[dst] = (double)pi[u + c] + est[u + c];
      if (out_r) out_r[dst] = (double)r[u + c];
      if (out_counts) out_counts[dst] = counts[u + c];
    }
  }
}

// ------------------------------------------------------------ host engine
// a node with more than 32 index walks in a column goes to a block; at most
// m / 32 such nodes per column
inline size_t index_heavy_bytes(int64_t m, int kt) { return ((size_t)m * kt / 32 + 1024 + 8) * sizeof(u64); }

template <int KT>
ppr_status index_walk_phase(ppr_graph* g, const float* r, double W, int ncols, unsigned* counts, double* est,
                            u64* walks, cudaStream_t st);

template <int KT>
static ppr_status run_approx(ppr_graph* g, const int32_t* src, int32_t k, const ppr_query_opts& o, double* out_pi,
                             double* out_r, uint32_t* out_counts, ppr_stats* stats, cudaStream_t st) {
  const int64_t n = g->n, m = g->m;
  const double alpha = o.alpha;
  const double mu = o.mu > 0.0 ? o.mu : 1.0 / (double)n;
  const double eps = o.eps;
  const double W = 2.0 * (2.0 * eps / 3.0 + 2.0) * std::log((double)n) / (eps * eps * mu);
  const double rmax = 1.0 / W;
  Workspace& ws = g->ws;
  const size_t cells = (size_t)n * KT;
  const int max_sweeps = o.max_sweeps > 0 ? o.max_sweeps : 4096;
  const int32_t max_steps = 1 << 16;
  // outputs the kernels can write directly (device memory or pinned host
  // memory); the rest is staged on the device and copied at the end
  double* pi_view = static_cast<double*>(device_view(out_pi));
  double* r_view = out_r ? static_cast<double*>(device_view(out_r)) : nullptr;
  uint32_t* c_view = out_counts ? static_cast<uint32_t*>(device_view(out_counts)) : nullptr;
  const bool pi_host = pi_view == nullptr;
  const bool r_host = out_r && r_view == nullptr;
  const bool c_host = out_counts && c_view == nullptr;

  ppr_graph::SweepPlan* plan = nullptr;
  PPR_TRY(get_plan(g, Lay32<KT>::L, &plan, st));
  const int64_t nscan = (n + kScanBlock - 1) / kScanBlock;
  // workspace: r, pi, y_a, y_b (FP32), est (f64), counts (u32), offsets, scan sums, staging
  size_t stage = 0;
  if (pi_host) stage += (size_t)k * n * 8;
  if (r_host) stage += (size_t)k * n * 8;
  if (c_host) stage += (size_t)k * n * 4;
  const size_t walk_b_bytes = (o.flags & PPR_FLAG_INDEX) ? index_heavy_bytes(m, KT) : (size_t)KT * (n + 1) * 8;
  const size_t need = cells * 4 * 4 + cells * 8 + cells * 4 + walk_b_bytes + (size_t)KT * nscan * 8 +
                      (size_t)plan->n_split * KT * 4 + stage;
  {
    size_t free_b = 0, total_b = 0;
    PPR_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    free_b = admission_free_bytes(free_b);
    size_t have = ws.walk_a.bytes + ws.walk_b.bytes + ws.walk_c.bytes + ws.stage.bytes + ws.heavy_acc.bytes;
    if (need > free_b + have) {
      set_error("admission refused: approximate batch needs %zu bytes, %zu free", need, free_b);
      return PPR_ERR_ADMIT;
    }
  }
  PPR_TRY(ws.walk_a.ensure(cells * 4 * 4 + cells * 8 + cells * 4));  // r, pi, ya, yb | est | counts
  const bool use_index = (o.flags & PPR_FLAG_INDEX) != 0;
  if (use_index && (!g->d_index || g->index_alpha != alpha)) {
    set_error(g->d_index ? "the walk index was built for another alpha" : "PPR_FLAG_INDEX needs ppr_index_build first");
    return PPR_ERR_ARG;
  }
  // walk offsets, or the heavy (node, column) list of an index query
  PPR_TRY(ws.walk_b.ensure(walk_b_bytes));
  PPR_TRY(ws.walk_c.ensure((size_t)KT * nscan * 8 + 4096));          // scan sums, counters
  const size_t acc_bytes = std::max<size_t>((size_t)plan->n_split * KT * 4, 4);
  const size_t cnt_bytes = std::max<size_t>((size_t)plan->n_split * 4, 4);
  PPR_TRY(ws.heavy_acc.ensure(std::max(acc_bytes, ws.heavy_acc.bytes)));
  PPR_TRY(ws.heavy_cnt.ensure(std::max(cnt_bytes, ws.heavy_cnt.bytes)));
  if (ws.heavy_acc.fresh || ws.heavy_cnt.fresh) {
    PPR_CUDA_TRY(cudaMemsetAsync(ws.heavy_acc.ptr, 0, ws.heavy_acc.bytes, st));
    PPR_CUDA_TRY(cudaMemsetAsync(ws.heavy_cnt.ptr, 0, ws.heavy_cnt.bytes, st));
    ws.heavy_acc.fresh = ws.heavy_cnt.fresh = false;
  }
  if (stage) PPR_TRY(ws.stage.ensure(stage));
  PPR_TRY(ws.counters.ensure(8192));
  if (!ws.pinned) {
    PPR_CUDA_TRY(cudaMallocHost(&ws.pinned, 65536));
    ws.pinned_bytes = 65536;
  }
  float* r = ws.walk_a.as<float>();
  float* pi = r + cells;
  float* ya = pi + cells;
  float* yb = ya + cells;
  double* est = reinterpret_cast<double*>(yb + cells);
  unsigned* counts = reinterpret_cast<unsigned*>(est + cells);
  int64_t* offs = ws.walk_b.as<int64_t>();
  int64_t* bsums = ws.walk_c.as<int64_t>();
  u64* ctr = reinterpret_cast<u64*>(ws.walk_c.as<char>() + (size_t)KT * nscan * 8);  // [0,KT) active [KT,2KT) steps
  double* rsum_d = reinterpret_cast<double*>(ctr + 2 * KT);                           // [KT]
  int* status = reinterpret_cast<int*>(rsum_d + KT);
  int32_t* d_src = ws.counters.as<int32_t>() + 1024;
  u64* hpin = static_cast<u64*>(ws.pinned);
  double* stage_p = ws.stage.as<double>();
  double* pi_dev = pi_host ? stage_p : pi_view;
  double* r_dev = !out_r ? nullptr : (r_host ? stage_p + (pi_host ? (size_t)k * n : 0) : r_view);
  uint32_t* c_dev = !out_counts ? nullptr
                                : (c_host ? reinterpret_cast<uint32_t*>(stage_p + (pi_host ? (size_t)k * n : 0) +
                                                                        (r_host ? (size_t)k * n : 0))
                                          : c_view);
  PPR_TRY(ensure_alpha(g, alpha, st));
  int bps = 0;
  PPR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, apx_sweep_kernel<KT>, 256, 0));
  const int sweep_grid = sm_count() * std::max(bps, 1);
  const int grid_ew = sm_count() * 8;
  cudaEvent_t e0, e1, e2;
  PPR_CUDA_TRY(cudaEventCreate(&e0));
  PPR_CUDA_TRY(cudaEventCreate(&e1));
  PPR_CUDA_TRY(cudaEventCreate(&e2));
  float ms_push = 0.f, ms_walk = 0.f;
  int64_t launches = 0, sweep_launches = 0;
  ppr_status status_out = PPR_OK;

  for (int32_t t0 = 0; t0 < k && status_out == PPR_OK; t0 += KT) {
    const int ncols = std::min<int32_t>(KT, k - t0);
    int32_t src_new[64];
    for (int c = 0; c < 64; ++c) src_new[c] = c < ncols ? g->h_new_of_old[src[t0 + c]] : -1;
    PPR_CUDA_TRY(cudaEventRecord(e0, st));
    PPR_CUDA_TRY(cudaMemsetAsync(r, 0, cells * 4 * 4, st));
    PPR_CUDA_TRY(cudaMemsetAsync(est, 0, cells * 8 + cells * 4, st));
    PPR_CUDA_TRY(cudaMemcpyAsync(d_src, src_new, sizeof(src_new), cudaMemcpyHostToDevice, st));
    apx_init_kernel<KT><<<1, 64, 0, st>>>(d_src, ncols, g->d_deg, (float)alpha, r, ya, pi);
    ++launches;
    // ---- push sweeps until no node is active w.r.t. 1/W
    ApxArgs aa;
    aa.items = plan->d_items;
    aa.in_rp = g->d_in_rp;
    aa.in_ci = g->d_in_ci;
    aa.deg = g->d_deg;
    aa.r = r;
    aa.pi = pi;
    aa.alpha = (float)alpha;
    aa.one_minus_alpha = (float)(1.0 - alpha);
    aa.rmax = (float)rmax;
    aa.npieces = plan->d_npieces;
    aa.heavy_acc = ws.heavy_acc.as<float>();
    aa.heavy_cnt = ws.heavy_cnt.as<unsigned int>();
    aa.active = ctr;
    aa.rsum = rsum_d;
    int sweeps = 0;
    float* yin = ya;
    float* yout = yb;
    while (true) {
      if (sweeps >= max_sweeps) {
        set_error("push sweeps did not reach an inactive state within %d sweeps", max_sweeps);
        status_out = PPR_ERR_NOT_CONVERGED;
        break;
      }
      PPR_CUDA_TRY(cudaMemsetAsync(ctr, 0, 8 * KT, st));
      PPR_CUDA_TRY(cudaMemsetAsync(rsum_d, 0, 8 * KT, st));
      aa.y_in = yin;
      aa.y_out = yout;
      aa.n_items = plan->n_items_all;
      apx_sweep_kernel<KT><<<sweep_grid, 256, 0, st>>>(aa);
      ++launches;
      ++sweep_launches;
      ++sweeps;
      std::swap(yin, yout);
      PPR_CUDA_TRY(cudaGetLastError());
      PPR_CUDA_TRY(cudaMemcpyAsync(hpin, ctr, 8 * KT, cudaMemcpyDeviceToHost, st));
      PPR_CUDA_TRY(cudaStreamSynchronize(st));
      u64 act = 0;
      for (int c = 0; c < ncols; ++c) act += hpin[c];
      if (act == 0) break;
    }
    if (status_out != PPR_OK) break;
    PPR_CUDA_TRY(cudaEventRecord(e1, st));
    // ---- walks (from the index when one is built and requested)
    if (use_index) {
      PPR_TRY(index_walk_phase<KT>(g, r, W, ncols, counts, est, ctr, st));
      PPR_CUDA_TRY(cudaEventRecord(e2, st));
      apx_finish_kernel<KT><<<grid_ew, 256, 0, st>>>(n, g->d_new_of_old, pi, est, r, counts, ncols, t0, pi_dev, r_dev,
                                                     c_dev);
      launches += 3;
      PPR_CUDA_TRY(cudaGetLastError());
      PPR_CUDA_TRY(cudaMemcpyAsync(hpin, ctr, 8 * KT, cudaMemcpyDeviceToHost, st));
      PPR_CUDA_TRY(cudaStreamSynchronize(st));
      float a1 = 0.f, a2 = 0.f;
      cudaEventElapsedTime(&a1, e0, e1);
      cudaEventElapsedTime(&a2, e1, e2);
      ms_push += a1;
      ms_walk += a2;
      if (stats)
        for (int c = 0; c < ncols; ++c) {
          ppr_stats& sx = stats[t0 + c];
          memset(&sx, 0, sizeof(sx));
          sx.sweeps = sweeps;
          sx.edges_swept = (int64_t)sweeps * m;
          sx.walks = (int64_t)hpin[c];
          sx.W = W;
        }
    } else {
      dim3 gc(grid_ew, ncols);
      walk_count_kernel<KT><<<gc, 256, 0, st>>>(n, g->d_new_of_old, r, W, ncols, offs);
      dim3 gs((unsigned)nscan, ncols);
      scan_block_kernel<<<gs, 256, 0, st>>>(n, offs, bsums, nscan);
      scan_sums_kernel<<<ncols, 256, 0, st>>>(n, offs, bsums, nscan);
      scan_add_kernel<<<gs, 256, 0, st>>>(n, offs, bsums, nscan);
      launches += 4;
      PPR_CUDA_TRY(cudaGetLastError());
      for (int c = 0; c < ncols; ++c)
        PPR_CUDA_TRY(cudaMemcpyAsync(hpin + c, offs + (size_t)c * (n + 1) + n, 8, cudaMemcpyDeviceToHost, st));
      PPR_CUDA_TRY(cudaMemsetAsync(ctr + KT, 0, 8 * KT, st));
      PPR_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
      PPR_CUDA_TRY(cudaStreamSynchronize(st));
      int64_t maxw = 0;
      std::vector<int64_t> walks(ncols);
      for (int c = 0; c < ncols; ++c) {
        walks[c] = (int64_t)hpin[c];
        maxw = std::max(maxw, walks[c]);
      }
      if (maxw > 0) {
        WalkArgs wa;
        wa.n = n;
        wa.out_rp = g->d_out_rp;
        wa.out_ci = g->d_out_ci;
        wa.deg = g->d_deg;
        wa.new_of_old = g->d_new_of_old;
        wa.offs = offs;
        wa.r = r;
        wa.counts = counts;
        wa.est = est;
        wa.steps = ctr + KT;
        wa.status = status;
        wa.key0 = (uint32_t)o.seed;
        wa.key1 = (uint32_t)(o.seed >> 32);
        wa.stop_below = (uint32_t)std::floor(alpha * 4294967296.0);
        wa.max_steps = max_steps;
        wa.col0 = t0;
        dim3 gw((unsigned)((maxw + 256LL * kWalksPerThread - 1) / (256LL * kWalksPerThread)), ncols);
        walk_kernel<KT><<<gw, 256, 0, st>>>(wa);
        ++launches;
        PPR_CUDA_TRY(cudaGetLastError());
      }
      PPR_CUDA_TRY(cudaEventRecord(e2, st));
      apx_finish_kernel<KT><<<grid_ew, 256, 0, st>>>(n, g->d_new_of_old, pi, est, r, counts, ncols, t0, pi_dev, r_dev,
                                                     c_dev);
      ++launches;
      PPR_CUDA_TRY(cudaGetLastError());
      PPR_CUDA_TRY(cudaMemcpyAsync(hpin, ctr + KT, 8 * KT, cudaMemcpyDeviceToHost, st));
      PPR_CUDA_TRY(cudaMemcpyAsync(hpin + KT, status, sizeof(int), cudaMemcpyDeviceToHost, st));
      PPR_CUDA_TRY(cudaStreamSynchronize(st));
      if (*reinterpret_cast<int*>(hpin + KT) != 0) {
        set_error("a random walk exceeded %d steps", max_steps);
        status_out = PPR_ERR_NOT_CONVERGED;
        break;
      }
      float a1 = 0.f, a2 = 0.f;
      cudaEventElapsedTime(&a1, e0, e1);
      cudaEventElapsedTime(&a2, e1, e2);
      ms_push += a1;
      ms_walk += a2;
      if (stats)
        for (int c = 0; c < ncols; ++c) {
          ppr_stats& s = stats[t0 + c];
          memset(&s, 0, sizeof(s));
          s.sweeps = sweeps;
          s.edges_swept = (int64_t)sweeps * m;
          s.walks = walks[c];
          s.walk_steps = (int64_t)hpin[c];
          s.W = W;
        }
    }
  }
  if (status_out == PPR_OK) {
    if (pi_host) PPR_CUDA_TRY(cudaMemcpyAsync(out_pi, pi_dev, (size_t)k * n * 8, cudaMemcpyDeviceToHost, st));
    if (r_host) PPR_CUDA_TRY(cudaMemcpyAsync(out_r, r_dev, (size_t)k * n * 8, cudaMemcpyDeviceToHost, st));
    if (c_host) PPR_CUDA_TRY(cudaMemcpyAsync(out_counts, c_dev, (size_t)k * n * 4, cudaMemcpyDeviceToHost, st));
    PPR_CUDA_TRY(cudaStreamSynchronize(st));
    if (stats)
      for (int32_t i = 0; i < k; ++i) {
        stats[i].ms_push = ms_push;
        stats[i].ms_walk = ms_walk;
        stats[i].ms_total = ms_push + ms_walk;
        stats[i].kernel_launches = launches;
        stats[i].sweep_launches = sweep_launches;
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  return status_out;
}

ppr_status query_approx(ppr_graph* g, const int32_t* src, int32_t k, const ppr_query_opts& o, double* out_pi,
                        double* out_r, uint32_t* out_counts, ppr_stats* stats, cudaStream_t st) {
  int kt = o.k_tile;
  if (kt == 0) {
    kt = 1;
    while (kt < k && kt < 16) kt <<= 1;
  }
  if ((size_t)g->n * kt >= ((size_t)1 << 32)) {
    set_error("n * k_tile must stay below 2^32");
    return PPR_ERR_ARG;
  }
  switch (kt) {
    case 1: return run_approx<1>(g, src, k, o, out_pi, out_r, out_counts, stats, st);
    case 2: return run_approx<2>(g, src, k, o, out_pi, out_r, out_counts, stats, st);
    case 4: return run_approx<4>(g, src, k, o, out_pi, out_r, out_counts, stats, st);
    case 8: return run_approx<8>(g, src, k, o, out_pi, out_r, out_counts, stats, st);
    case 16: return run_approx<16>(g, src, k, o, out_pi, out_r, out_counts, stats, st);
    case 32: return run_approx<32>(g, src, k, o, out_pi, out_r, out_counts, stats, st);
    default: set_error("APPROX k_tile must be 0, 1, 2, 4, 8, 16 or 32"); return PPR_ERR_ARG;
  }
}

}  // namespace ppr

// ========================================================= SpeedPPR-Index
// SpeedPPR needs at most d_v walks from a node v (Sec. 6.2), so the endpoints
// of d_v walks per node -- m in all -- answer every eps.  The walk stored for
// out-edge slot e (the caller's CSR position of v's k-th out-edge) uses
// Philox-4x32-10 with counter (e_lo, e_hi, t/2, 0x1D3A); the endpoint is kept
// at the slot of the relabelled out-CSR that holds the same edge.
namespace ppr {

constexpr int kIndexSlotsPerThread = 16;

__global__ void __launch_bounds__(256) index_build_kernel(int64_t n, int64_t m, const int32_t* __restrict__ out_rp,
                                                          const int32_t* __restrict__ out_ci,
                                                          const int32_t* __restrict__ old_of_new,
                                                          const int64_t* __restrict__ rp_orig, uint32_t key0,
                                                          uint32_t key1, uint32_t stop_below, int32_t max_steps,
                                                          int32_t* __restrict__ index, int* status) {
  const int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kIndexSlotsPerThread;
  if (j0 >= m) return;
  const int64_t j1 = min(j0 + (int64_t)kIndexSlotsPerThread, m);
  int64_t lo = 0, hi = n - 1;  // node owning slot j0: last u with out_rp[u] <= j0
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (out_rp[mid] <= j0) lo = mid; else hi = mid - 1;
  }
  int64_t u = lo;
  for (int64_t j = j0; j < j1; ++j) {
    while (out_rp[u + 1] <= j) ++u;
    const int64_t e = rp_orig[old_of_new[u]] + (j - out_rp[u]);
    int32_t cur = (int32_t)u;
    uint4 words = make_uint4(0, 0, 0, 0);
    bool ok = true;
    for (int32_t t = 0;; ++t) {
      if ((t & 1) == 0)
        words = philox4x32_10(make_uint4((uint32_t)e, (uint32_t)((u64)e >> 32), (uint32_t)(t >> 1), 0x1D3Au), key0,
                              key1);
      if (((t & 1) ? words.z : words.x) < stop_below) break;
      if (t >= max_steps) { ok = false; break; }
      const int32_t e0 = __ldg(&out_rp[cur]);
      const int32_t d = __ldg(&out_rp[cur + 1]) - e0;
      cur = __ldg(&out_ci[e0 + (int32_t)__umulhi((t & 1) ? words.w : words.y, (uint32_t)d)]);
    }
    if (!ok) atomicExch(status, 1);
    index[j] = cur;
  }
}

// walk phase from the index: W_v = min(ceil(r(v) W), d_v) stored endpoints of v
template <int KT>
__global__ void __launch_bounds__(256) index_query_kernel(int64_t n, const int32_t* __restrict__ out_rp,
                                                          const int32_t* __restrict__ index,
                                                          const float* __restrict__ r, double W,
                                                          unsigned* __restrict__ counts, double* __restrict__ est,
                                                          u64* __restrict__ heavy, u64* __restrict__ n_heavy,
                                                          u64* __restrict__ walks) {
  const int c = blockIdx.y;
  u64 mine = 0;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const float rv = r[(size_t)u * KT + c];
    if (!(rv > 0.f)) continue;
    const int32_t e0 = out_rp[u];
    const int64_t d = out_rp[u + 1] - e0;
    const int64_t wv = min((int64_t)ceil(__dmul_rn((double)rv, W)), d);
    mine += (u64)wv;
    if (wv > 32) {
      heavy[atomicAdd(n_heavy, 1ull)] = ((u64)u << 6) | (u64)c;
      continue;
    }
    const double inc = (double)rv / (double)wv;
    for (int64_t k = 0; k < wv; ++k) {
      const int32_t t = __ldg(&index[e0 + k]);
      atomicAdd(&counts[(size_t)t * KT + c], 1u);
      atomicAdd(&est[(size_t)t * KT + c], inc);
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) mine += __shfl_xor_sync(kAllLanes, mine, off);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&walks[c], mine);
}

template <int KT>
__global__ void __launch_bounds__(256) index_query_heavy_kernel(const int32_t* __restrict__ out_rp,
                                                                const int32_t* __restrict__ index,
                                                                const float* __restrict__ r, double W,
                                                                const u64* __restrict__ heavy,
                                                                const u64* __restrict__ n_heavy,
                                                                unsigned* __restrict__ counts,
                                                                double* __restrict__ est) {
  const u64 nh = *n_heavy;
  for (u64 h = blockIdx.x; h < nh; h += gridDim.x) {
    const u64 rec = heavy[h];
    const int64_t u = (int64_t)(rec >> 6);
    const int c = (int)(rec & 63);
    const float rv = r[(size_t)u * KT + c];
    const int32_t e0 = out_rp[u];
    const int64_t d = out_rp[u + 1] - e0;
    const int64_t wv = min((int64_t)ceil(__dmul_rn((double)rv, W)), d);
    const double inc = (double)rv / (double)wv;
    for (int64_t k = threadIdx.x; k < wv; k += blockDim.x) {
      const int32_t t = __ldg(&index[e0 + k]);
      atomicAdd(&counts[(size_t)t * KT + c], 1u);
      atomicAdd(&est[(size_t)t * KT + c], inc);
    }
  }
}

template <int KT>
ppr_status index_walk_phase(ppr_graph* g, const float* r, double W, int ncols, unsigned* counts, double* est,
                            u64* walks, cudaStream_t st) {
  const int64_t n = g->n;
  if (g->ws.walk_b.bytes < index_heavy_bytes(g->m, KT)) {
    set_error("index query workspace too small");
    return PPR_ERR_ARG;
  }
  u64* nh = g->ws.walk_b.as<u64>();
  u64* heavy = nh + 8;
  PPR_CUDA_TRY(cudaMemsetAsync(nh, 0, sizeof(u64), st));
  PPR_CUDA_TRY(cudaMemsetAsync(walks, 0, sizeof(u64) * KT, st));
  const int grid = sm_count() * 8;
  index_query_kernel<KT><<<dim3(grid, ncols), 256, 0, st>>>(n, g->d_out_rp, g->d_index, r, W, counts, est, heavy, nh,
                                                            walks);
  index_query_heavy_kernel<KT><<<grid, 256, 0, st>>>(g->d_out_rp, g->d_index, r, W, heavy, nh, counts, est);
  PPR_CUDA_TRY(cudaGetLastError());
  return PPR_OK;
}

}  // namespace ppr

using namespace ppr;

extern "C" ppr_status ppr_index_build(ppr_graph* g, uint64_t seed, double alpha, void* cuda_stream) {
  clear_error();
  if (!g || !(alpha > 0.0 && alpha < 1.0)) {
    set_error("index_build needs a graph and alpha in (0, 1)");
    return PPR_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int64_t n = g->n, m = g->m;
  // the caller's row pointers (original order) from the stored out-degrees
  std::vector<int64_t> rp(n + 1, 0);
  for (int64_t v = 0; v < n; ++v) rp[v + 1] = rp[v] + g->h_out_deg[g->h_new_of_old[v]];
  int64_t* d_rp = nullptr;
  int* d_status = nullptr;
  PPR_CUDA_TRY(cudaMalloc(&d_rp, sizeof(int64_t) * (n + 1)));
  if (cudaMalloc(&d_status, sizeof(int)) != cudaSuccess) {
    cudaFree(d_rp);
    set_error("out of device memory");
    return PPR_ERR_OOM;
  }
  if (!g->d_index && cudaMalloc(&g->d_index, sizeof(int32_t) * std::max<int64_t>(m, 1)) != cudaSuccess) {
    g->d_index = nullptr;
    cudaFree(d_rp);
    cudaFree(d_status);
    set_error("out of device memory for the walk index (%lld bytes)", (long long)(4 * m));
    return PPR_ERR_OOM;
  }
  cudaMemcpyAsync(d_rp, rp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(d_status, 0, sizeof(int), st);
  const int64_t threads = (m + kIndexSlotsPerThread - 1) / kIndexSlotsPerThread;
  index_build_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      n, m, g->d_out_rp, g->d_out_ci, g->d_old_of_new, d_rp, (uint32_t)seed, (uint32_t)(seed >> 32),
      (uint32_t)std::floor(alpha * 4294967296.0), 1 << 16, g->d_index, d_status);
  int status = 0;
  cudaError_t e = cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_rp);
  cudaFree(d_status);
  PPR_CUDA_TRY(e);
  if (status) {
    set_error("an index walk exceeded 2^16 steps");
    return PPR_ERR_NOT_CONVERGED;
  }
  g->index_seed = seed;
  g->index_alpha = alpha;
  return PPR_OK;
}

extern "C" ppr_status ppr_index_get(const ppr_graph* g, int32_t* endpoints) {
  clear_error();
  if (!g || !endpoints) { set_error("graph and endpoints must be non-NULL"); return PPR_ERR_ARG; }
  if (!g->d_index) { set_error("no walk index built for this graph"); return PPR_ERR_ARG; }
  const int64_t n = g->n, m = g->m;
  std::vector<int32_t> idx(m), rp_new(n + 1, 0);
  PPR_CUDA_TRY(cudaMemcpy(idx.data(), g->d_index, sizeof(int32_t) * m, cudaMemcpyDeviceToHost));
  PPR_CUDA_TRY(cudaMemcpy(rp_new.data(), g->d_out_rp, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost));
  std::vector<int32_t> old_of_new(n);
  for (int64_t v = 0; v < n; ++v) old_of_new[g->h_new_of_old[v]] = (int32_t)v;
  int64_t e = 0;
  for (int64_t v = 0; v < n; ++v) {
    const int64_t u = g->h_new_of_old[v];
    for (int64_t j = rp_new[u]; j < rp_new[u + 1]; ++j) endpoints[e++] = old_of_new[idx[j]];
  }
  return PPR_OK;
}
