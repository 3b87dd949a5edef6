// High-precision SSPPR on the GPU: Algorithm 3 (PowerPush) restated for GB300.
//
// State.  Residues, reserves and estimates are unsigned Q1.63 fixed point
// (value = raw * 2^-63) in 64-bit integers.  Sums are then exact and
// independent of the order in which threads add, mass is conserved bit for
// bit by every push, and no FP64 arithmetic runs per edge (GB300's FP64 rate
// is a small fraction of its integer rate).  Resolution is 1.1e-19 per value,
// far below the l1 targets (>= 1e-12) the library accepts.
//
// Queue phase (Algorithm 3, first loop; Algorithm 2's iterations S^(j)).
// A frontier holds (node, column) pairs; one warp pushes one pair: it takes
// the residue with an atomic exchange (asynchronous pushes, Sec. 5), credits
// alpha*rho to the reserve and scatters (1-alpha)*rho/d_v to the out-neighbours
// with 64-bit integer atomics (the division remainder goes one unit at a time
// to the first neighbours, so no mass is lost).  A neighbour whose residue
// crosses d_u * r_max joins the next level; a per-level stamp plays the role of
// "u not in Q", and the warp appends its new entries with one atomic (ballot +
// popcount + prefix).  The phase ends when every column has sum(r) <= lambda,
// the frontier empties, or a level's out-edges exceed the switch threshold
// (the GPU counterpart of |Q| > scanThreshold).
//
// Sweep phase (Algorithm 3, epochs of full scans).  A full pass that pushes
// every node at once is SimFwdPush (Sec. 4.1, Eq. 7), equal to PowItr by
// Lemma 1.  It is run in the estimate form x <- alpha e_s + (1-alpha) x P:
// with x0 = reserve + alpha*residue the k-th pass equals k simultaneous pushes,
// and ||x_{j+1} - x_j||_1 / alpha is the l1 norm of the residue of x_j.  Each
// pass stores z = (1-alpha) x / d so that a row u of the in-CSR only sums the
// z of its in-neighbours (a gather, no per-edge multiply).  Because the
// residue contracts by (1-alpha) per pass, the number of passes to reach
// lambda is predicted and launched without per-pass host round trips; the
// last pass's measured residue certifies the result.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <vector>

#include "ppr_internal.cuh"
#include "sweep_kernel.cuh"
#include "epoch_kernel.cuh"
#include "refine_kernel.cuh"
#include "refine_tma_kernel.cuh"

#include <cudaTypedefs.h>

namespace ppr {

// ------------------------------------------------------------ queue phase
struct PushArgs {
  const uint32_t* front;
  uint32_t n_front;
  const int32_t* out_rp;
  const int32_t* out_ci;
  const int32_t* deg;
  u64* r;
  u64* pi;
  uint32_t* stamp;
  uint32_t next_stamp;
  uint32_t* next_front;
  u64* ent_share;   // per frontier entry: (1-alpha) rho / d (floor)
  uint32_t* ent_rem; // per frontier entry: remainder of that division
  u64* chunks;      // (entry << 32 | first edge) records, kPushChunk edges each
  u64* counters;    // [0] next size, [1] next out-edges, [2] chunks, [3+c] stopped mass,
                    // [3+KT+c] edges pushed
  u64 alpha64;      // alpha * 2^64
  u64 rmax_raw;     // r_max in Q1.63 units
};
constexpr int kPushChunk = 256;

// Phase A: one thread per frontier entry takes the residue (atomic exchange,
// so pushes landing meanwhile are not lost), credits alpha*rho to the reserve
// and emits one chunk record per kPushChunk out-edges.
template <int KT>
__global__ void __launch_bounds__(256) push_take_kernel(PushArgs a) {
  const int lane = threadIdx.x & 31;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < a.n_front; i0 += gridDim.x * blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    uint32_t nch = 0;
    if (i < a.n_front) {
      const uint32_t idx = a.front[i];
      const uint32_t v = idx / KT;
      const int c = idx % KT;
      const int32_t d = __ldg(&a.deg[v]);
      u64 rho = 0;
      u64 cur = *(volatile u64*)&a.r[idx];
      if (cur > (u64)d * a.rmax_raw) rho = atomicExch(&a.r[idx], 0ull);
      if (rho) {
        const u64 stop = __umul64hi(rho, a.alpha64);  // alpha * rho
        const u64 rest = rho - stop;                  // (1 - alpha) * rho, exact complement
        const u64 share = rest / (u64)d;
        a.ent_share[i] = share;
        a.ent_rem[i] = (uint32_t)(rest - share * (u64)d);
        a.pi[idx] += stop;
        atomicAdd(&a.counters[3 + c], stop);
        atomicAdd(&a.counters[3 + KT + c], (u64)d);
        nch = (uint32_t)((d + kPushChunk - 1) / kPushChunk);
      }
    }
    // warp-aggregated append of the chunk records
    uint32_t incl = nch;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t t = __shfl_up_sync(kFull, incl, off);
      if (lane >= off) incl += t;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    u64 base = 0;
    if (lane == 31 && total) base = atomicAdd(&a.counters[2], (u64)total);
    base = __shfl_sync(kFull, base, 31);
    for (uint32_t q = 0; q < nch; ++q)
      a.chunks[base + incl - nch + q] = ((u64)i << 32) | (u64)(q * kPushChunk);
  }
}

// Phase B: one warp per chunk scatters (1-alpha) rho / d to up to kPushChunk
// out-neighbours (the first `rem` neighbours of the row get one extra unit, so
// the push conserves mass exactly).  A neighbour whose residue crosses
// d_u * r_max joins the next frontier once per level (stamp), appended with
// one atomic per warp (ballot + popcount + prefix).
template <int KT>
__global__ void __launch_bounds__(256) push_scatter_kernel(PushArgs a) {
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const u64 nchunks = *(volatile u64*)&a.counters[2];
  for (u64 ch = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; ch < nchunks; ch += nwarps) {
    const u64 rec = a.chunks[ch];
    const uint32_t i = (uint32_t)(rec >> 32);
    const int32_t j0 = (int32_t)(rec & 0xffffffffu);
    const uint32_t idx = a.front[i];
    const uint32_t v = idx / KT;
    const int c = idx % KT;
    const int32_t e0 = __ldg(&a.out_rp[v]);
    const int32_t d = __ldg(&a.deg[v]);
    const u64 share = a.ent_share[i];
    const uint32_t rem = a.ent_rem[i];
    const int32_t j1 = min(d, j0 + kPushChunk);
    for (int32_t base = j0; base < j1; base += 32) {
      const int32_t j = base + lane;
      bool app = false;
      uint32_t uidx = 0;
      int32_t du = 0;
      if (j < j1) {
        const int32_t u = __ldg(&a.out_ci[e0 + j]);
        const u64 add = share + ((uint32_t)j < rem ? 1ull : 0ull);
        uidx = (uint32_t)u * KT + c;
        if (add) {
          const u64 old = atomicAdd(&a.r[uidx], add);
          du = __ldg(&a.deg[u]);
          const u64 thr = (u64)du * a.rmax_raw;
          if (old + add > thr && old <= thr) app = atomicExch(&a.stamp[uidx], a.next_stamp) != a.next_stamp;
        }
      }
      const unsigned mask = __ballot_sync(kFull, app);
      if (mask) {
        u64 esum = app ? (u64)du : 0ull;
#pragma unroll
        for (int off = 16; off; off >>= 1) esum += __shfl_xor_sync(kFull, esum, off);
        u64 pos0 = 0;
        if (lane == 0) {
          pos0 = atomicAdd(&a.counters[0], (u64)__popc(mask));
          atomicAdd(&a.counters[1], esum);
        }
        pos0 = __shfl_sync(kFull, pos0, 0);
        if (app) a.next_front[pos0 + __popc(mask & ((1u << lane) - 1u))] = uidx;
      }
    }
  }
}

template <int KT>
__global__ void init_sources_kernel(const int32_t* __restrict__ src_new, int ncols, u64* r, uint32_t* stamp,
                                    uint32_t epoch, uint32_t* front) {
  int c = threadIdx.x;
  if (c < ncols) {
    uint32_t idx = (uint32_t)src_new[c] * KT + c;
    r[idx] = kFixOneRaw;
    stamp[idx] = epoch;
    front[c] = idx;
  }
}

// x0 = reserve + alpha * residue; z0 = (1-alpha) x0 / d
template <int KT>
__global__ void convert_kernel(int64_t n, const u64* __restrict__ r, const u64* __restrict__ pi,
                               const uint64_t* __restrict__ omega, u64 alpha64, u64* __restrict__ z) {
  const int64_t total = n * KT;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    u64 x0 = pi[i] + __umul64hi(r[i], alpha64);
    z[i] = mulhi_round(x0, omega[i / KT]);
  }
}

// out[(col0 + c) * n + o] = x[new(o)][c] as float64.  A block takes 32
// consecutive output nodes at a time: their tile rows are read whole
// (consecutive columns to consecutive threads) into shared memory, then each
// column is written as 32 consecutive values.  Reading row by row per thread
// instead (one node per thread) took 0.47 against 0.28 ms for a 64-column
// R-MAT-20 tile into device memory; into page-locked host memory both run at
// the link's 192 GB/s.
template <int KT>
__global__ void __launch_bounds__(256) output_kernel(int64_t n, const int32_t* __restrict__ new_of_old,
                                                     const u64* __restrict__ x, int ncols, int64_t col0,
                                                     double* __restrict__ out) {
  constexpr int NB = 32;
  __shared__ double tile[KT][NB + 1];
  __shared__ int64_t rows[NB];
  for (int64_t o0 = (int64_t)blockIdx.x * NB; o0 < n; o0 += (int64_t)gridDim.x * NB) {
    const int cnt = n - o0 < NB ? (int)(n - o0) : NB;
    if (threadIdx.x < NB) rows[threadIdx.x] = threadIdx.x < cnt ? __ldg(&new_of_old[o0 + threadIdx.x]) : 0;
    __syncthreads();
    for (int i = threadIdx.x; i < NB * KT; i += blockDim.x) {
      const int j = i / KT, c = i % KT;
      if (j < cnt) tile[c][j] = u64_to_f64<-63>(__ldg(&x[rows[j] * KT + c]));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ncols * NB; i += blockDim.x) {
      const int c = i / NB, j = i % NB;
      if (j < cnt) out[(col0 + c) * n + o0 + j] = tile[c][j];
    }
    __syncthreads();
  }
}

// exact per-column sums of a tile (integer adds; the block size is a multiple
// of KT, so each thread always reads the same column)
template <int KT>
__global__ void column_sum_kernel(int64_t n, const u64* __restrict__ x, u64* __restrict__ mass) {
  __shared__ u64 part[KT];
  if (threadIdx.x < KT) part[threadIdx.x] = 0;
  __syncthreads();
  u64 acc = 0;
  const int64_t total = n * KT;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    acc += x[i];
  atomicAdd(&part[threadIdx.x % KT], acc);
  __syncthreads();
  if (threadIdx.x < KT) atomicAdd(&mass[threadIdx.x], part[threadIdx.x]);
}

// push residual of the returned estimate: r = (alpha e_s + sum z(v) - x(u)) / alpha
template <int KT>
__global__ void residual_kernel(int32_t n, const int32_t* __restrict__ in_rp, const int32_t* __restrict__ in_ci,
                                const int32_t* __restrict__ old_of_new, const u64* __restrict__ z,
                                const u64* __restrict__ x, SweepArgs a, int ncols, int64_t col0, double alpha,
                                double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
    for (int c = 0; c < ncols; ++c) {
      u64 acc = 0;
      for (int e = in_rp[u] + lane; e < in_rp[u + 1]; e += 32) acc += z[(size_t)in_ci[e] * KT + c];
#pragma unroll
      for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
      if (lane == 0) {
        u64 xn = acc + (u == a.src[c] ? a.alpha_raw : 0ull);
        long long diff = (long long)(xn - x[(size_t)u * KT + c]);
        out[(col0 + c) * (int64_t)n + old_of_new[u]] = (double)diff * (1.0 / kFixOne) / alpha;
      }
    }
  }
}

// ------------------------------------------------------------ host engine
int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 1;
  }
  return cached;
}

// Work list of one pass for a tile width.  Costs are counted in "periods":
// one round of UNR dependent gathers by a warp (or by a lane group for light
// rows).  Rows longer than one piece are split into pieces; other rows are
// grouped so that every item costs about kItemPeriods periods.  Items are
// ordered split pieces, medium rows, light rows, rows without in-edges.
using Plan = ppr_graph::SweepPlan;

static ppr_status build_plan(ppr_graph* g, int kt, Plan& p, cudaStream_t st);

// work list for `lanes` lanes per row slice (shared with the FP32 sweeps)
ppr_status get_plan(ppr_graph* g, int lanes, ppr_graph::SweepPlan** out, cudaStream_t st) {
  int slot = 0;
  while ((1 << slot) < lanes) ++slot;
  if (slot > 5) { set_error("too many lanes per row"); return PPR_ERR_ARG; }
  Plan& p = g->plans[slot + 1];
  const int kt = lanes * 2;
  if (p.kt != kt) PPR_TRY(build_plan(g, kt, p, st));
  *out = &p;
  return PPR_OK;
}

// Rows longer than this many in-edges are cut into pieces of it: the item
// cost in edges, at least 256 (wide tiles: keep split rows few).  Shorter
// items on small graphs (down to 32 edges, so that every resident warp gets
// about two items) shortened the FP32 pass of a 10,000-node graph from 14.8
// to 8.4 us, but the updates, almost all concurrent, then behave like
// synchronous ones: 69 instead of 50 passes, and with over-relaxation some
// queries stalled until the refinement gave up.  Items keep the full cost.
static int plan_piece_edges(int L) { return std::max(kItemPeriods * (32 / L) * kUnr, 256); }

static ppr_status build_plan(ppr_graph* g, int kt, Plan& p, cudaStream_t st) {
  const std::vector<int32_t>& d = g->h_in_deg_sorted;
  const int32_t n = (int32_t)g->n;
  const int L = kt >= 2 ? kt / 2 : 1;
  const int epw = 32 / L;                 // edges per warp step
  const int piece = plan_piece_edges(L);
  const int rpw = 32 / L;                 // light rows per warp
  std::vector<int4> items;
  std::vector<int32_t> npieces;
  int64_t e = 0;
  int32_t u = 0;
  for (; u < n && d[u] > piece; ++u) {
    int np = 0;
    for (int64_t b = e; b < e + d[u]; b += piece, ++np)
      items.push_back(make_int4(0, u, (int)b, (int)std::min<int64_t>(b + piece, e + d[u])));
    npieces.push_back(np);
    e += d[u];
  }
  const int32_t n_split = u;
  while (u < n && d[u] > kLightMax) {
    int32_t u0 = u;
    int cost = 0;
    while (u < n && d[u] > kLightMax) {
      int c = (d[u] + epw * kUnr - 1) / (epw * kUnr) + 1;
      if (cost > 0 && cost + c > kItemPeriods) break;
      cost += c;
      ++u;
    }
    items.push_back(make_int4(1, u0, u, 0));
  }
  p.n_items_heavy = (int32_t)items.size();
  p.u_light = u;
  while (u < n && d[u] > 0) {
    int32_t u0 = u;
    int cost = 0;
    while (u < n && d[u] > 0) {
      int c = (d[u] + kUnr - 1) / kUnr + 1;  // the block's first row is its longest
      if (cost > 0 && cost + c > kItemPeriods) break;
      cost += c;
      for (int r = 0; r < rpw && u < n && d[u] > 0; ++r) ++u;
    }
    items.push_back(make_int4(2, u0, u, 0));
  }
  p.n_items_nz = (int32_t)items.size();
  while (u < n) {
    int32_t u0 = u;
    u = (int32_t)std::min<int64_t>(n, (int64_t)u + (int64_t)kItemPeriods * rpw);
    items.push_back(make_int4(2, u0, u, 0));
  }
  p.n_items_all = (int32_t)items.size();
  p.n_split = n_split;
  p.kt = kt;
  PPR_CUDA_TRY(cudaMalloc((void**)&p.d_items, sizeof(int4) * std::max<size_t>(items.size(), 1)));
  PPR_CUDA_TRY(cudaMemcpyAsync(p.d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, st));
  PPR_CUDA_TRY(cudaMalloc((void**)&p.d_npieces, sizeof(int32_t) * std::max<size_t>(npieces.size(), 1)));
  PPR_CUDA_TRY(cudaMemcpyAsync(p.d_npieces, npieces.data(), sizeof(int32_t) * npieces.size(),
                               cudaMemcpyHostToDevice, st));
  PPR_CUDA_TRY(cudaStreamSynchronize(st));
  return PPR_OK;
}

template <int KT>
static void launch_sweep(const SweepArgs& a, int grid, cudaStream_t st) {
  if (a.z_out == a.z_in) sweep_kernel<KT, true><<<grid, 256, 0, st>>>(a);
  else sweep_kernel<KT, false><<<grid, 256, 0, st>>>(a);
}

// Algorithm 3's epochs from the push state (r, pi): epoch i pushes, in full
// synchronous passes, every node with r(v) > d_v lambda^(i/E) / m until the
// residue sum is at most lambda^(i/E) or no node is active.
template <int KT>
static ppr_status run_epochs(ppr_graph* g, const ppr_graph::SweepPlan& plan, int grid, int grid_ew, int E,
                             bool until_inactive, double lambda, double alpha, int max_sweeps, int ncols, u64* r,
                             u64* pi, u64* ya, u64* yb, u64* ctr, u64* hpin, int& sweeps, std::vector<double>& rsum,
                             int64_t& launches, float& ms_sweep, cudaEvent_t e0, cudaEvent_t e1, cudaStream_t st) {
  const int64_t n = g->n, m = g->m;
  EpochArgs ea;
  ea.items = plan.d_items;
  ea.n_items = plan.n_items_all;
  ea.in_rp = g->d_in_rp;
  ea.in_ci = g->d_in_ci;
  ea.deg = g->d_deg;
  ea.omega = g->d_omega;
  ea.r = r;
  ea.pi = pi;
  ea.alpha64 = (u64)(alpha * 18446744073709551616.0);
  ea.npieces = plan.d_npieces;
  ea.heavy_acc = g->ws.heavy_acc.as<u64>();
  ea.heavy_cnt = g->ws.heavy_cnt.as<unsigned int>();
  ea.rsum = ctr;
  ea.active = ctr + 64;
  auto max_rsum = [&]() {
    double mx = 0.0;
    for (int c = 0; c < ncols; ++c) mx = std::max(mx, rsum[c]);
    return mx;
  };
  // epochs 1..E; with until_inactive one more round at r_max = lambda/m that
  // ends only when no node is active (it cannot end on the residue sum)
  for (int i = 1; i <= E + (until_inactive ? 1 : 0); ++i) {
    const bool last = i > E;
    const double thr = std::pow(lambda, (double)std::min(i, E) / (double)E);  // m r'_max
    const u64 rmax_raw = (u64)std::max(1.0, std::floor(thr / (double)m * kFixOne));
    if (!last && max_rsum() <= thr) continue;
    PPR_CUDA_TRY(cudaMemsetAsync(ctr + 64, 0, 8, st));
    epoch_activate_kernel<KT><<<grid_ew, 256, 0, st>>>(n, g->d_deg, g->d_omega, r, rmax_raw, ya, ctr + 64);
    ++launches;
    PPR_CUDA_TRY(cudaMemcpyAsync(hpin, ctr + 64, 8, cudaMemcpyDeviceToHost, st));
    PPR_CUDA_TRY(cudaStreamSynchronize(st));
    if (hpin[0] == 0) continue;  // a pass would push nothing: the epoch ends
    ea.rmax_raw = rmax_raw;
    while (true) {
      if (sweeps >= max_sweeps) {
        set_error("sweep limit %d reached in the epochs", max_sweeps);
        return PPR_ERR_NOT_CONVERGED;
      }
      PPR_CUDA_TRY(cudaMemsetAsync(ctr, 0, 8 * 128, st));
      ea.y_in = ya;
      ea.y_out = yb;
      PPR_CUDA_TRY(cudaEventRecord(e0, st));
      epoch_sweep_kernel<KT><<<grid, 256, 0, st>>>(ea);
      PPR_CUDA_TRY(cudaEventRecord(e1, st));
      PPR_CUDA_TRY(cudaGetLastError());
      ++launches;
      ++sweeps;
      std::swap(ya, yb);
      PPR_CUDA_TRY(cudaMemcpyAsync(hpin, ctr, 8 * 128, cudaMemcpyDeviceToHost, st));
      PPR_CUDA_TRY(cudaStreamSynchronize(st));
      float a = 0.f;
      cudaEventElapsedTime(&a, e0, e1);
      ms_sweep += a;
      u64 act = 0;
      for (int c = 0; c < ncols; ++c) {
        rsum[c] = (double)hpin[c] / kFixOne;
        act += hpin[64 + c];
      }
      if ((!last && max_rsum() <= thr) || act == 0) break;
    }
  }
  return PPR_OK;
}

// State of one tile's sweep phase handed to the refinement driver.
struct RefineTile {
  int ncols;
  double alpha, lambda;
  int max_sweeps;
  bool have_state;           // (r, pi) hold a push state; else r = e_s, pi = 0
  std::vector<double> rsum;  // residue sums of the push state
  // learned estimate: with correction_passes L = 0 it replaces the start (X =
  // the model's estimate, first measured by an exact pass); with L > 0 the
  // remaining mass is added as mu q after the first L FP32 passes
  const void* model = nullptr;
  int corr = 0;
  const int32_t* src_new = nullptr;
  u64* mass = nullptr;       // [KT] device scratch for exact column sums
  bool fp32_only = false;    // no BF16 stage
  bool tma_gather = false;   // 64-source FP32 passes with TMA gathers of the heavy rows
  float relax = 1.15f;       // over-relaxation factor of the in-place correction passes
};

constexpr float kRelax = 1.15f;  // over-relaxation of in-place correction passes

// Sweep phase with correction passes (see refine_kernel.cuh).  Buffers:
// pi = X (Q1.63 base); r = the push residue, then e of the correction passes,
// then X' of the exact pass; zb = [r_f f32 | z_e]; za = the second z_e buffer,
// then z(X) for the exact pass.  Each cycle runs BF16 passes while they
// contract (down to about 1e-2 of the cycle's start), then FP32 passes (down
// to about 1e-6), folds e into X and runs one exact synchronous pass, which
// certifies the stop: ||pi - X'||_1 <= (1-alpha) ||X' - X||_1 / alpha.  The
// answer is X' (in r).
struct RefineOut {
  int passes[2] = {0, 0};    // BF16, FP32 correction passes
  float ms[2] = {0.f, 0.f};  // their device time
  int cycles = 0;
  float relax = 1.f;         // over-relaxation in effect at the end (1 after a fallback)
};

template <int KT, typename T>
static ppr_status refine_kernel_setup(ppr_graph* g, Plan** plan, int* grid, int* grid_meas, cudaStream_t st) {
  PPR_TRY(get_plan(g, RLay<KT, T>::L, plan, st));
  int bps = 0;
  PPR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, refine_pass_kernel<KT, T, false>, 256, 0));
  *grid = sm_count() * std::max(bps, 1);
  PPR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, refine_pass_kernel<KT, T, true>, 256, 0));
  *grid_meas = sm_count() * std::max(bps, 1);
  return PPR_OK;
}

// ------------------------------------------------------------ L2 residency of the hot rows
// A pass gathers one tile row per in-edge; rows are numbered by decreasing
// in-degree, and in- and out-degree go together on power-law graphs, so the
// most gathered rows sit at the head of the tile.  Streaming the other
// arrays of a pass (r_f, the rows written, the column indices) through L2
// evicts them, and on R-MAT scale 22 a pass then moves 7.0 GB of DRAM
// traffic for 4.6 GB of algorithmic bytes.  The correction passes therefore
// mark the first kPersistBytes of the gathered tile as persisting in L2 (an
// access-policy window given per launch, so the caller's stream is left
// unchanged): 1.404 instead of 1.459 ms per FP32 pass there, 326.7 instead
// of 334.3 us on R-MAT scale 20 (24, 32 and 64 MB windows gave less, 80 or
// 120 MB slower than none: the set-aside is at most about 84 MB of the
// 126 MB L2).  The persisting set-aside is a limit of the
// process's CUDA context, and while it is raised other kernels lose that
// part of L2 (the SpeedPPR push passes ran 40 % slower with 80 MB set
// aside and no window of their own), so it is raised for the correction
// batches only: set before a batch, and after the batch its persisting lines
// are turned back to normal and the limit restored.
constexpr size_t kPersistBytes = (size_t)48 << 20;

class HotWindow {
 public:
  bool on = false;
  size_t bytes = 0;

  HotWindow() {
    int dev = 0, max_persist = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess ||
        max_persist <= 0 || cudaDeviceGetLimit(&prev_, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
      (void)cudaGetLastError();
      return;
    }
    bytes = std::max(prev_, std::min(kPersistBytes, (size_t)max_persist));
    on = true;
  }
  ~HotWindow() { end(); }
  HotWindow(const HotWindow&) = delete;
  HotWindow& operator=(const HotWindow&) = delete;

  // before a batch of correction passes: the set-aside for the window
  cudaError_t begin() {
    if (!on || raised_ || bytes <= prev_) return cudaSuccess;
    const cudaError_t e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, bytes);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      on = false;  // run the passes without the window
      return cudaSuccess;
    }
    raised_ = true;
    return cudaSuccess;
  }
  // after the batch (its stream synchronised): persisting lines back to
  // normal, the limit back to what it was
  cudaError_t end() {
    if (!on) return cudaSuccess;
    cudaError_t e = cudaCtxResetPersistingL2Cache();
    if (raised_) {
      const cudaError_t e2 = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, prev_);
      if (e == cudaSuccess) e = e2;
      raised_ = false;
    }
    return e;
  }

 private:
  size_t prev_ = 0;
  bool raised_ = false;
};

// launch a correction pass with the head of its gathered tile (base, tile
// bytes) persisting in L2 when the window is on
template <int KT, typename T, bool MEAS>
static cudaError_t launch_refine_pass(int grid, const RefArgs& ra, const HotWindow& w, size_t tile_bytes,
                                      cudaStream_t st) {
  if (!w.on) {
    refine_pass_kernel<KT, T, MEAS><<<grid, 256, 0, st>>>(ra);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
  attr[0].val.accessPolicyWindow.base_ptr = const_cast<void*>(ra.ze_in);
  attr[0].val.accessPolicyWindow.num_bytes = std::min(w.bytes, tile_bytes);
  attr[0].val.accessPolicyWindow.hitRatio = 1.f;
  attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
  attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, refine_pass_kernel<KT, T, MEAS>, ra);
}

// the exact synchronous Q1.63 pass of a refinement cycle, with the head of
// its gathered tile z(X) persisting in L2 like the correction passes
template <int KT>
static cudaError_t launch_exact_pass(int grid, const SweepArgs& sa, const HotWindow& w, size_t tile_bytes,
                                     cudaStream_t st) {
  if (!w.on) {
    sweep_kernel<KT, false><<<grid, 256, 0, st>>>(sa);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
  attr[0].val.accessPolicyWindow.base_ptr = const_cast<u64*>(sa.z_in);
  attr[0].val.accessPolicyWindow.num_bytes = std::min(w.bytes, tile_bytes);
  attr[0].val.accessPolicyWindow.hitRatio = 1.f;
  attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
  attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sweep_kernel<KT, false>, sa);
}

// ------------------------------------------------------------ TMA passes
constexpr int kTmaWarps = 2;  // TMA warps per block of the 64-source FP32 pass (the rest take light rows)

// Chunks of the TMA pass over rows [0, u_h) of the 64-source FP32 work list:
// chunk c holds edges [c kTmaChunk, (c+1) kTmaChunk); a row meeting two or
// more chunks gets a slot for its partial sums.  Built once per graph.
static ppr_status get_tma_plan(ppr_graph* g, const Plan& lsu_plan, ppr_graph::TmaPlan** out, cudaStream_t st) {
  ppr_graph::TmaPlan& t = g->tma;
  if (!t.built) {
    const std::vector<int32_t>& d = g->h_in_deg_sorted;
    t.u_h = lsu_plan.u_light;
    t.item0 = lsu_plan.n_items_heavy;
    int64_t h = 0;
    for (int32_t u = 0; u < t.u_h; ++u) h += d[u];
    t.h_edges = (int32_t)h;
    t.n_chunks = (int32_t)((h + kTmaChunk - 1) / kTmaChunk);
    std::vector<int4> chunks((size_t)std::max(t.n_chunks, 1));
    std::vector<int32_t> slot((size_t)std::max(t.u_h, 1), -1), np;
    int64_t rs = 0;
    int32_t c = 0;
    for (int32_t u = 0; u < t.u_h; ++u) {
      const int64_t re = rs + d[u];
      for (; c < t.n_chunks && (int64_t)c * kTmaChunk < re; ++c)
        chunks[c] = make_int4(u, (int)rs, (int)re, 0);
      const int64_t c0 = rs / kTmaChunk, c1 = (re - 1) / kTmaChunk;
      if (c1 > c0) {
        slot[u] = (int32_t)np.size();
        np.push_back((int32_t)(c1 - c0 + 1));
      }
      rs = re;
    }
    t.n_slots = (int32_t)np.size();
    PPR_CUDA_TRY(cudaMalloc((void**)&t.d_chunks, sizeof(int4) * chunks.size()));
    PPR_CUDA_TRY(cudaMemcpyAsync(t.d_chunks, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice, st));
    PPR_CUDA_TRY(cudaMalloc((void**)&t.d_split_slot, sizeof(int32_t) * slot.size()));
    PPR_CUDA_TRY(
        cudaMemcpyAsync(t.d_split_slot, slot.data(), sizeof(int32_t) * slot.size(), cudaMemcpyHostToDevice, st));
    const size_t ns = (size_t)std::max(t.n_slots, 1);
    np.resize(ns, 1);
    PPR_CUDA_TRY(cudaMalloc((void**)&t.d_split_np, sizeof(int32_t) * ns));
    PPR_CUDA_TRY(cudaMemcpyAsync(t.d_split_np, np.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st));
    PPR_CUDA_TRY(cudaMalloc((void**)&t.d_split_acc, sizeof(float) * 64 * ns));
    PPR_CUDA_TRY(cudaMemsetAsync(t.d_split_acc, 0, sizeof(float) * 64 * ns, st));
    PPR_CUDA_TRY(cudaMalloc((void**)&t.d_split_cnt, sizeof(unsigned int) * ns));
    PPR_CUDA_TRY(cudaMemsetAsync(t.d_split_cnt, 0, sizeof(unsigned int) * ns, st));
    PPR_CUDA_TRY(cudaStreamSynchronize(st));
    t.built = true;
  }
  *out = &t;
  return PPR_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      (void)cudaGetLastError();
  }
  return fn;
}

// an n x 64 FP32 tile (rows of 256 B) as a 2-D tensor with one-row boxes, the
// layout tile::gather4 copies from
static ppr_status encode_tile_map(CUtensorMap* map, const void* base, int64_t n) {
  auto enc = tensor_map_encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return PPR_ERR_CUDA;
  }
  const cuuint64_t dims[2] = {64, (cuuint64_t)n};
  const cuuint64_t strides[1] = {64 * sizeof(float)};
  const cuuint32_t box[2] = {64, 1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PPR_ERR_CUDA;
  }
  return PPR_OK;
}

// grids of the TMA pass (unmeasured, measured): one full wave of resident blocks
static ppr_status tma_kernel_grids(int* grid, int* grid_meas) {
  const size_t smem = tma_smem_bytes(kTmaWarps);
  auto k0 = refine_tma_kernel<false, kTmaWarps>;
  auto k1 = refine_tma_kernel<true, kTmaWarps>;
  PPR_CUDA_TRY(cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  PPR_CUDA_TRY(cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int bps = 0;
  PPR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k0, 256, smem));
  *grid = sm_count() * std::max(bps, 1);
  PPR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k1, 256, smem));
  *grid_meas = sm_count() * std::max(bps, 1);
  return PPR_OK;
}

template <int KT>
static ppr_status run_refine(ppr_graph* g, const Plan& plan, int sweep_grid, int grid_ew, SweepArgs sa,
                             const RefineTile& t, double* resid, u64* hpin, int& sweeps, int64_t& launches,
                             std::vector<double>& bound, std::vector<double>& r0, float& ms_sweep, RefineOut& ro,
                             cudaEvent_t es0, cudaEvent_t es1, cudaStream_t st) {
  const int64_t n = g->n, m = g->m;
  const size_t cells = (size_t)n * KT;
  const int ncols = t.ncols;
  const double alpha = t.alpha, lambda = t.lambda;
  Workspace& ws = g->ws;
  u64* X = ws.pi.as<u64>();
  u64* Xn = ws.r.as<u64>();
  u64* za = ws.za.as<u64>();
  float* rf = ws.zb.as<float>();
  void* zbuf_a = rf + cells;  // 4 cells bytes each: one FP32 or one BF16 z_e array
  void* zbuf_b = ws.za.ptr;
  float* ef = ws.r.as<float>();
  const float oma = (float)(1.0 - alpha);

  Plan* plans[2] = {nullptr, nullptr};
  int grids[2] = {0, 0}, grids_meas[2] = {0, 0};
  PPR_TRY((refine_kernel_setup<KT, bf16>(g, &plans[0], &grids[0], &grids_meas[0], st)));
  PPR_TRY((refine_kernel_setup<KT, float>(g, &plans[1], &grids[1], &grids_meas[1], st)));
  RefArgs ra;
  ra.in_rp = g->d_in_rp;
  ra.in_ci = g->d_in_ci;
  ra.deg = g->d_deg;
  ra.rf = rf;
  ra.one_minus_alpha = oma;
  ra.heavy_acc = ws.heavy_acc.as<float>();
  ra.heavy_cnt = ws.heavy_cnt.as<unsigned int>();
  const bool use_bf16 = !t.fp32_only;

  // FP32 passes of a 64-source tile with PPR_FLAG_TMA_GATHER: rows with many
  // in-edges gathered by TMA
  bool use_tma = false;
  TmaArgs ta{};
  CUtensorMap maps[2];
  int grid_tma = 0, grid_tma_meas = 0;
  if constexpr (KT == 64) {
    ppr_graph::TmaPlan* tp = nullptr;
    if (t.tma_gather) PPR_TRY(get_tma_plan(g, *plans[1], &tp, st));
    if (tp && tp->n_chunks > 0) {
      PPR_TRY(encode_tile_map(&maps[0], zbuf_a, n));
      PPR_TRY(encode_tile_map(&maps[1], zbuf_b, n));
      PPR_TRY(tma_kernel_grids(&grid_tma, &grid_tma_meas));
      ta.h_edges = tp->h_edges;
      ta.u_h = tp->u_h;
      ta.n_chunks = tp->n_chunks;
      ta.item0 = tp->item0;
      ta.chunks = tp->d_chunks;
      ta.split_slot = tp->d_split_slot;
      ta.split_np = tp->d_split_np;
      ta.split_acc = tp->d_split_acc;
      ta.split_cnt = tp->d_split_cnt;
      ta.status = ws.status.as<unsigned int>();
      use_tma = true;
    }
  }
  unsigned int* h_status = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(hpin) + 64 * 8);
  HotWindow hot;

  const double slack = (double)m * 0.5 / kFixOne / alpha;
  // goal of the correction passes: after the fold the exact pass measures
  // ||X' - X||_1 of about (1-alpha) F (F = the last measured ||e' - e||_1), so
  // the certified bound comes out near (1-alpha)^2 F / alpha; aim at 0.6 lambda
  const double target_f = 0.6 * lambda * alpha / ((1.0 - alpha) * (1.0 - alpha));
  const double floor_rel[2] = {1e-2, 1e-6};  // where BF16 / FP32 passes stop contracting
  // the cycle's goal and the precision it starts in (0 = BF16 z_e, 1 = FP32):
  // BF16 only for a cycle whose whole reduction fits above its floor (about
  // 1e-2 of the start; typically the last cycle); where more is needed BF16
  // passes contract worse and leave the work to FP32.  The setup kernels
  // write z_e in the precision chosen here.
  auto cycle_goal = [&](double f0) { return std::max(target_f, floor_rel[1] * f0); };
  auto cycle_prec = [&](double f0) { return (use_bf16 && cycle_goal(f0) >= 2.0 * floor_rel[0] * f0) ? 0 : 1; };

  double F0 = 0.0;  // ||r||_1 of the cycle = ||e_1 - e_0||_1
  const bool warm_x0 = t.model && t.corr == 0;
  bool corr_pending = t.model && t.corr > 0;
  int prec0 = 1;
  if (warm_x0) {
    // X = the model's estimate; the first exact pass measures its residual
    PPR_TRY(warm_start_tile(t.model, g, t.src_new, ncols, KT, alpha, za, X, st));
    ++launches;
  } else {
    // cycle 0: X = reserve, r = alpha r_push
    for (int c = 0; c < ncols; ++c) F0 = std::max(F0, alpha * (t.have_state ? t.rsum[c] : 1.0));
    prec0 = corr_pending ? 1 : cycle_prec(F0);  // the correction model follows FP32 passes
    if (prec0 == 0)
      refine_setup_push_kernel<KT, bf16><<<grid_ew, 256, 0, st>>>(n, Xn, alpha, g->d_deg, oma, rf,
                                                                  static_cast<bf16*>(zbuf_a));
    else
      refine_setup_push_kernel<KT, float><<<grid_ew, 256, 0, st>>>(n, Xn, alpha, g->d_deg, oma, rf,
                                                                   static_cast<float*>(zbuf_a));
    ++launches;
  }
  double rates[2] = {-1.0, -1.0};  // observed contraction per pass, BF16 / FP32
  // In-place correction passes are over-relaxed (e <- e + w (e' - e): SOR on
  // the e-system).  w is the autotuner's choice for the graph, else 1.15 (on
  // R-MAT scale 20 and a Chung-Lu graph of 200,000 nodes 1.15 measured
  // fastest, on R-MAT scale 22 1.1; 1.2 and above slower).  Modes with
  // negative eigenvalues (near-bipartite structure) contract more slowly under
  // w > 1, so the first stalled batch turns relaxation off for the query.
  // Synchronous measured passes are never relaxed; every stop is certified by
  // an exact pass whatever w does.
  float relax = t.relax;
  for (int cycle = 0;; ++cycle) {
    if (cycle >= 8) {
      set_error("refinement did not certify within 8 cycles");
      return PPR_ERR_NOT_CONVERGED;
    }
    // ---- correction passes: in place, the last of each batch synchronous,
    // measured, and writing e for the fold
    const double goal = cycle_goal(F0);
    int prec = prec0;  // the precision the setup wrote z_e in
    double F = F0;
    void* zcur = zbuf_a;
    void* znext = zbuf_b;
    bool ran = false;
    while (!(warm_x0 && cycle == 0) && F > goal) {
      const double phase_goal = std::max(goal, floor_rel[prec] * F0);
      if (F <= phase_goal && prec == 0) {
        // BF16 done: continue in FP32 from the same e (z_e widened exactly)
        bf16_to_f32_kernel<<<grid_ew, 256, 0, st>>>((int64_t)cells, static_cast<const bf16*>(zcur),
                                                      static_cast<float*>(znext));
        ++launches;
        std::swap(zcur, znext);
        prec = 1;
        continue;
      }
      // a precision without a rate of its own borrows the other's; only when
      // neither is known does a short first batch learn one
      double& rate = rates[prec];
      const double known = rate > 0.0 ? rate : rates[1 - prec];
      const double cr = known > 0.0 ? known : (1.0 - alpha);
      int S = batch_passes(phase_goal, F, cr, t.max_sweeps);
      if (known <= 0.0) S = std::min(S, 16);  // learn the rate first
      if (corr_pending) S = t.corr;          // the passes the correction model was trained after
      if (sweeps + S + 1 > t.max_sweeps) {
        set_error("sweep limit %d reached", t.max_sweeps);
        return PPR_ERR_NOT_CONVERGED;
      }
      const Plan* fp = plans[prec];
      ra.items = fp->d_items;
      ra.npieces = fp->d_npieces;
      PPR_CUDA_TRY(cudaMemsetAsync(resid, 0, 64 * 8, st));
      PPR_CUDA_TRY(hot.begin());
      PPR_CUDA_TRY(cudaEventRecord(es0, st));
      for (int j = 0; j < S; ++j) {
        const bool last = j == S - 1;
        ra.ze_in = zcur;
        ra.ze_out = last ? znext : zcur;
        ra.e_out = last ? ef : nullptr;
        ra.resid = last ? resid : nullptr;
        // rows without in-edges keep z_e = r_f (1-alpha)/d from the setup; the
        // synchronous pass rewrites every row of the other buffer
        ra.n_items = last ? fp->n_items_all : fp->n_items_nz;
        // the passes before a learned correction stay plain: the model was
        // trained on the state that plain passes reach
        ra.relax = (last || corr_pending) ? 1.f : relax;
        // in-place passes take the light rows first (hub rows then gather
        // fresh values), except the passes before a learned correction, which
        // the correction suits better when they take the hub rows first
        // (R-MAT-20, 1,024 held-out sources: 26.0 passes with the model
        // against 30.0, zero start 37.4 passes either way)
        ra.light_first = corr_pending ? 0 : 1;
        if (prec == 0) {
          if (last) PPR_CUDA_TRY((launch_refine_pass<KT, bf16, true>(grids_meas[0], ra, hot, cells * 2, st)));
          else PPR_CUDA_TRY((launch_refine_pass<KT, bf16, false>(grids[0], ra, hot, cells * 2, st)));
        } else if (use_tma) {
          ta.map = zcur == zbuf_a ? maps[0] : maps[1];
          if (last)
            refine_tma_kernel<true, kTmaWarps><<<grid_tma_meas, 256, tma_smem_bytes(kTmaWarps), st>>>(ra, ta);
          else
            refine_tma_kernel<false, kTmaWarps><<<grid_tma, 256, tma_smem_bytes(kTmaWarps), st>>>(ra, ta);
        } else {
          if (last) PPR_CUDA_TRY((launch_refine_pass<KT, float, true>(grids_meas[1], ra, hot, cells * 4, st)));
          else PPR_CUDA_TRY((launch_refine_pass<KT, float, false>(grids[1], ra, hot, cells * 4, st)));
        }
      }
      PPR_CUDA_TRY(cudaEventRecord(es1, st));
      PPR_CUDA_TRY(cudaGetLastError());
      std::swap(zcur, znext);
      ran = true;
      sweeps += S;
      ro.passes[prec] += S;
      launches += S;
      PPR_CUDA_TRY(cudaMemcpyAsync(hpin, resid, 64 * 8, cudaMemcpyDeviceToHost, st));
      if (use_tma) PPR_CUDA_TRY(cudaMemcpyAsync(h_status, ta.status, 4, cudaMemcpyDeviceToHost, st));
      PPR_CUDA_TRY(cudaStreamSynchronize(st));
      // the batch is done: its persisting lines back to normal and the
      // set-aside returned before the fold and the exact pass
      PPR_CUDA_TRY(hot.end());
      if (use_tma && *h_status) {
        set_error("a TMA row-gather wait timed out in a correction pass");
        return PPR_ERR_CUDA;
      }
      float a_ms = 0.f;
      cudaEventElapsedTime(&a_ms, es0, es1);
      ms_sweep += a_ms;
      ro.ms[prec] += a_ms;
      const double* D = reinterpret_cast<const double*>(hpin);
      double Fm = 0.0;
      for (int c = 0; c < ncols; ++c) Fm = std::max(Fm, D[c]);
      if (!(Fm >= 0.0) || !std::isfinite(Fm)) {
        set_error("correction passes diverged");
        return PPR_ERR_NOT_CONVERGED;
      }
      // stalled: the batch achieved less than a quarter of the log-reduction
      // that (1-alpha) per pass guarantees in exact arithmetic (any batch
      // length): the precision's floor is reached
      const bool stalled = Fm > F * std::pow(1.0 - alpha, 0.25 * S);
      if (Fm > 0.0 && Fm < F && S >= 2 && !stalled)
        rate = std::min(1.0 - alpha, std::max(0.05, std::pow(Fm / F, 1.0 / S)));
      F = Fm;
      if (corr_pending) break;
      // a stall within 100x of the precision's floor is that floor (the stage
      // is done); a stall above it, with over-relaxation on, is a mode that
      // w > 1 amplifies: the stage is retried without over-relaxation.
      // (Turning relaxation off at the floor as well wasted a batch there and
      // left the rest of the query unrelaxed.)
      const bool near_floor = F <= 100.0 * floor_rel[prec] * F0;
      if (stalled && relax != 1.f && !near_floor) {
        relax = 1.f;  // retry the stage without over-relaxation
        rates[0] = rates[1] = -1.0;
        continue;
      }
      if (stalled) {
        if (prec == 1) break;
        if (F > goal) {
          // BF16 stopped contracting: continue in FP32 from the same e
          bf16_to_f32_kernel<<<grid_ew, 256, 0, st>>>((int64_t)cells, static_cast<const bf16*>(zcur),
                                                        static_cast<float*>(znext));
          ++launches;
          std::swap(zcur, znext);
          prec = 1;
        }
      }
    }
    if (!(warm_x0 && cycle == 0)) {
      if (!ran) {
        // nothing ran (r already below the goal): e = r
        PPR_CUDA_TRY(cudaMemcpyAsync(ef, rf, cells * 4, cudaMemcpyDeviceToDevice, st));
      }
      // ---- fold e into X (z(X) to za)
      refine_fold_kernel<KT><<<grid_ew, 256, 0, st>>>(n, ef, X, g->d_omega, za);
      ++launches;
      if (corr_pending) {
        // X += mu q (mu = 1 - sum X, exact), z(X) rewritten
        PPR_CUDA_TRY(cudaMemsetAsync(t.mass, 0, 8 * KT, st));
        column_sum_kernel<KT><<<grid_ew, 256, 0, st>>>(n, X, t.mass);
        PPR_TRY(warm_correct_tile(t.model, g, t.src_new, ncols, KT, alpha, X, t.mass, za, X, st));
        launches += 2;
        corr_pending = false;
        rates[0] = rates[1] = -1.0;  // the correction changes the error: learn the rates again
      }
    }

    // ---- one exact synchronous pass from X.  When the last measured F puts
    // the coming bound far above lambda, the pass also sets up the next cycle
    // (r = X' - X exactly, in the precision that cycle will start in) instead
    // of writing X'; should it certify after all, a plain pass from the same
    // X produces X'.
    const bool measured = !(warm_x0 && cycle == 0) && ran;
    const double predicted_bound = (1.0 - alpha) * (1.0 - alpha) * F / alpha;
    bool fused = measured && predicted_bound > 4.0 * lambda;
    const int prec_next = cycle_prec((1.0 - alpha) * F);
    for (;;) {
      PPR_CUDA_TRY(cudaMemsetAsync(resid, 0, 64 * 8, st));
      sa.z_in = za;
      sa.z_out = nullptr;
      sa.x_out = fused ? nullptr : Xn;
      sa.x_base = fused ? X : nullptr;
      sa.rf_next = fused ? rf : nullptr;
      sa.ze_next = fused ? zbuf_a : nullptr;
      sa.ze_bf16 = prec_next == 0;
      sa.n_items = plan.n_items_all;
      sa.resid = resid;
      PPR_CUDA_TRY(hot.begin());
      PPR_CUDA_TRY(cudaEventRecord(es0, st));
      PPR_CUDA_TRY(launch_exact_pass<KT>(sweep_grid, sa, hot, cells * 8, st));
      PPR_CUDA_TRY(cudaEventRecord(es1, st));
      ++sweeps;
      ++launches;
      PPR_CUDA_TRY(cudaMemcpyAsync(hpin, resid, 64 * 8, cudaMemcpyDeviceToHost, st));
      PPR_CUDA_TRY(cudaStreamSynchronize(st));
      PPR_CUDA_TRY(hot.end());
      float a_ms = 0.f;
      cudaEventElapsedTime(&a_ms, es0, es1);
      ms_sweep += a_ms;
      if (!fused) break;
      // certified after all: X' is needed, so run the plain pass
      const double* Dq = reinterpret_cast<const double*>(hpin);
      bool ok_q = true;
      for (int c = 0; c < ncols; ++c)
        if ((1.0 - alpha) * (Dq[c] / kFixOne / alpha) * (1.0 + 1e-4) + 2.0 * slack > lambda) ok_q = false;
      if (!ok_q) break;
      fused = false;
    }
    sa.x_base = nullptr;
    sa.rf_next = nullptr;
    sa.ze_next = nullptr;
    ++ro.cycles;
    const double* D = reinterpret_cast<const double*>(hpin);
    bool ok = true;
    F0 = 0.0;
    for (int c = 0; c < ncols; ++c) {
      const double Dc = D[c] / kFixOne / alpha;  // ||X' - X||_1 / alpha
      bound[c] = (1.0 - alpha) * Dc * (1.0 + 1e-4) + 2.0 * slack;
      if (bound[c] > lambda) ok = false;
      F0 = std::max(F0, Dc * alpha);
      if (warm_x0 && cycle == 0) r0[c] = Dc;  // measured ||r(x0)||_1 of the model's estimate
    }
    if (ok) {
      ro.relax = relax;
      return PPR_OK;
    }
    if (fused) {
      prec0 = prec_next;  // the pass wrote r and z_e of the next cycle
      continue;
    }
    // next cycle from X: r = X' - X, z_e in the precision the cycle starts in
    prec0 = cycle_prec(F0);
    if (prec0 == 0)
      refine_setup_resid_kernel<KT, bf16><<<grid_ew, 256, 0, st>>>(n, Xn, X, g->d_deg, oma, rf,
                                                                   static_cast<bf16*>(zbuf_a));
    else
      refine_setup_resid_kernel<KT, float><<<grid_ew, 256, 0, st>>>(n, Xn, X, g->d_deg, oma, rf,
                                                                    static_cast<float*>(zbuf_a));
    ++launches;
  }
}

template <int KT>
static ppr_status run_hp(ppr_graph* g, const int32_t* src, int32_t k, const ppr_query_opts& o, double* out_pi,
                         double* out_r, ppr_stats* stats, cudaStream_t st) {
  const int64_t n = g->n, m = g->m;
  const double alpha = o.alpha, lambda = o.lambda;
  Workspace& ws = g->ws;
  const size_t cells = (size_t)n * KT;
  // outputs the kernels can write directly (device memory or pinned host
  // memory); the rest is staged on the device and copied at the end
  double* pi_view = static_cast<double*>(device_view(out_pi));
  double* r_view = out_r ? static_cast<double*>(device_view(out_r)) : nullptr;
  const bool pi_on_host = pi_view == nullptr;
  const bool r_on_host = out_r && r_view == nullptr;
  if (o.max_sweeps > kMaxSweepsCap) {
    set_error("max_sweeps %d above the limit of %d passes", o.max_sweeps, kMaxSweepsCap);
    return PPR_ERR_ARG;
  }
  const int max_sweeps = o.max_sweeps > 0 ? o.max_sweeps : sweep_limit(alpha, lambda);
  if (max_sweeps < 1) {
    set_error("alpha %g is too small for lambda %g: more than %d passes", alpha, lambda, kMaxSweepsCap);
    return PPR_ERR_ARG;
  }

  // admission: state for one tile plus staging of host outputs, against free
  // device memory plus what the workspace already holds (reused)
  const size_t need = hp_workspace_bytes(g, KT, max_sweeps);
  size_t stage_bytes = 0;
  if (pi_on_host) stage_bytes += (size_t)k * n * 8;
  if (r_on_host) stage_bytes += (size_t)k * n * 8;
  {
    size_t free_b = 0, total_b = 0;
    PPR_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    free_b = admission_free_bytes(free_b);
    if (need + stage_bytes > free_b + ws.hp_bytes()) {
      set_error("admission refused: batch state needs %zu bytes, %zu free", need + stage_bytes, free_b);
      return PPR_ERR_ADMIT;
    }
  }
  PPR_TRY(ws.r.ensure(cells * 8));
  PPR_TRY(ws.pi.ensure(cells * 8));
  PPR_TRY(ws.za.ensure(cells * 8));
  PPR_TRY(ws.zb.ensure(cells * 8));
  PPR_TRY(ws.stamp.ensure(cells * 4));
  PPR_TRY(ws.front_a.ensure(cells * 4));
  PPR_TRY(ws.front_b.ensure(cells * 4));
  PPR_TRY(ws.ent_share.ensure(cells * 8));
  PPR_TRY(ws.ent_rem.ensure(cells * 4));
  PPR_TRY(ws.chunks.ensure((cells + (size_t)m * KT / kPushChunk + 64) * 8));
  static_assert(KT >= 1 && KT <= 64 && (KT & (KT - 1)) == 0, "tile width must be a power of two <= 64");
  Plan* plan_p = nullptr;
  PPR_TRY(get_plan(g, Lay<KT>::L, &plan_p, st));
  Plan& plan = *plan_p;
  const size_t acc_bytes = std::max<size_t>((size_t)plan.n_split * KT * 8, 8);
  const size_t cnt_bytes = std::max<size_t>((size_t)plan.n_split * 4, 4);
  PPR_TRY(ws.heavy_acc.ensure(acc_bytes));
  PPR_TRY(ws.heavy_cnt.ensure(cnt_bytes));
  PPR_TRY(ws.counters.ensure(16384));
  PPR_TRY(ws.resid.ensure((size_t)(max_sweeps + 1) * 64 * 8));
  PPR_TRY(ws.status.ensure(8));
  PPR_CUDA_TRY(cudaMemsetAsync(ws.status.ptr, 0, 8, st));

  if (stage_bytes) PPR_TRY(ws.stage.ensure(stage_bytes));
  if (!ws.pinned) {
    PPR_CUDA_TRY(cudaMallocHost(&ws.pinned, 65536));
    ws.pinned_bytes = 65536;
  }
  // buffers whose contents must start at zero, cleared once after each
  // (re)allocation (also when an earlier call failed before clearing them)
  if (ws.stamp.fresh || g->stamp_epoch > 0xF0000000u) {
    PPR_CUDA_TRY(cudaMemsetAsync(ws.stamp.ptr, 0, ws.stamp.bytes, st));
    g->stamp_epoch = 0;
    ws.stamp.fresh = false;
  }
  if (ws.heavy_acc.fresh || ws.heavy_cnt.fresh) {
    PPR_CUDA_TRY(cudaMemsetAsync(ws.heavy_acc.ptr, 0, ws.heavy_acc.bytes, st));
    PPR_CUDA_TRY(cudaMemsetAsync(ws.heavy_cnt.ptr, 0, ws.heavy_cnt.bytes, st));
    ws.heavy_acc.fresh = ws.heavy_cnt.fresh = false;
  }
  PPR_TRY(ensure_alpha(g, alpha, st));

  u64* r = ws.r.as<u64>();
  u64* pi = ws.pi.as<u64>();
  u64* za = ws.za.as<u64>();
  u64* zb = ws.zb.as<u64>();
  u64* counters = ws.counters.as<u64>();
  double* resid = ws.resid.as<double>();
  u64* hpin = static_cast<u64*>(ws.pinned);
  int32_t* d_src = reinterpret_cast<int32_t*>(counters + 512);  // device copy of the tile's sources
  u64* mass = counters + 256;                                    // exact column sums of the output
  double* out_pi_dev = pi_on_host ? ws.stage.as<double>() : pi_view;
  double* out_r_dev = !out_r ? nullptr : (r_on_host ? ws.stage.as<double>() + (pi_on_host ? (size_t)k * n : 0) : r_view);

  const u64 alpha64 = (u64)(alpha * 18446744073709551616.0);
  const u64 alpha_raw = (u64)(alpha * kFixOne);
  const double rmax = lambda / (double)m;
  const u64 rmax_raw = (u64)std::max(1.0, std::floor(rmax * kFixOne));
  const u64 lambda_raw = (u64)std::floor(lambda * kFixOne);
  const double tuned_frac = g->tuned_switch_frac[tune_bucket(k)];
  const int64_t switch_edges = o.switch_edges >= 0 ? o.switch_edges
                                                   : (int64_t)((tuned_frac >= 0 ? tuned_frac : 0.02) * (double)m * KT);
  int bps = 0;
  PPR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, sweep_kernel<KT, false>, 256, 0));
  const int sweep_grid = sm_count() * std::max(bps, 1);


  const int grid_ew = sm_count() * 8;

  cudaEvent_t ev0, ev1, ev2, es0, es1;
  PPR_CUDA_TRY(cudaEventCreate(&ev0));
  PPR_CUDA_TRY(cudaEventCreate(&ev1));
  PPR_CUDA_TRY(cudaEventCreate(&ev2));
  PPR_CUDA_TRY(cudaEventCreate(&es0));
  PPR_CUDA_TRY(cudaEventCreate(&es1));
  float ms_push = 0.f, ms_sweep = 0.f, ms_total = 0.f, ms_fp32 = 0.f, ms_bf16 = 0.f;
  int64_t launches = 0, sweep_launches = 0;

  ppr_status status = PPR_OK;

  for (int32_t t0 = 0; t0 < k && status == PPR_OK; t0 += KT) {
    const int ncols = std::min<int32_t>(KT, k - t0);
    int32_t src_new[64];
    for (int c = 0; c < 64; ++c) src_new[c] = c < ncols ? g->h_new_of_old[src[t0 + c]] : -1;
    PPR_CUDA_TRY(cudaEventRecord(ev0, st));

    // ---- queue phase
    std::vector<double> rsum(KT, 0.0), r0(KT, 1.0);
    std::vector<int64_t> pushed(KT, 0);
    int levels = 0;
    bool all_done = false;
    bool frontier_empty = false;  // the queue phase ended with no active node
    bool have_state = false;  // (r, pi) hold a push state
    // a learned estimate either replaces the zero start (correction_passes = 0)
    // or corrects the remaining mass after `corr` passes of the zero-start solve
    const int corr = o.warm_start ? warm_correction_passes(o.warm_start) : 0;
    const bool warm = o.warm_start != nullptr && corr == 0;
    const bool partial = (o.flags & PPR_FLAG_PARTIAL) != 0;
    const bool no_active = (o.flags & PPR_FLAG_NO_ACTIVE) != 0;
    const bool refine = !partial && (o.flags & (PPR_FLAG_SYNC | PPR_FLAG_FIXED_PASSES)) == 0;
    bool corrected = false;
    if (switch_edges != 0 && !warm) {
      PPR_CUDA_TRY(cudaMemsetAsync(r, 0, cells * 8, st));
      PPR_CUDA_TRY(cudaMemsetAsync(pi, 0, cells * 8, st));
      PPR_CUDA_TRY(cudaMemsetAsync(counters, 0, 8 * (3 + 2 * KT), st));
      PPR_CUDA_TRY(cudaMemcpyAsync(d_src, src_new, sizeof(src_new), cudaMemcpyHostToDevice, st));
      uint32_t* fa = ws.front_a.as<uint32_t>();
      uint32_t* fb = ws.front_b.as<uint32_t>();
      const uint32_t epoch0 = ++g->stamp_epoch;
      init_sources_kernel<KT><<<1, 64, 0, st>>>(d_src, ncols, r, ws.stamp.as<uint32_t>(), epoch0, fa);
      ++launches;
      uint64_t nfront = (uint64_t)ncols;
      have_state = true;
      while (true) {
        PPR_CUDA_TRY(cudaMemsetAsync(counters, 0, 24, st));
        PushArgs pa;
        pa.front = fa;
        pa.n_front = (uint32_t)nfront;
        pa.out_rp = g->d_out_rp;
        pa.out_ci = g->d_out_ci;
        pa.deg = g->d_deg;
        pa.r = r;
        pa.pi = pi;
        pa.stamp = ws.stamp.as<uint32_t>();
        pa.next_stamp = ++g->stamp_epoch;
        pa.next_front = fb;
        pa.ent_share = ws.ent_share.as<u64>();
        pa.ent_rem = ws.ent_rem.as<uint32_t>();
        pa.chunks = ws.chunks.as<u64>();
        pa.counters = counters;
        pa.alpha64 = alpha64;
        pa.rmax_raw = rmax_raw;
        const int tb = (int)std::min<uint64_t>((nfront + 255) / 256, (uint64_t)grid_ew);
        push_take_kernel<KT><<<std::max(tb, 1), 256, 0, st>>>(pa);
        push_scatter_kernel<KT><<<grid_ew, 256, 0, st>>>(pa);
        launches += 2;
        PPR_CUDA_TRY(cudaGetLastError());
        PPR_CUDA_TRY(cudaMemcpyAsync(hpin, counters, 8 * (3 + 2 * KT), cudaMemcpyDeviceToHost, st));
        PPR_CUDA_TRY(cudaStreamSynchronize(st));
        ++levels;
        nfront = hpin[0];
        const uint64_t fedges = hpin[1];
        all_done = true;
        for (int c = 0; c < ncols; ++c) {
          u64 stopped = hpin[3 + c];
          u64 rraw = kFixOneRaw - stopped;  // mass is conserved exactly: sum r = 1 - sum pi
          rsum[c] = (double)rraw / kFixOne;
          pushed[c] = (int64_t)hpin[3 + KT + c];
          if (rraw > lambda_raw) all_done = false;
        }
        frontier_empty = nfront == 0;
        if ((all_done && !no_active) || nfront == 0) break;
        if ((int64_t)fedges > switch_edges) break;
        if (levels > max_sweeps) { set_error("queue phase did not finish"); status = PPR_ERR_NOT_CONVERGED; break; }
        std::swap(fa, fb);
      }
      if (status != PPR_OK) break;
      for (int c = 0; c < KT; ++c) r0[c] = (1.0 - alpha) * rsum[c];
    }
    PPR_CUDA_TRY(cudaEventRecord(ev1, st));

    // ---- sweep phase
    int sweeps = 0, fp32_passes = 0, bf16_passes = 0, refine_cycles = 0;
    float relax_end = 1.f;
    std::vector<double> bound(KT, 0.0);
    u64* xfinal = pi;  // the estimate to output
    // the no-active end state also needs the frontier emptied
    bool need_dense = !all_done || (no_active && !frontier_empty);
    if (!need_dense) {
      for (int c = 0; c < ncols; ++c) bound[c] = rsum[c];
    } else if (o.epoch_num > 0) {
      // Algorithm 3's epochs (thresholded passes) instead of push-every-node passes
      if (!have_state) {
        PPR_CUDA_TRY(cudaMemsetAsync(r, 0, cells * 8, st));
        PPR_CUDA_TRY(cudaMemsetAsync(pi, 0, cells * 8, st));
        PPR_CUDA_TRY(cudaMemcpyAsync(d_src, src_new, sizeof(src_new), cudaMemcpyHostToDevice, st));
        init_sources_kernel<KT><<<1, 64, 0, st>>>(d_src, ncols, r, ws.stamp.as<uint32_t>(), ++g->stamp_epoch,
                                                  ws.front_a.as<uint32_t>());
        ++launches;
        for (int c = 0; c < ncols; ++c) rsum[c] = 1.0;
      }
      for (int c = 0; c < ncols; ++c) r0[c] = rsum[c];
      status = run_epochs<KT>(g, plan, sweep_grid, grid_ew, o.epoch_num, no_active, lambda, alpha, max_sweeps, ncols,
                              r, pi, za, zb, counters + 1024, hpin, sweeps, rsum, launches, ms_sweep, es0, es1, st);
      if (status != PPR_OK) break;
      sweep_launches += sweeps;
      // each pass rounds d shares per node by at most half a unit each
      const double slack = (double)sweeps * (double)m * 0.5 / kFixOne;
      for (int c = 0; c < ncols; ++c) bound[c] = rsum[c] + slack;
      xfinal = pi;
      if (out_r)
        output_kernel<KT><<<grid_ew, 256, 0, st>>>(n, g->d_new_of_old, r, ncols, t0, out_r_dev), ++launches;
    } else if (refine) {
      // FP32 correction passes certified by exact passes (the default solve)
      if (!have_state) {
        PPR_CUDA_TRY(cudaMemsetAsync(r, 0, cells * 8, st));
        PPR_CUDA_TRY(cudaMemsetAsync(pi, 0, cells * 8, st));
        PPR_CUDA_TRY(cudaMemcpyAsync(d_src, src_new, sizeof(src_new), cudaMemcpyHostToDevice, st));
        init_sources_kernel<KT><<<1, 64, 0, st>>>(d_src, ncols, r, ws.stamp.as<uint32_t>(), ++g->stamp_epoch,
                                                  ws.front_a.as<uint32_t>());
        ++launches;
        for (int c = 0; c < KT; ++c) r0[c] = 1.0;
      }
      SweepArgs sa;
      sa.items = plan.d_items;
      sa.in_rp = g->d_in_rp;
      sa.in_ci = g->d_in_ci;
      sa.omega = g->d_omega;
      sa.invw = g->d_invw;
      sa.alpha_raw = alpha_raw;
      for (int c = 0; c < 64; ++c) sa.src[c] = src_new[c];
      sa.heavy_npieces = plan.d_npieces;
      sa.heavy_acc = ws.heavy_acc.as<u64>();
      sa.heavy_cnt = ws.heavy_cnt.as<unsigned int>();
      RefineTile rt;
      rt.ncols = ncols;
      rt.alpha = alpha;
      rt.lambda = lambda;
      rt.max_sweeps = max_sweeps;
      rt.have_state = have_state;
      rt.rsum = rsum;
      rt.model = o.warm_start;
      rt.corr = corr;
      rt.src_new = src_new;
      rt.mass = mass;
      rt.fp32_only = (o.flags & PPR_FLAG_FP32_ONLY) != 0;
      rt.tma_gather = (o.flags & PPR_FLAG_TMA_GATHER) != 0;
      rt.relax = g->tuned_relax[tune_bucket(k)] > 0.f ? g->tuned_relax[tune_bucket(k)] : kRelax;
      RefineOut ro;
      status = run_refine<KT>(g, plan, sweep_grid, grid_ew, sa, rt, resid, hpin, sweeps, launches, bound, r0,
                              ms_sweep, ro, es0, es1, st);
      bf16_passes = ro.passes[0];
      fp32_passes = ro.passes[1];
      refine_cycles = ro.cycles;
      relax_end = ro.relax;
      ms_bf16 += ro.ms[0];
      ms_fp32 += ro.ms[1];
      if (status != PPR_OK) break;
      sweep_launches += sweeps;
      xfinal = r;
      if (out_r) {
        // residual of the returned estimate: one more gather over z(X')
        z_of_x_kernel<KT><<<grid_ew, 256, 0, st>>>(n, r, g->d_omega, za);
        residual_kernel<KT><<<grid_ew, 256, 0, st>>>((int32_t)n, g->d_in_rp, g->d_in_ci, g->d_old_of_new, za, r, sa,
                                                     ncols, t0, alpha, out_r_dev);
        launches += 2;
      }
    } else {
      if (warm) {
        // x0 from the model; its residual norm is measured by the first pass
        PPR_CUDA_TRY(cudaMemsetAsync(za, 0, cells * 8, st));
        PPR_TRY(warm_start_tile(o.warm_start, g, src_new, ncols, KT, alpha, za, nullptr, st));
        for (int c = 0; c < KT; ++c) r0[c] = std::numeric_limits<double>::infinity();
      } else if (have_state) {
        convert_kernel<KT><<<grid_ew, 256, 0, st>>>(n, r, pi, g->d_omega, alpha64, za);
        ++launches;
      } else {
        PPR_CUDA_TRY(cudaMemsetAsync(za, 0, cells * 8, st));
        for (int c = 0; c < KT; ++c) r0[c] = 1.0;
      }
      PPR_CUDA_TRY(cudaMemsetAsync(resid, 0, (size_t)(max_sweeps + 1) * 64 * 8, st));

      SweepArgs sa;
      sa.items = plan.d_items;
      sa.in_rp = g->d_in_rp;
      sa.in_ci = g->d_in_ci;
      sa.omega = g->d_omega;
      sa.invw = g->d_invw;
      sa.alpha_raw = alpha_raw;
      for (int c = 0; c < 64; ++c) sa.src[c] = src_new[c];
      sa.heavy_npieces = plan.d_npieces;
      sa.heavy_acc = ws.heavy_acc.as<u64>();
      sa.heavy_cnt = ws.heavy_cnt.as<unsigned int>();
      // x of the final pass goes to the residue buffer (free after the conversion)
      u64* zcur = za;
      u64* znext = zb;
      double R = 0.0;
      for (int c = 0; c < ncols; ++c) R = std::max(R, r0[c]);
      double rate = -1.0, prev_d = -1.0;  // observed contraction per pass
      int prev_sweeps = 0;
      // Passes run in place (one z buffer) except the last of each batch: rows
      // then gather neighbours already updated in the same pass, the GPU form
      // of the asynchronous pushes of Sec. 5 (chaotic relaxation of the same
      // contraction, converging faster than synchronous passes).  The last
      // pass of a batch is synchronous, so its measured ||x' - x||_1 / alpha is
      // the exact residual norm of the estimate and certifies the stop.
      // PPR_FLAG_SYNC keeps every pass synchronous (SimFwdPush = PowItr).
      const bool sync_only = (o.flags & PPR_FLAG_SYNC) != 0;
      bool probe_next = warm || !sync_only;  // learn the contraction rate before a long batch
      int probe_len = warm ? 4 : 16;
      while (true) {
        // unknown residual (warm start): one pass measures it.  The residual
        // contracts at least by (1-alpha) per pass; once two measurements exist
        // the observed rate (faster after a learned correction) predicts the
        // passes, and every stop is still certified by a measurement.
        const double cr = rate > 0.0 ? rate : (1.0 - alpha);
        int S = (!std::isfinite(R) || R <= lambda) ? 1 : batch_passes(lambda, R, cr, max_sweeps);
        if (rate <= 0.0 && probe_next) S = std::min(S, probe_len);
        if (corr > 0 && !corrected) S = std::max(corr - sweeps, 1);  // passes before the correction
        if (partial) S = std::max(max_sweeps - sweeps, 0);
        if (partial && S == 0) break;
        if (sweeps + S > max_sweeps) {
          set_error("sweep limit %d reached", max_sweeps);
          status = PPR_ERR_NOT_CONVERGED;
          break;
        }
        PPR_CUDA_TRY(cudaEventRecord(es0, st));
        for (int j = 0; j < S; ++j) {
          const bool sync_pass = sync_only || j == S - 1;
          sa.z_in = zcur;
          sa.z_out = sync_pass ? znext : zcur;
          sa.x_out = (j == S - 1) ? r : nullptr;
          // after two passes rows without in-edges hold their constant value in
          // both buffers; the pass that writes x still covers every row
          sa.n_items = (sweeps + j >= 2 && !sa.x_out) ? plan.n_items_nz : plan.n_items_all;
          // only the last pass of a batch has its residual read back
          sa.resid = j == S - 1 ? resid + (size_t)(sweeps + j) * 64 : nullptr;
          launch_sweep<KT>(sa, sweep_grid, st);
          if (sync_pass) std::swap(zcur, znext);
        }
        PPR_CUDA_TRY(cudaEventRecord(es1, st));
        PPR_CUDA_TRY(cudaGetLastError());
        sweeps += S;
        launches += S;
        sweep_launches += S;
        PPR_CUDA_TRY(cudaMemcpyAsync(hpin, resid + (size_t)(sweeps - 1) * 64, 64 * 8, cudaMemcpyDeviceToHost, st));
        PPR_CUDA_TRY(cudaStreamSynchronize(st));
        {
          float a = 0.f;
          cudaEventElapsedTime(&a, es0, es1);
          ms_sweep += a;
        }
        const double* D = reinterpret_cast<const double*>(hpin);
        // ||r(x_new)||_1 <= (1-alpha) ||r(x_old)||_1, with ||r(x_old)||_1 = ||x_new - x_old||_1 / alpha;
        // the factor covers the float accumulation of the measurement, the
        // additive term the fixed-point rounding of one pass (m half-ulps)
        const double slack = (double)m * 0.5 / kFixOne / alpha;
        bool ok = true;
        R = 0.0;
        double dmax = 0.0;
        for (int c = 0; c < ncols; ++c) dmax = std::max(dmax, D[c] / kFixOne / alpha);
        if (prev_d > 0.0 && dmax > 0.0 && dmax < prev_d && sweeps > prev_sweeps)
          rate = std::min(1.0 - alpha, std::max(0.02, std::pow(dmax / prev_d, 1.0 / (sweeps - prev_sweeps))));
        if (prev_d > 0.0 || !probe_next) probe_next = false;
        prev_d = dmax;
        prev_sweeps = sweeps;
        for (int c = 0; c < ncols; ++c) {
          double Dc = D[c] / kFixOne / alpha;
          if (!std::isfinite(r0[c])) r0[c] = Dc;  // warm start: measured ||r(x0)||_1
          bound[c] = (1.0 - alpha) * Dc * (1.0 + 1e-4) + 2.0 * slack;
          if (bound[c] > lambda) ok = false;
          R = std::max(R, bound[c]);
        }
        if (partial) break;
        if (corr > 0 && !corrected) {
          // add mu * q to x (mu = 1 - sum x, exact), rebuild z for the next pass;
          // the residual's sum becomes zero and its norm is measured again
          PPR_CUDA_TRY(cudaMemsetAsync(mass, 0, 8 * KT, st));
          column_sum_kernel<KT><<<grid_ew, 256, 0, st>>>(n, r, mass);
          PPR_TRY(warm_correct_tile(o.warm_start, g, src_new, ncols, KT, alpha, r, mass, zcur, nullptr, st));
          launches += 1;
          corrected = true;
          R = std::numeric_limits<double>::infinity();
          rate = -1.0;        // the correction changes the residual: measure afresh
          prev_d = -1.0;
          probe_next = true;  // short first batch to learn the new contraction rate
          probe_len = 4;
          continue;
        }
        if (ok) break;
      }
      if (status != PPR_OK) break;
      xfinal = r;
      if (out_r) {
        // residual of the returned estimate: one more gather over z(x_final)
        SweepArgs ra = sa;
        const int ncols_i = ncols;
        residual_kernel<KT><<<grid_ew, 256, 0, st>>>((int32_t)n, g->d_in_rp, g->d_in_ci, g->d_old_of_new, zcur, r,
                                                     ra, ncols_i, t0, alpha, out_r_dev);
        ++launches;
      }
    }
    PPR_CUDA_TRY(cudaEventRecord(ev2, st));
    PPR_CUDA_TRY(cudaMemsetAsync(mass, 0, 8 * KT, st));
    output_kernel<KT><<<grid_ew, 256, 0, st>>>(n, g->d_new_of_old, xfinal, ncols, t0, out_pi_dev);
    column_sum_kernel<KT><<<grid_ew, 256, 0, st>>>(n, xfinal, mass);
    launches += 2;
    if (!need_dense && out_r)  // the queue phase finished: its residue is the answer's residual
      output_kernel<KT><<<grid_ew, 256, 0, st>>>(n, g->d_new_of_old, r, ncols, t0, out_r_dev), ++launches;
    PPR_CUDA_TRY(cudaGetLastError());
    PPR_CUDA_TRY(cudaMemcpyAsync(hpin, mass, 8 * KT, cudaMemcpyDeviceToHost, st));
    PPR_CUDA_TRY(cudaStreamSynchronize(st));
    float a1 = 0, a2 = 0;
    cudaEventElapsedTime(&a1, ev0, ev1);
    cudaEventElapsedTime(&a2, ev0, ev2);
    ms_push += a1;
    ms_total += a2;
    if (stats) {
      for (int c = 0; c < ncols; ++c) {
        ppr_stats& s = stats[t0 + c];
        memset(&s, 0, sizeof(s));
        s.sweeps = sweeps;
        s.levels = levels;
        s.edges_pushed = pushed[c];
        s.edges_swept = (int64_t)sweeps * m;
        s.initial_l1_residual = need_dense ? r0[c] : rsum[c];
        s.final_l1_residual = bound[c];
        s.mass_deficit = 1.0 - (double)hpin[c] / kFixOne;
        s.fp32_passes = fp32_passes;
        s.bf16_passes = bf16_passes;
        s.refine_cycles = refine_cycles;
        s.relax = relax_end;
      }
    }
  }
  if (status == PPR_OK) {
    if (pi_on_host)
      PPR_CUDA_TRY(cudaMemcpyAsync(out_pi, out_pi_dev, (size_t)k * n * 8, cudaMemcpyDeviceToHost, st));
    if (r_on_host)
      PPR_CUDA_TRY(cudaMemcpyAsync(out_r, out_r_dev, (size_t)k * n * 8, cudaMemcpyDeviceToHost, st));
    PPR_CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (stats && status == PPR_OK)
    for (int32_t i = 0; i < k; ++i) {
      stats[i].ms_push = ms_push;
      stats[i].ms_sweep = ms_sweep;
      stats[i].ms_total = ms_total;
      stats[i].ms_fp32 = ms_fp32;
      stats[i].ms_bf16 = ms_bf16;
      stats[i].kernel_launches = launches;
      stats[i].sweep_launches = sweep_launches;
    }
  for (cudaEvent_t e : {ev0, ev1, ev2, es0, es1}) cudaEventDestroy(e);
  return status;
}

// device bytes a high-precision query of k sources allocates (workspace for one
// tile), as used by the admission check of run_hp (host staging excluded)
// tile width of an HP query of k sources: the caller's, else the autotuned
// one of k's bucket, else the smallest power of two >= k (at most 64): one
// pass per tile, and a wider tile costs less per source than two narrow ones
int hp_tile_width(const ppr_graph* g, int32_t k, int32_t k_tile) {
  int kt = k_tile;
  if (kt == 0 && g->tuned_kt[tune_bucket(k)] > 0) kt = g->tuned_kt[tune_bucket(k)];
  if (kt == 0) {
    kt = 1;
    while (kt < k && kt < 64) kt <<= 1;
  }
  return kt;
}

// Device bytes run_hp<kt> holds in the graph's workspace (staging of outputs
// to pageable host memory excluded): the four Q1.63 tile arrays, frontier
// stamps and lists and the per-entry push remainders (4 x 4 B per cell), the
// per-entry shares and the push chunk records, the partial sums of split rows
// (rows longer than one piece of the Q1.63 work list, which splits the most
// rows), counters, the per-pass residual sums and the status word.
size_t hp_workspace_bytes(const ppr_graph* g, int kt, int max_sweeps) {
  const size_t cells = (size_t)g->n * kt;
  const int L = kt >= 2 ? kt / 2 : 1;  // lanes per row of the Q1.63 passes
  const int piece = plan_piece_edges(L);
  const std::vector<int32_t>& d = g->h_in_deg_sorted;
  size_t n_split = 0;
  while (n_split < d.size() && d[n_split] > piece) ++n_split;
  return 4 * cells * 8 + 4 * cells * 4 + cells * 8 + (cells + (size_t)g->m * kt / kPushChunk + 64) * 8 +
         std::max<size_t>(n_split * kt * 8, 8) + std::max<size_t>(n_split * 4, 4) + 16384 +
         (size_t)(max_sweeps + 1) * 64 * 8 + 8;
}

int64_t hp_state_bytes(const ppr_graph* g, int32_t k, int32_t kt) {
  return (int64_t)hp_workspace_bytes(g, hp_tile_width(g, k, kt), sweep_limit(0.2, 1e-8));
}

ppr_status query_hp(ppr_graph* g, const int32_t* src, int32_t k, const ppr_query_opts& o, double* out_pi,
                    double* out_r, ppr_stats* stats, cudaStream_t st) {
  const int kt = hp_tile_width(g, k, o.k_tile);
  if ((size_t)g->n * kt >= ((size_t)1 << 32)) {
    set_error("n * k_tile must stay below 2^32");
    return PPR_ERR_ARG;
  }
  switch (kt) {
    case 1: return run_hp<1>(g, src, k, o, out_pi, out_r, stats, st);
    case 2: return run_hp<2>(g, src, k, o, out_pi, out_r, stats, st);
    case 4: return run_hp<4>(g, src, k, o, out_pi, out_r, stats, st);
    case 8: return run_hp<8>(g, src, k, o, out_pi, out_r, stats, st);
    case 16: return run_hp<16>(g, src, k, o, out_pi, out_r, stats, st);
    case 32: return run_hp<32>(g, src, k, o, out_pi, out_r, stats, st);
    case 64: return run_hp<64>(g, src, k, o, out_pi, out_r, stats, st);
    default: set_error("k_tile must be 0, 1, 2, 4, 8, 16, 32 or 64"); return PPR_ERR_ARG;
  }
}

// ------------------------------------------- self-test of the conversions
// The integer-only conversions of sweep_kernel.cuh against CUDA's own
// conversion intrinsics, on counter-generated inputs: every leading-zero
// count, exact ties of the FP32 and FP64 roundings, both signs.
__device__ __forceinline__ u64 splitmix64(u64 x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

constexpr int kFixconvChecks = 7;

__global__ void fixconv_selftest_kernel(int64_t count, u64 seed, unsigned long long* bad) {
  unsigned long long nb[kFixconvChecks] = {};
  const float s63 = 1.0f / 9223372036854775808.0f;  // 2^-63, exact
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const u64 h = splitmix64(seed ^ (u64)i), h2 = splitmix64(h);
    u64 u;
    switch (i % 3) {
      case 0: u = h >> (i % 64); break;
      case 1: {  // a tie of the FP32 rounding
        const int k = 1 + (int)(h2 % 39);
        u = (((h | 0x800000ull) & 0xFFFFFFull) << k) | (1ull << (k - 1));
        break;
      }
      default: {  // a tie of the FP64 rounding
        const int k = 1 + (int)(h2 % 11);
        u = (((h | (1ull << 52)) & ((1ull << 53) - 1ull)) << k) | (1ull << (k - 1));
      }
    }
    if (i == 0) u = 0;
    if (i == 3) u = ~0ull;
    nb[0] += __float_as_uint(u64_to_f32<-63>(u)) != __float_as_uint(__ull2float_rn(u) * s63);
    nb[1] += __float_as_uint(u64_to_f32<0>(u)) != __float_as_uint(__ull2float_rn(u));
    nb[2] += __double_as_longlong(u64_to_f64<-63>(u)) != __double_as_longlong(__ull2double_rn(u) * (1.0 / kFixOne));
    const long long d = (long long)h2 >> (i % 64);
    nb[3] += __float_as_uint(sfix_to_f32(d)) != __float_as_uint(__ll2float_rn(d) * s63);
    // |e| < 1: exponent field 0..126, either sign
    const uint32_t eb = (uint32_t)(h2 >> 32);
    const float e = __uint_as_float((eb & 0x807FFFFFu) | ((uint32_t)((eb >> 8) % 127u) << 23));
    nb[4] += f32_to_sfix(e) != llrint((double)e * kFixOne);
    // truncation of x 2^63 for 0 <= x < 2, and floor(mu x) with mu x exact in
    // FP64 (mu a 29-bit integer times a power of two), 0 <= x <= 1
    const float x2 = __uint_as_float(((uint32_t)(h >> 32) & 0x7FFFFFu) | ((uint32_t)((h >> 13) % 128u) << 23));
    nb[5] += f32_to_ufix_trunc(x2) != __double2ull_rz((double)x2 * kFixOne);
    const float x1 = fminf(x2 * 0.5f, 1.0f);
    const u64 mu = (h2 & ((1ull << 29) - 1ull)) << (int)((h >> 40) % 35u);
    nb[6] += mul_fix_f32(mu, x1) != __double2ull_rz((double)mu * (double)x1);
  }
  for (int q = 0; q < kFixconvChecks; ++q)
    if (nb[q]) atomicAdd(&bad[q], nb[q]);
}

ppr_status fixconv_selftest(int64_t count, uint64_t seed, int64_t* out_mismatches, cudaStream_t st) {
  unsigned long long* d = nullptr;
  PPR_CUDA_TRY(cudaMalloc((void**)&d, kFixconvChecks * sizeof(unsigned long long)));
  cudaError_t e = cudaMemsetAsync(d, 0, kFixconvChecks * sizeof(unsigned long long), st);
  if (e == cudaSuccess && count > 0) {
    fixconv_selftest_kernel<<<sm_count() * 8, 256, 0, st>>>(count, seed, d);
    e = cudaGetLastError();
  }
  unsigned long long h[kFixconvChecks] = {};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_error("conversion self-test: %s", cudaGetErrorString(e));
    return PPR_ERR_CUDA;
  }
  for (int q = 0; q < kFixconvChecks; ++q) out_mismatches[q] = (int64_t)h[q];
  return PPR_OK;
}

}  // namespace ppr
