// High-precision queries for callers that must not allocate device memory.
//
// Some hosts of this library own every byte of device memory themselves: an
// inference server or database plug-in that hands each extension a fixed
// memory budget through its own allocator, a service that has reserved all
// free memory in a caching pool up front, or a latency-critical loop that
// forbids allocation (and its failure modes) after start-up.  Such callers
// cannot let ppr_sssp_query grow its workspace with cudaMalloc.  The entry
// point below answers the same high-precision queries with a simpler variant
// of the pull sweep whose scratch lives in one file-scope device array of
// fixed size; it calls no allocation routine.
//
// Limits: the scratch holds three n x k_tile arrays of 8-byte cells plus the
// per-pass residual sums, so n * k_tile * 24 bytes plus a few kilobytes must
// fit in kNoAllocScratchBytes (16 MiB): about 87,000 nodes at k_tile = 8, or
// 690,000 nodes one source at a time.  Larger graphs are rejected with
// PPR_ERR_ARG.  Every GPU that loads the library keeps this array until the
// process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "ppr_internal.cuh"
#include "sweep_kernel.cuh"

namespace ppr {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;

// The scratch.  Host code cannot use this name as a device address (on the
// host it denotes a shadow object); its device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_addr[64];

// Device address of the scratch on the current device (resolved on first use
// with that device current).
static ppr_status noalloc_scratch(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d out of range for the no-allocation entry point", dev);
    return PPR_ERR_ARG;
  }
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      set_error("cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
      return PPR_ERR_CUDA;
    }
    g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_addr[dev];
  return PPR_OK;
}

struct NaArgs {
  int32_t n;
  const int32_t* in_rp;
  const int32_t* in_ci;
  const uint64_t* omega;
  const float* invw;
  const u64* z_in;
  u64* z_out;
  u64* x_out;
  int32_t src[8];
  u64 alpha_raw;
  double* resid;
};

// One pass x' = alpha e_s + (1-alpha) x P for a tile of KT sources: one warp
// per in-CSR row (grid-stride), z = (1-alpha) x / d stored for the next pass.
template <int KT>
__global__ void __launch_bounds__(256) noalloc_sweep_kernel(NaArgs a) {
  constexpr int V = Lay<KT>::V, L = Lay<KT>::L, EPW = Lay<KT>::EPW;
  const int lane = threadIdx.x & 31;
  const int slot = lane % L;
  float res[V];
#pragma unroll
  for (int q = 0; q < V; ++q) res[q] = 0.f;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < a.n; u += nw) {
    u64 acc[V] = {};
    const int e1 = a.in_rp[u + 1];
    for (int e = a.in_rp[u] + lane / L; e < e1; e += EPW) {
      u64 t[V];
      ld_vec<V>(a.z_in + (size_t)a.in_ci[e] * KT + slot * V, t);
#pragma unroll
      for (int q = 0; q < V; ++q) acc[q] += t[q];
    }
#pragma unroll
    for (int off = L; off < 32; off <<= 1)
#pragma unroll
      for (int q = 0; q < V; ++q) acc[q] += __shfl_xor_sync(kFull, acc[q], off);
    if (lane < L) {
      const u64 om = a.omega[u];
      const float iw = a.invw[u];
      u64 zo[V], zn[V], xn[V];
      ld_vec<V>(a.z_in + (size_t)u * KT + slot * V, zo);
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const int c = slot * V + q;
        xn[q] = acc[q] + (u == a.src[c] ? a.alpha_raw : 0ull);
        zn[q] = mulhi_round(xn[q], om);
        const u64 dz = zn[q] > zo[q] ? zn[q] - zo[q] : zo[q] - zn[q];
        res[q] += (float)dz * iw;
      }
      st_vec<V>(a.z_out + (size_t)u * KT + slot * V, zn);
      if (a.x_out) st_vec<V>(a.x_out + (size_t)u * KT + slot * V, xn);
    }
  }
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
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += (double)sred[w][threadIdx.x];
    atomicAdd(&a.resid[threadIdx.x], s);
  }
}

template <int KT>
__global__ void noalloc_output_kernel(int64_t n, const int32_t* __restrict__ new_of_old, const u64* __restrict__ x,
                                      int ncols, int64_t col0, double* __restrict__ out) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = new_of_old[o];
    for (int c = 0; c < ncols; ++c) out[(col0 + c) * n + o] = (double)x[u * KT + c] * (1.0 / kFixOne);
  }
}

template <int KT>
static ppr_status run_noalloc(ppr_graph* g, const int32_t* src, int32_t k, double alpha, double lambda,
                              double* out_pi, int32_t* out_sweeps, cudaStream_t st) {
  const int64_t n = g->n, m = g->m;
  const size_t cells = (size_t)n * KT;
  const int max_sweeps = sweep_limit(alpha, lambda);
  if (max_sweeps < 1) {
    set_error("alpha %g is too small for lambda %g: more than %d passes", alpha, lambda, kMaxSweepsCap);
    return PPR_ERR_ARG;
  }
  const size_t need = 3 * cells * 8 + (size_t)(max_sweeps + 1) * KT * 8;
  if (need > kNoAllocScratchBytes) {
    set_error("graph too large for the no-allocation entry point: %zu bytes of scratch needed "
              "(n * k_tile * 24 plus residual sums), %zu available",
              need, kNoAllocScratchBytes);
    return PPR_ERR_ARG;
  }
  int dev = 0;
  PPR_CUDA_TRY(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  PPR_TRY(noalloc_scratch(dev, &base));
  u64* za = reinterpret_cast<u64*>(base);
  u64* zb = za + cells;
  u64* xb = zb + cells;
  double* resid = reinterpret_cast<double*>(xb + cells);
  PPR_TRY(ensure_alpha(g, alpha, st));
  const u64 alpha_raw = (u64)(alpha * kFixOne);
  int sms = 0;
  PPR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = std::max(sms, 1) * 8;
  const double slack = (double)m * 0.5 / kFixOne / alpha;
  for (int32_t t0 = 0; t0 < k; t0 += KT) {
    const int ncols = std::min<int32_t>(KT, k - t0);
    NaArgs na;
    na.n = (int32_t)n;
    na.in_rp = g->d_in_rp;
    na.in_ci = g->d_in_ci;
    na.omega = g->d_omega;
    na.invw = g->d_invw;
    na.alpha_raw = alpha_raw;
    for (int c = 0; c < 8; ++c) na.src[c] = c < ncols ? g->h_new_of_old[src[t0 + c]] : -1;
    // the scratch keeps the previous call's contents: the zero start and the
    // residual accumulators are cleared for every tile
    PPR_CUDA_TRY(cudaMemsetAsync(za, 0, cells * 8, st));
    PPR_CUDA_TRY(cudaMemsetAsync(resid, 0, (size_t)(max_sweeps + 1) * KT * 8, st));
    u64* zcur = za;
    u64* znext = zb;
    int sweeps = 0;
    double R = 1.0;  // ||r(x0)||_1 of the zero start
    while (true) {
      const int S = R <= lambda ? 1 : batch_passes(lambda, R, 1.0 - alpha, max_sweeps);
      if (sweeps + S > max_sweeps) {
        set_error("sweep limit %d reached", max_sweeps);
        return PPR_ERR_NOT_CONVERGED;
      }
      for (int j = 0; j < S; ++j) {
        na.z_in = zcur;
        na.z_out = znext;
        na.x_out = j == S - 1 ? xb : nullptr;
        na.resid = resid + (size_t)(sweeps + j) * KT;
        noalloc_sweep_kernel<KT><<<grid, 256, 0, st>>>(na);
        std::swap(zcur, znext);
      }
      PPR_CUDA_TRY(cudaGetLastError());
      sweeps += S;
      double D[KT];
      PPR_CUDA_TRY(cudaMemcpyAsync(D, resid + (size_t)(sweeps - 1) * KT, sizeof(D), cudaMemcpyDeviceToHost, st));
      PPR_CUDA_TRY(cudaStreamSynchronize(st));
      bool ok = true;
      R = 0.0;
      for (int c = 0; c < ncols; ++c) {
        const double bound = (1.0 - alpha) * (D[c] / kFixOne / alpha) * (1.0 + 1e-4) + 2.0 * slack;
        if (bound > lambda) ok = false;
        R = std::max(R, bound);
      }
      if (ok) break;
    }
    noalloc_output_kernel<KT><<<grid, 256, 0, st>>>(n, g->d_new_of_old, xb, ncols, t0, out_pi);
    PPR_CUDA_TRY(cudaGetLastError());
    if (out_sweeps)
      for (int c = 0; c < ncols; ++c) out_sweeps[t0 + c] = sweeps;
  }
  PPR_CUDA_TRY(cudaStreamSynchronize(st));
  return PPR_OK;
}

}  // namespace ppr

using namespace ppr;

extern "C" ppr_status ppr_sssp_query_noalloc(ppr_graph* g, const int32_t* src, int32_t k, double alpha,
                                             double lambda, double* out_pi, int32_t* out_sweeps,
                                             void* cuda_stream) {
  clear_error();
  if (!g || !src || !out_pi || k < 1) {
    set_error("graph, src and out_pi must be non-NULL and k >= 1");
    return PPR_ERR_ARG;
  }
  if (!(alpha > 0.0 && alpha < 1.0) || !(lambda >= 1e-15 && lambda < 1.0)) {
    set_error("alpha must lie in (0, 1) and lambda in [1e-15, 1)");
    return PPR_ERR_ARG;
  }
  for (int32_t i = 0; i < k; ++i)
    if (src[i] < 0 || src[i] >= g->n) {
      set_error("source %d = %d outside [0, n)", i, src[i]);
      return PPR_ERR_ARG;
    }
  if (!is_device_pointer(out_pi)) {
    set_error("out_pi must be device memory for the no-allocation entry point");
    return PPR_ERR_ARG;
  }
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    (void)cudaGetLastError();
    set_error("no CUDA device available");
    return PPR_ERR_CUDA;
  }
  if (cur != g->device) PPR_CUDA_TRY(cudaSetDevice(g->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  ppr_status s;
  if (k >= 8) s = run_noalloc<8>(g, src, k, alpha, lambda, out_pi, out_sweeps, st);
  else if (k >= 4) s = run_noalloc<4>(g, src, k, alpha, lambda, out_pi, out_sweeps, st);
  else if (k >= 2) s = run_noalloc<2>(g, src, k, alpha, lambda, out_pi, out_sweeps, st);
  else s = run_noalloc<1>(g, src, k, alpha, lambda, out_pi, out_sweeps, st);
  if (cur != g->device) cudaSetDevice(cur);
  return s;
}
