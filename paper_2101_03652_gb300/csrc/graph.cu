// Graph store: validation of the CSR contract, relabelling by in-degree,
// construction of the in-CSR (transpose) and upload to the device.
//
// The paper stores node ids sorted and concatenates the adjacency lists in id
// order so that a full scan of the edge array is sequential (Sec. 5, "Global
// Sequential Scan").  Here the pull sweeps read the in-adjacency row by row,
// and rows are renumbered by decreasing in-degree so that rows of similar
// length sit next to each other: one sweep kernel can then give long rows to
// whole warps and short rows to small lane groups with little divergence, and
// the most frequently gathered nodes (in R-MAT, in- and out-degree are
// strongly correlated) occupy a small, cache-friendly id range.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <thread>

#include "ppr_internal.cuh"

namespace ppr {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}
void clear_error() { g_last_error.clear(); }
const char* last_error_cstr() { return g_last_error.c_str(); }

static std::atomic<int64_t> g_inject_free{-1};
static std::atomic<int64_t> g_inject_alloc{0};

size_t admission_free_bytes(size_t free_bytes) {
  const int64_t cap = g_inject_free.load();
  return cap >= 0 ? std::min(free_bytes, (size_t)cap) : free_bytes;
}

ppr_status DevBuf::ensure(size_t want) {
  if (want <= bytes && ptr) return PPR_OK;
  release();
  if (want == 0) return PPR_OK;
  if (g_inject_alloc.load() > 0 && g_inject_alloc.fetch_sub(1) == 1) {
    set_error("device allocation of %zu bytes failed: injected allocation failure", want);
    return PPR_ERR_OOM;
  }
  cudaError_t e = cudaMalloc(&ptr, want);
  if (e != cudaSuccess) {
    ptr = nullptr;
    bytes = 0;
    (void)cudaGetLastError();
    set_error("device allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
    return PPR_ERR_OOM;
  }
  bytes = want;
  fresh = true;
  return PPR_OK;
}
void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}
size_t Workspace::device_bytes() const {
  size_t b = 0;
  for (const DevBuf* d : {&r, &pi, &za, &zb, &stamp, &front_a, &front_b, &ent_share, &ent_rem, &chunks, &heavy_acc,
                          &heavy_cnt, &counters, &resid, &status, &stage, &walk_a, &walk_b, &walk_c})
    b += d->bytes;
  return b;
}

size_t Workspace::hp_bytes() const {
  size_t b = 0;
  for (const DevBuf* d : {&r, &pi, &za, &zb, &stamp, &front_a, &front_b, &ent_share, &ent_rem, &chunks, &heavy_acc,
                          &heavy_cnt, &counters, &resid, &status, &stage})
    b += d->bytes;
  return b;
}

void Workspace::release() {
  for (DevBuf* b : {&r, &pi, &za, &zb, &stamp, &front_a, &front_b, &ent_share, &ent_rem, &chunks, &heavy_acc,
                    &heavy_cnt, &counters, &resid, &status, &stage, &walk_a, &walk_b, &walk_c})
    b->release();
  if (pinned) cudaFreeHost(pinned);
  pinned = nullptr;
  pinned_bytes = 0;
}

// Address kernels can write an output through: device or managed memory as
// is; page-locked host memory through its mapped device address (on a
// Grace-Blackwell node the GPU writes it over the coherent CPU-GPU link, so
// no staging copy is needed); NULL for pageable host memory, which is staged.
void* device_view(void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return a.devicePointer;
  return nullptr;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// per-node scale factors for alpha: omega = round((1-alpha) 2^64 / d), invw = d/(1-alpha)
__global__ void alpha_scale_kernel(int64_t n, const int32_t* __restrict__ deg, uint64_t one_minus_alpha_64,
                                   float inv_one_minus_alpha, uint64_t* omega, float* invw) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    uint64_t d = (uint64_t)deg[u];
    omega[u] = (one_minus_alpha_64 + d / 2) / d;
    invw[u] = (float)d * inv_one_minus_alpha;
  }
}

ppr_status ensure_alpha(ppr_graph* g, double alpha, cudaStream_t st) {
  if (g->cached_alpha == alpha) return PPR_OK;
  // (1-alpha) * 2^64 is exact in double arithmetic and below 2^64 for alpha in (0,1)
  uint64_t oma = (uint64_t)((1.0 - alpha) * 18446744073709551616.0);
  alpha_scale_kernel<<<1216, 256, 0, st>>>(g->n, g->d_deg, oma, (float)(1.0 / (1.0 - alpha)), g->d_omega,
                                            g->d_invw);
  PPR_CUDA_TRY(cudaGetLastError());
  g->cached_alpha = alpha;
  return PPR_OK;
}

}  // namespace ppr

using namespace ppr;

static ppr_status validate_csr(const int64_t* rp, const int32_t* ci, int64_t n, int64_t m) {
  if (rp[0] != 0 || rp[n] != m) {
    set_error("row_ptr[0] must be 0 and row_ptr[n] must equal m (%lld)", (long long)m);
    return PPR_ERR_GRAPH;
  }
  int threads = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<int64_t> bad(threads, -1);
  std::vector<std::thread> th;
  for (int t = 0; t < threads; ++t) {
    th.emplace_back([&, t] {
      int64_t lo = n * t / threads, hi = n * (t + 1) / threads;
      for (int64_t v = lo; v < hi && bad[t] < 0; ++v) {
        int64_t a = rp[v], b = rp[v + 1];
        if (b <= a || a < 0 || b > m) { bad[t] = v; break; }
        for (int64_t e = a; e < b; ++e) {
          int32_t u = ci[e];
          if (u < 0 || u >= n || u == v || (e > a && u <= ci[e - 1])) { bad[t] = v; break; }
        }
      }
    });
  }
  for (auto& x : th) x.join();
  for (int t = 0; t < threads; ++t)
    if (bad[t] >= 0) {
      set_error("node %lld violates the graph contract (out-degree >= 1, ids in range, rows sorted, "
                "no duplicates, no self-loops)", (long long)bad[t]);
      return PPR_ERR_GRAPH;
    }
  return PPR_OK;
}

template <class T>
static ppr_status upload(T** dst, const T* src, size_t count, cudaStream_t st) {
  PPR_CUDA_TRY(cudaMalloc((void**)dst, sizeof(T) * std::max<size_t>(count, 1)));
  PPR_CUDA_TRY(cudaMemcpyAsync(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice, st));
  return PPR_OK;
}

static void free_graph_arrays(ppr_graph* g) {
  for (void* p : {(void*)g->d_new_of_old, (void*)g->d_old_of_new, (void*)g->d_out_rp, (void*)g->d_out_ci,
                  (void*)g->d_in_rp, (void*)g->d_in_ci, (void*)g->d_deg, (void*)g->d_omega, (void*)g->d_invw,
                  (void*)g->d_piece_row, (void*)g->d_piece_e0, (void*)g->d_heavy_npieces, (void*)g->d_index})
    if (p) cudaFree(p);
  for (auto& pl : g->plans) {
    if (pl.d_items) cudaFree(pl.d_items);
    if (pl.d_npieces) cudaFree(pl.d_npieces);
  }
  for (void* p : {(void*)g->tma.d_chunks, (void*)g->tma.d_split_slot, (void*)g->tma.d_split_np,
                  (void*)g->tma.d_split_acc, (void*)g->tma.d_split_cnt})
    if (p) cudaFree(p);
}

static ppr_status build_and_upload(ppr_graph* g, const int64_t* rp, const int32_t* ci, cudaStream_t st) {
  const int64_t n = g->n, m = g->m;
  // in-degrees and the relabelling
  std::vector<int32_t> indeg(n, 0);
  for (int64_t e = 0; e < m; ++e) indeg[ci[e]]++;
  std::vector<int32_t> old_of_new(n);
  std::iota(old_of_new.begin(), old_of_new.end(), 0);
  std::stable_sort(old_of_new.begin(), old_of_new.end(),
                   [&](int32_t a, int32_t b) { return indeg[a] > indeg[b]; });
  g->h_new_of_old.assign(n, 0);
  for (int64_t i = 0; i < n; ++i) g->h_new_of_old[old_of_new[i]] = (int32_t)i;
  const std::vector<int32_t>& nw = g->h_new_of_old;
  g->h_in_deg_sorted.resize(n);
  for (int64_t i = 0; i < n; ++i) g->h_in_deg_sorted[i] = indeg[old_of_new[i]];

  // out-CSR in new ids; each row keeps the caller's neighbour order (walks
  // pick the k-th out-neighbour, so the order is part of the walk definition)
  std::vector<int32_t> out_rp(n + 1, 0), deg(n);
  for (int64_t i = 0; i < n; ++i) {
    int64_t v = old_of_new[i];
    deg[i] = (int32_t)(rp[v + 1] - rp[v]);
    out_rp[i + 1] = out_rp[i] + deg[i];
  }
  g->h_out_deg = deg;
  std::vector<int32_t> out_ci(m);
  {
    int threads = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (int t = 0; t < threads; ++t)
      th.emplace_back([&, t] {
        for (int64_t i = n * t / threads; i < n * (t + 1) / threads; ++i) {
          int64_t v = old_of_new[i];
          int64_t w = out_rp[i];
          for (int64_t e = rp[v]; e < rp[v + 1]; ++e) out_ci[w++] = nw[ci[e]];
        }
      });
    for (auto& x : th) x.join();
  }
  // in-CSR (transpose) in new ids; rows ascending because sources are visited in order
  std::vector<int32_t> in_rp(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) in_rp[i + 1] = in_rp[i] + g->h_in_deg_sorted[i];
  std::vector<int32_t> in_ci(m), fill(in_rp.begin(), in_rp.end() - 1);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = out_rp[i]; e < out_rp[i + 1]; ++e) in_ci[fill[out_ci[e]]++] = (int32_t)i;

  PPR_TRY(upload(&g->d_new_of_old, nw.data(), n, st));
  PPR_TRY(upload(&g->d_old_of_new, old_of_new.data(), n, st));
  PPR_TRY(upload(&g->d_out_rp, out_rp.data(), n + 1, st));
  PPR_TRY(upload(&g->d_out_ci, out_ci.data(), m, st));
  PPR_TRY(upload(&g->d_in_rp, in_rp.data(), n + 1, st));
  PPR_TRY(upload(&g->d_in_ci, in_ci.data(), m, st));
  PPR_TRY(upload(&g->d_deg, deg.data(), n, st));
  PPR_CUDA_TRY(cudaMalloc((void**)&g->d_omega, sizeof(uint64_t) * n));
  PPR_CUDA_TRY(cudaMalloc((void**)&g->d_invw, sizeof(float) * n));

  // rows with in-degree above heavy_deg are split into pieces of piece_edges in-edges
  g->heavy_deg = 2048;
  g->piece_edges = 1024;
  int32_t nh = 0;
  while (nh < n && g->h_in_deg_sorted[nh] > g->heavy_deg) ++nh;
  std::vector<int32_t> prow, pe0, npieces(std::max(nh, 1), 0);
  for (int32_t u = 0; u < nh; ++u)
    for (int64_t e = in_rp[u]; e < in_rp[u + 1]; e += g->piece_edges) {
      prow.push_back(u);
      pe0.push_back((int32_t)e);
      npieces[u]++;
    }
  g->n_heavy = nh;
  g->n_pieces = (int32_t)prow.size();
  PPR_TRY(upload(&g->d_piece_row, prow.data(), prow.size(), st));
  PPR_TRY(upload(&g->d_piece_e0, pe0.data(), pe0.size(), st));
  PPR_TRY(upload(&g->d_heavy_npieces, npieces.data(), npieces.size(), st));
  PPR_CUDA_TRY(cudaStreamSynchronize(st));
  return PPR_OK;
}

extern "C" {

void ppr_default_opts(ppr_query_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->alpha = 0.2;
  o->lambda = 1e-8;
  o->eps = 0.5;
  o->mu = 0.0;
  o->seed = 0x5eedull;
  o->k_tile = 0;
  o->epoch_num = 0;
  o->switch_edges = -1;
  o->max_sweeps = 0;
  o->warm_start = nullptr;
}

ppr_status ppr_graph_load(const int64_t* row_ptr, const int32_t* col_idx, int64_t n, int64_t m,
                          void* cuda_stream, ppr_graph** out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return PPR_ERR_ARG; }
  *out = nullptr;
  if (!row_ptr || !col_idx || n < 1) { set_error("row_ptr/col_idx NULL or n < 1"); return PPR_ERR_ARG; }
  if (n >= (int64_t)1 << 31 || m < n || m >= (int64_t)1 << 31) {
    set_error("need n <= m < 2^31 (n=%lld m=%lld)", (long long)n, (long long)m);
    return PPR_ERR_GRAPH;
  }
  PPR_TRY(validate_csr(row_ptr, col_idx, n, m));
  int dev = -1, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1 || cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    set_error("no CUDA device available");
    return PPR_ERR_CUDA;
  }
  ppr_graph* g = new ppr_graph();
  g->n = n;
  g->m = m;
  g->device = dev;
  ppr_status s = build_and_upload(g, row_ptr, col_idx, (cudaStream_t)cuda_stream);
  if (s != PPR_OK) {
    free_graph_arrays(g);
    delete g;
    return s;
  }
  *out = g;
  return PPR_OK;
}

void ppr_free(ppr_graph* g) {
  if (!g) return;
  cudaDeviceSynchronize();
  free_graph_arrays(g);
  g->ws.release();
  delete g;
}

ppr_status ppr_inject(int32_t hook, int64_t value) {
  clear_error();
  if (hook == PPR_INJECT_FREE_BYTES) {
    g_inject_free.store(value < 0 ? -1 : value);
    return PPR_OK;
  }
  if (hook == PPR_INJECT_ALLOC_FAIL) {
    g_inject_alloc.store(value < 0 ? 0 : value);
    return PPR_OK;
  }
  set_error("unknown injection hook %d", hook);
  return PPR_ERR_ARG;
}

int64_t ppr_workspace_bytes(const ppr_graph* g) { return g ? (int64_t)g->ws.device_bytes() : -1; }

ppr_status ppr_selftest_fixconv(int64_t count, uint64_t seed, int64_t* out_mismatches, void* cuda_stream) {
  clear_error();
  if (count < 0 || !out_mismatches) {
    set_error("conversion self-test needs count >= 0 and out_mismatches");
    return PPR_ERR_ARG;
  }
  return fixconv_selftest(count, seed, out_mismatches, (cudaStream_t)cuda_stream);
}

int64_t ppr_graph_n(const ppr_graph* g) { return g ? g->n : 0; }
int64_t ppr_graph_m(const ppr_graph* g) { return g ? g->m : 0; }

}  // extern "C"
