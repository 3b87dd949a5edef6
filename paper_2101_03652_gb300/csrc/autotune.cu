// Autotuner for the tile width, the queue->sweep switch threshold and the
// over-relaxation factor of the in-place correction passes.
//
// The paper fixes scanThreshold = n/4 for its CPU (Algorithm 3), a cache
// heuristic.  On the GPU the right switch point and the number of sources to
// solve together depend on the graph and on k, so both are measured: the
// calibration batch is answered with each candidate setting, timed with CUDA
// events on the caller's stream, and the fastest setting is kept in the graph
// for later calls with k_tile = 0 / switch_edges = -1 and a similar k.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ppr_internal.cuh"

using namespace ppr;

namespace ppr {
int tune_bucket(int32_t k) {
  int b = 0;
  while ((1 << b) < k && b < 6) ++b;
  return b;  // k -> ceil(log2 k), capped at 64 sources
}
}  // namespace ppr

extern "C" ppr_status ppr_autotune(ppr_graph* g, const int32_t* src, int32_t k, const ppr_query_opts* base,
                                   double* out_pi, ppr_query_opts* best, double* best_ms, void* cuda_stream) {
  clear_error();
  if (!g || !src || k < 1 || !out_pi || !best) {
    set_error("autotune needs a graph, k >= 1 calibration sources, out_pi and best");
    return PPR_ERR_ARG;
  }
  ppr_query_opts o;
  if (base) o = *base; else ppr_default_opts(&o);
  o.warm_start = nullptr;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::vector<int> kts;
  for (int kt = 1; kt <= 64; kt <<= 1) {
    kts.push_back(kt);
    if (kt >= k) break;
  }
  const double fracs[] = {0.0, 0.002, 0.02, 0.1};
  cudaEvent_t e0, e1;
  PPR_CUDA_TRY(cudaEventCreate(&e0));
  PPR_CUDA_TRY(cudaEventCreate(&e1));
  double best_t = INFINITY;
  ppr_query_opts best_o = o;
  ppr_status s = PPR_OK;
  const int b = tune_bucket(k);
  g->tuned_relax[b] = 0.f;  // widths and switches are compared at the default w
  // mean time of `reps` calls with setting c (INFINITY when one fails to
  // certify; other errors end the tuning)
  auto timed = [&](const ppr_query_opts& c, int reps) -> double {
    double sum = 0.0;
    for (int rep = 0; rep < reps; ++rep) {
      cudaEventRecord(e0, st);
      s = ppr_sssp_query(g, src, k, PPR_HP, &c, out_pi, nullptr, nullptr, nullptr, st);
      cudaEventRecord(e1, st);
      if (s == PPR_ERR_NOT_CONVERGED) {
        s = PPR_OK;
        return INFINITY;
      }
      if (s != PPR_OK) return INFINITY;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      sum += ms;
    }
    return sum / reps;
  };
  // stage 1: every width and switch, one timed call each
  std::vector<std::pair<double, ppr_query_opts>> scored;
  for (int kt : kts) {
    for (double f : fracs) {
      ppr_query_opts c = o;
      c.k_tile = kt;
      c.switch_edges = (int64_t)(f * (double)g->m * kt);
      // one untimed call allocates the workspace for this width
      s = ppr_sssp_query(g, src, k, PPR_HP, &c, out_pi, nullptr, nullptr, nullptr, st);
      if (s == PPR_ERR_ADMIT) { s = PPR_OK; break; }  // wider tiles do not fit: skip them
      if (s != PPR_OK) break;
      const double t = timed(c, 1);
      if (s != PPR_OK) break;
      scored.push_back({t, c});
    }
    if (s != PPR_OK) break;
  }
  // stage 2: the pass count of in-place passes varies by a few passes from
  // call to call, so single timings of close settings pick at random; the
  // three fastest are timed again over three calls and the best mean wins
  std::sort(scored.begin(), scored.end(),
            [](const std::pair<double, ppr_query_opts>& x, const std::pair<double, ppr_query_opts>& y) {
              return x.first < y.first;
            });
  for (size_t i = 0; i < scored.size() && i < 3 && s == PPR_OK; ++i) {
    if (!std::isfinite(scored[i].first)) break;
    const double t = timed(scored[i].second, 3);
    if (s == PPR_OK && t < best_t) {
      best_t = t;
      best_o = scored[i].second;
    }
  }
  // the over-relaxation factor for the best width and switch: the pass
  // count of the in-place passes varies from call to call (the order of
  // updates is not fixed), so each candidate is judged by its mean time over
  // three calls (a factor that stalls now and then, and falls back to plain
  // passes, loses)
  const float ws[] = {1.05f, 1.1f, 1.15f};
  float best_w = 0.f;
  double best_wt = INFINITY;
  for (int i = 0; i < 3 && s == PPR_OK && std::isfinite(best_t); ++i) {
    g->tuned_relax[b] = ws[i];
    const double t = timed(best_o, 3);  // a factor under which a call does not certify scores INFINITY
    if (s == PPR_OK && t < best_wt) {
      best_wt = t;
      best_w = ws[i];
    }
  }
  g->tuned_relax[b] = best_w;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != PPR_OK) return s;
  if (!std::isfinite(best_t)) {
    // no width and switch answered the calibration batch within max_sweeps:
    // nothing is kept, later calls use the defaults
    set_error("autotune: no candidate setting certified the calibration batch");
    return PPR_ERR_NOT_CONVERGED;
  }
  *best = best_o;
  if (best_ms) *best_ms = std::isfinite(best_wt) ? best_wt : best_t;
  g->tuned_kt[b] = best_o.k_tile;
  g->tuned_switch_frac[b] = (double)best_o.switch_edges / ((double)g->m * best_o.k_tile);
  return PPR_OK;
}
