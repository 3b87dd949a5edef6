// C entry points: argument checking, device selection and mode dispatch.
#include <cmath>
#include <cstring>

#include "ppr_internal.cuh"

namespace ppr {
const char* last_error_cstr();
}
using namespace ppr;

extern "C" {

const char* ppr_last_error(void) { return last_error_cstr(); }

int64_t ppr_query_state_bytes(const ppr_graph* g, int32_t k, int32_t k_tile) {
  if (!g || k < 1 || k_tile < 0 || k_tile > 64 || (k_tile & (k_tile - 1))) return -1;
  return hp_state_bytes(g, k, k_tile);
}

ppr_status ppr_sssp_query(ppr_graph* g, const int32_t* src, int32_t k, ppr_mode mode, const ppr_query_opts* opts,
                          double* out_pi, double* out_r, uint32_t* out_walk_counts, ppr_stats* stats,
                          void* cuda_stream) {
  clear_error();
  if (!g || !src || !out_pi || k < 1) {
    set_error("graph, src and out_pi must be non-NULL and k >= 1");
    return PPR_ERR_ARG;
  }
  ppr_query_opts o;
  if (opts) o = *opts; else ppr_default_opts(&o);
  if (!(o.alpha > 0.0 && o.alpha < 1.0)) { set_error("alpha must lie in (0, 1)"); return PPR_ERR_ARG; }
  if (o.max_sweeps < 0 || o.switch_edges < -1) { set_error("max_sweeps/switch_edges out of range"); return PPR_ERR_ARG; }
  for (int32_t i = 0; i < k; ++i)
    if (src[i] < 0 || src[i] >= g->n) {
      set_error("source %d = %d outside [0, n)", i, src[i]);
      return PPR_ERR_ARG;
    }
  if (mode == PPR_HP) {
    if (!(o.lambda > 0.0 && o.lambda < 1.0) || !std::isfinite(o.lambda) || o.lambda < 1e-15) {
      set_error("lambda must lie in [1e-15, 1)");
      return PPR_ERR_ARG;
    }
    if (o.epoch_num < 0 || o.epoch_num > 64) { set_error("epoch_num must lie in [0, 64]"); return PPR_ERR_ARG; }
    if (o.epoch_num > 0 && o.warm_start) { set_error("epoch_num and warm_start exclude each other"); return PPR_ERR_ARG; }
    if ((o.flags & PPR_FLAG_NO_ACTIVE) && o.epoch_num == 0) {
      set_error("PPR_FLAG_NO_ACTIVE needs the residue form: set epoch_num > 0");
      return PPR_ERR_ARG;
    }
    if (out_walk_counts) { set_error("walk counts exist only in APPROX mode"); return PPR_ERR_ARG; }
  } else if (mode == PPR_APPROX) {
    if (!(o.eps > 0.0) || !std::isfinite(o.eps)) { set_error("eps must be > 0"); return PPR_ERR_ARG; }
    if (o.mu < 0.0 || o.mu > 1.0) { set_error("mu must lie in [0, 1] (0 means 1/n)"); return PPR_ERR_ARG; }
    if (o.warm_start) { set_error("warm_start applies to HP mode only"); return PPR_ERR_ARG; }
  } else {
    set_error("unknown mode %d", (int)mode);
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
  ppr_status s = mode == PPR_HP ? query_hp(g, src, k, o, out_pi, out_r, stats, st)
                                : query_approx(g, src, k, o, out_pi, out_r, out_walk_counts, stats, st);
  if (cur != g->device) cudaSetDevice(cur);
  return s;
}

}  // extern "C"
