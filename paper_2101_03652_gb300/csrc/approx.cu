// Approximate SSPPR (SpeedPPR, Algorithm 4).
#include "ppr_internal.cuh"

namespace ppr {

ppr_status query_approx(ppr_graph* g, const int32_t* src, int32_t k, const ppr_query_opts& o, double* out_pi,
                        double* out_r, uint32_t* out_counts, ppr_stats* stats, cudaStream_t st) {
  (void)g; (void)src; (void)k; (void)o; (void)out_pi; (void)out_r; (void)out_counts; (void)stats; (void)st;
  set_error("APPROX mode is not built yet");
  return PPR_ERR_ARG;
}

}  // namespace ppr
