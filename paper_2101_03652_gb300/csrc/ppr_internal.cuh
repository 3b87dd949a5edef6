// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include <string>
#include <vector>

#include "ppr.h"

namespace ppr {

void set_error(const char* fmt, ...);
void clear_error();

#define PPR_CUDA_TRY(expr)                                                                        \
  do {                                                                                            \
    cudaError_t e_ = (expr);                                                                      \
    if (e_ != cudaSuccess) {                                                                      \
      ::ppr::set_error("CUDA error %s at %s:%d (%s)", cudaGetErrorString(e_), __FILE__, __LINE__, \
                       #expr);                                                                    \
      return e_ == cudaErrorMemoryAllocation ? PPR_ERR_OOM : PPR_ERR_CUDA;                        \
    }                                                                                             \
  } while (0)

#define PPR_TRY(expr)                 \
  do {                                \
    ppr_status s_ = (expr);           \
    if (s_ != PPR_OK) return s_;      \
  } while (0)

// Passes a high-precision query may run: 4 ceil(ln lambda / ln(1 - alpha)) + 64
// (four times the zero-start PowItr count of Eq. 6, plus slack), computed in
// double.  Returns -1 when that exceeds kMaxSweepsCap, i.e. when alpha is so
// small for lambda that the count would not fit the per-pass buffers.
constexpr int kMaxSweepsCap = 1 << 17;
inline int sweep_limit(double alpha, double lambda) {
  const double s = 4.0 * std::ceil(std::log(lambda) / std::log(1.0 - alpha)) + 64.0;
  return (s >= 1.0 && s <= (double)kMaxSweepsCap) ? (int)s : -1;
}

// Passes of a batch: ceil(ln(goal / F) / ln(rate)), at least 1, computed in
// double and clamped to cap + 1 so that the cast cannot overflow (a caller that
// finds more than cap passes reports the sweep limit).
inline int batch_passes(double goal, double F, double rate, int cap) {
  const double s = std::ceil(std::log(goal / F) / std::log(rate) - 1e-12);
  if (!(s >= 1.0)) return 1;
  return s > (double)cap ? cap + 1 : (int)s;
}

// Fixed-point format of the high-precision path: unsigned Q1.63, value = raw * 2^-63.
constexpr double kFixOne = 9223372036854775808.0;  // 2^63
constexpr uint64_t kFixOneRaw = 0x8000000000000000ull;

// A device allocation that grows on demand and is reused across queries.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  bool fresh = false;  // newly allocated, contents undefined (the user clears it once initialised)
  ppr_status ensure(size_t want);
  void release();
  template <class T>
  T* as() const { return static_cast<T*>(ptr); }
};

// Free device bytes as the admission checks see them: the measured value,
// capped by the host-side test hook of ppr_inject (PPR_INJECT_FREE_BYTES).
// The other hook (PPR_INJECT_ALLOC_FAIL) acts in DevBuf::ensure.
size_t admission_free_bytes(size_t free_bytes);

struct Workspace {
  DevBuf r, pi, za, zb;          // n*KT uint64 each (HP): residue, reserve, ping-pong z
  DevBuf stamp;                  // n*KT uint32 frontier membership stamps
  DevBuf front_a, front_b;       // frontier lists (n*KT uint32)
  DevBuf ent_share, ent_rem;     // per frontier entry: share and remainder of a push
  DevBuf chunks;                 // edge-chunk records of a frontier level
  DevBuf heavy_acc, heavy_cnt;   // partial sums of split rows
  DevBuf counters;               // small device counters
  DevBuf resid;                  // per-sweep per-column residual sums (double)
  DevBuf status;                 // device status word of the TMA passes (timed-out waits)
  DevBuf stage;                  // device staging for host outputs
  DevBuf walk_a, walk_b, walk_c; // APPROX path buffers
  void* pinned = nullptr;        // small pinned host buffer for readbacks
  size_t pinned_bytes = 0;
  void release();
  size_t device_bytes() const;   // device bytes held by all buffers above
  size_t hp_bytes() const;       // the part a high-precision query reuses
};

}  // namespace ppr

struct ppr_graph {
  int64_t n = 0, m = 0;
  int device = -1;
  // relabelling: nodes sorted by in-degree (descending, ties by original id)
  std::vector<int32_t> h_new_of_old;   // new id of an original id
  std::vector<int32_t> h_in_deg_sorted;  // in-degree of new id (non-increasing)
  std::vector<int32_t> h_out_deg;        // out-degree of new id
  int32_t* d_new_of_old = nullptr;     // n
  int32_t* d_old_of_new = nullptr;     // n
  int32_t* d_out_rp = nullptr;         // n+1, out-CSR in new ids (original neighbour order)
  int32_t* d_out_ci = nullptr;         // m
  int32_t* d_in_rp = nullptr;          // n+1, in-CSR in new ids (rows ascending)
  int32_t* d_in_ci = nullptr;          // m
  int32_t* d_deg = nullptr;            // n, out-degree in new ids
  // alpha-dependent per-node scale factors, cached for the last alpha used
  double cached_alpha = -1.0;
  uint64_t* d_omega = nullptr;         // round((1-alpha)/d * 2^64)
  float* d_invw = nullptr;             // d / (1-alpha)
  // heavy-row split for the pull sweep (rows with in-degree > heavy_deg)
  int32_t heavy_deg = 0, piece_edges = 0;
  int32_t n_heavy = 0, n_pieces = 0;
  int32_t* d_piece_row = nullptr;
  int32_t* d_piece_e0 = nullptr;
  int32_t* d_heavy_npieces = nullptr;
  uint32_t stamp_epoch = 0;
  // SpeedPPR-Index: endpoint (new id) of the stored walk of every out-edge slot
  int32_t* d_index = nullptr;
  uint64_t index_seed = 0;
  double index_alpha = 0.0;
  // autotuned settings per k bucket (ceil(log2 k), 0..6); 0 / negative = untuned
  int tuned_kt[7] = {0, 0, 0, 0, 0, 0, 0};
  double tuned_switch_frac[7] = {-1, -1, -1, -1, -1, -1, -1};
  float tuned_relax[7] = {0, 0, 0, 0, 0, 0, 0};  // over-relaxation of the in-place passes; 0 = default
  // per tile width: the sweep work list (index = log2 of the tile width, widths 1..64)
  struct SweepPlan {
    int kt = 0;
    int32_t n_items_all = 0, n_items_nz = 0;
    int32_t n_split = 0;          // rows cut into pieces (the first n_split rows)
    int32_t n_items_heavy = 0;    // items before the first light-row item
    int32_t u_light = 0;          // first row with at most kLightMax in-edges
    int4* d_items = nullptr;
    int32_t* d_npieces = nullptr; // pieces per split row
  } plans[7];
  // chunks of the TMA correction passes (rows [0, u_h), edges [0, h_edges))
  struct TmaPlan {
    bool built = false;
    int32_t u_h = 0, h_edges = 0, n_chunks = 0, n_slots = 0, item0 = 0;
    int4* d_chunks = nullptr;         // per chunk: {row of its first edge, row start, row end, 0}
    int32_t* d_split_slot = nullptr;  // per row < u_h: slot of a row meeting two or more chunks, else -1
    int32_t* d_split_np = nullptr;    // per slot: chunks the row meets
    float* d_split_acc = nullptr;     // per slot: 64 partial sums
    unsigned int* d_split_cnt = nullptr;
  } tma;
  ppr::Workspace ws;
};

namespace ppr {
ppr_status ensure_alpha(ppr_graph* g, double alpha, cudaStream_t st);
ppr_status query_hp(ppr_graph* g, const int32_t* src, int32_t k, const ppr_query_opts& o, double* out_pi,
                    double* out_r, ppr_stats* stats, cudaStream_t st);
ppr_status query_approx(ppr_graph* g, const int32_t* src, int32_t k, const ppr_query_opts& o, double* out_pi,
                        double* out_r, uint32_t* out_counts, ppr_stats* stats, cudaStream_t st);
ppr_status fixconv_selftest(int64_t count, uint64_t seed, int64_t* out_mismatches, cudaStream_t st);
bool is_device_pointer(const void* p);
void* device_view(void* p);
ppr_status get_plan(ppr_graph* g, int lanes, ppr_graph::SweepPlan** out, cudaStream_t st);
int sm_count();
// z0 (and x0 when not NULL) of the model's estimate for a solver tile
ppr_status warm_start_tile(const void* model, ppr_graph* g, const int32_t* src_new, int ncols, int kt, double alpha,
                           unsigned long long* z0, unsigned long long* x0, cudaStream_t st);
int warm_correction_passes(const void* model);
int64_t hp_state_bytes(const ppr_graph* g, int32_t k, int32_t kt);
int hp_tile_width(const ppr_graph* g, int32_t k, int32_t k_tile);
size_t hp_workspace_bytes(const ppr_graph* g, int kt, int max_sweeps);
int tune_bucket(int32_t k);
// x + mu q with mu = 1 - sum x: z of it, and the corrected x when x_out is not NULL
ppr_status warm_correct_tile(const void* model, ppr_graph* g, const int32_t* src_new, int ncols, int kt, double alpha,
                             const unsigned long long* x, const unsigned long long* mass, unsigned long long* z,
                             unsigned long long* x_out, cudaStream_t st);
}  // namespace ppr
