/*
 * ppr.h — C ABI of the GB300 single-source Personalized PageRank library.
 *
 * Method: Wu, Gan, Wei, Zhang, "Unifying the Global and Local Approaches: An
 * Efficient Power Iteration with Forward Push", SIGMOD'21 (arXiv 2101.03652).
 *
 *   PPR pi(s, t): probability that an alpha-random walk from s stops at t
 *   (Sec. 2); the vector pi_s solves pi_s = alpha e_s + (1-alpha) pi_s P (Eq. 1)
 *   with P_v = A_v / d_v.
 *   HP-SSPPR (Sec. 2): return pi_hat with ||pi_hat - pi_s||_1 <= lambda.
 *   Approx-SSPPR (Sec. 2): |pi_hat(s,v) - pi(s,v)| <= eps pi(s,v) for every
 *   pi(s,v) >= mu, with probability 1 - 1/n (SpeedPPR, Algorithm 4).
 *
 * Graphs are directed CSR: row_ptr int64[n+1] (row_ptr[0] = 0, non-decreasing),
 * col_idx int32[m], out-neighbours of v in col_idx[row_ptr[v] .. row_ptr[v+1]).
 * Every node needs out-degree >= 1 (no dead ends, Sec. 2); rows must be sorted
 * ascending with no duplicates and no self-loops; m < 2^31.
 *
 * All functions return a ppr_status (negative on error); ppr_last_error()
 * gives a thread-local message.  On PPR_ERR_ARG / PPR_ERR_GRAPH nothing is
 * written.  The library never falls back to the CPU: without a usable CUDA
 * device every call returns PPR_ERR_CUDA.
 */
#ifndef PPR_GB300_H
#define PPR_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ppr_graph ppr_graph; /* opaque; owns the device copy of the graph */

typedef enum {
  PPR_OK = 0,
  PPR_ERR_ARG = -1,           /* bad argument (range, null pointer, unknown mode) */
  PPR_ERR_GRAPH = -2,         /* graph violates the CSR / no-dead-end contract */
  PPR_ERR_OOM = -3,           /* device or host allocation failed */
  PPR_ERR_NOT_CONVERGED = -4, /* a bounded device loop hit its limit */
  PPR_ERR_CUDA = -5,          /* CUDA runtime error or no device */
  PPR_ERR_ADMIT = -6          /* not enough free device memory for the batch state */
} ppr_status;

#define PPR_FLAG_PARTIAL 1 /* HP: stop after max_sweeps passes, uncertified */
#define PPR_FLAG_INDEX 4   /* APPROX: read the walks from the index of ppr_index_build */
#define PPR_FLAG_SYNC 2    /* HP: every pass synchronous (SimFwdPush, equal to PowItr by Lemma 1);
                              by default passes run in place except the certifying last
                              pass of each batch (asynchronous updates, Sec. 5) */
#define PPR_FLAG_NO_ACTIVE 16 /* HP, with epoch_num > 0: end in a state where no node is
                              active w.r.t. r_max = lambda/m (the Remark after Algorithm 3):
                              the queue phase runs until its frontier is empty instead of
                              stopping at sum r <= lambda, and after the epochs thresholded
                              passes at lambda/m continue until no node is active.  With a
                              switch_edges that no level reaches, the call is FIFO-FwdPush
                              (Algorithm 2) by levels on the GPU */
#define PPR_FLAG_FP32_ONLY 32 /* HP: correction passes with FP32 z_e only (no BF16 stage) */
#define PPR_FLAG_TMA_GATHER 64 /* HP: in the FP32 correction passes of 64-source tiles, two
                              warps of each block gather the rows with more than 16 in-edges
                              by TMA (four-row tile::gather4 copies into shared memory) while
                              the other warps take the light rows with vector loads.  Same
                              answers; on R-MAT graphs slower than the default, where every
                              warp gathers with per-lane 16-byte loads (0.54 against 0.33 ms
                              per pass at scale 20, 2.2 against 1.5 ms at scale 22) */
#define PPR_FLAG_FIXED_PASSES 8 /* HP: every pass in Q1.63.  By default the dense phase
                              solves for the remaining error e = pi - X with BF16 and FP32 passes,
                              folds e into the Q1.63 estimate X and certifies with one
                              exact synchronous Q1.63 pass (iterative refinement); the
                              bound and its guarantee are the same either way */

typedef enum {
  PPR_HP = 0,     /* high precision: ||pi_hat - pi||_1 <= lambda (PowerPush, Algorithm 3) */
  PPR_APPROX = 1  /* approximate: SpeedPPR, Algorithm 4 (FP32 push + Philox walks) */
} ppr_mode;

typedef struct {
  double alpha;            /* stop probability of the alpha-random walk, in (0,1) (Sec. 2) */
  double lambda;           /* HP l1 target, > 0 (Sec. 2 uses min(1/m, 1e-8)) */
  double eps;              /* APPROX relative error, > 0 */
  double mu;               /* APPROX value threshold; 0 means 1/n */
  uint64_t seed;           /* APPROX: Philox-4x32-10 key for the walks */
  int32_t k_tile;          /* sources solved together per pass: 1,2,4,...,64; 0 = auto */
  int32_t epoch_num;       /* dense phase: 0 = push every node each sweep (SimFwdPush,
                              Sec. 4.1); >0 = Algorithm 3's epochs with thresholds
                              lambda^(i/epoch_num)/m */
  int64_t switch_edges;    /* queue->sweep switch (Algorithm 3 line "Q.size() <=
                              scanThreshold"): switch once a frontier level holds more
                              than this many out-edges over the tile; -1 = auto, 0 = no
                              queue phase (sweeps from the start) */
  int32_t max_sweeps;      /* bound on dense sweeps; 0 = 4*ceil(ln lambda/ln(1-alpha))+64;
                              at most 131072 (a larger bound, or an alpha so small that
                              the default exceeds it, is PPR_ERR_ARG) */
  int32_t flags;           /* OR of the PPR_FLAG_* bits above.  PPR_FLAG_PARTIAL (HP)
                              returns the estimate after exactly max_sweeps passes
                              without certifying lambda (the stats' final_l1_residual
                              is then the bound reached) */
  const void* warm_start;  /* HP only: a ppr_model* of the same graph, or NULL for the
                              zero start.  A model without correction passes supplies
                              the start (the queue phase is skipped); a model with
                              correction passes L adds its correction after the first
                              L passes of the dense phase */
} ppr_query_opts;

typedef struct {
  int32_t sweeps;              /* dense passes run for this source's tile (correction and
                                  exact passes together in the default HP mode) */
  int32_t levels;              /* frontier levels (queue phase) */
  int64_t edges_pushed;        /* out-edges scattered in the queue phase (this source) */
  int64_t edges_swept;         /* in-edges gathered by dense sweeps (m per sweep) */
  int64_t walks;               /* APPROX: random walks started */
  int64_t walk_steps;          /* APPROX: total walk moves */
  double initial_l1_residual;  /* ||r||_1 when the dense phase started */
  double final_l1_residual;    /* certified bound on ||pi - pi_hat||_1 (HP) */
  double mass_deficit;         /* 1 - sum(pi_hat) = sum(pi - pi_hat), so |mass_deficit| is at
                                  most final_l1_residual (it equals ||r||_1 when the answer is
                                  a push reserve, e.g. a queue-only or epoch query) */
  double ms_push;               /* device time of the queue phase (whole call) */
  double ms_sweep;              /* device time of the sweep kernels alone (whole call) */
  double ms_walk;               /* APPROX: device time of the walk phase */
  double ms_total;              /* device time of the whole call */
  int64_t kernel_launches;      /* kernels this call launched */
  int64_t sweep_launches;       /* of which sweep-kernel launches */
  double W;                     /* APPROX: walk budget of Eq. 8 (natural log) */
  int32_t fp32_passes;          /* HP: of `sweeps`, correction passes with FP32 z_e */
  int32_t refine_cycles;        /* HP: fold + exact-pass cycles of the refinement */
  double ms_fp32;               /* HP: device time of the FP32 correction passes (part of ms_sweep) */
  int32_t bf16_passes;          /* HP: of `sweeps`, correction passes with BF16 z_e (the rest
                                   of `sweeps` are Q1.63) */
  int32_t reserved;
  double ms_bf16;               /* HP: device time of the BF16 correction passes (part of ms_sweep) */
  double relax;                 /* HP: over-relaxation factor w of the in-place correction passes
                                   at the end of the call (the autotuner's choice for the graph,
                                   else 1.15; 1 when no in-place pass ran or a stalled batch
                                   turned it off) */
} ppr_stats;

/* Fill opts with defaults: alpha 0.2, lambda 1e-8, eps 0.5, mu 0 (=1/n),
 * seed 0x5eed, k_tile 0, epoch_num 0, switch_edges -1, max_sweeps 0. */
void ppr_default_opts(ppr_query_opts* opts);

/*
 * Copy a CSR graph (host arrays; the caller keeps ownership) to the device.
 * The library stores out- and in-adjacency (the in-CSR is the transpose used
 * by pull sweeps, Algorithm 3's scans), relabelled by in-degree so that rows
 * of similar length are contiguous.  Work is enqueued on `cuda_stream`
 * (cudaStream_t or NULL) and completed before return.
 * Errors: PPR_ERR_ARG (null pointers, n < 1), PPR_ERR_GRAPH (contract above),
 * PPR_ERR_OOM, PPR_ERR_CUDA.
 */
ppr_status ppr_graph_load(const int64_t* row_ptr, const int32_t* col_idx, int64_t n, int64_t m,
                          void* cuda_stream, ppr_graph** out);

/*
 * Answer k single-source queries.  src: host int32[k], each in [0, n);
 * duplicates allowed; src order is the output row order.
 *   out_pi  : k x n row-major float64, device or host memory (caller-owned).
 *   out_r   : optional (NULL) k x n float64, device or host: HP = the push
 *             residual r = (alpha e_s + (1-alpha) pi_hat P - pi_hat)/alpha of the
 *             returned pi_hat; APPROX = the FP32 residue the walks started from.
 *   out_walk_counts: optional k x n uint32 (APPROX only) walk endpoint counts.
 *   stats   : optional host array of k entries.
 * HP mode follows Algorithm 3: a frontier push (the queue phase) until a
 * level's out-edges exceed the switch threshold, then dense pull passes.  By
 * default the dense phase is an iterative refinement: the remaining error
 * e = pi - X of the Q1.63 estimate X (the push reserve) solves
 * e = r + (1-alpha) e P (Eq. 7 with r in place of alpha e_s), which BF16 and
 * FP32 passes solve (in place, over-relaxed), then e is folded into X and one
 * exact synchronous Q1.63 pass measures ||X' - X||_1; the returned X' has
 * ||pi_hat - pi||_1 <= (1-alpha) ||X' - X||_1 / alpha + rounding <= lambda
 * (stats[i].final_l1_residual).  Flags select the other dense phases (all
 * passes Q1.63, synchronous PowItr passes, Algorithm 3's epochs).  APPROX
 * follows Algorithm 4.  Work runs on `cuda_stream`; the call returns after
 * the stream has finished the query.  HP correction passes keep the most
 * gathered rows of their tile persisting in L2 (a per-launch access-policy
 * window): for each batch of these passes the call raises the CUDA
 * context's persisting-L2 limit to 48 MB if it is lower, and after the batch
 * turns every persisting line of the context back to normal
 * (cudaCtxResetPersistingL2Cache) and restores the limit, which also affects
 * windows that other work of the same process set.  Errors: PPR_ERR_ARG,
 * PPR_ERR_ADMIT (state does not
 * fit in free device memory), PPR_ERR_NOT_CONVERGED, PPR_ERR_OOM, PPR_ERR_CUDA.
 */
ppr_status ppr_sssp_query(ppr_graph* g, const int32_t* src, int32_t k, ppr_mode mode,
                          const ppr_query_opts* opts, double* out_pi, double* out_r,
                          uint32_t* out_walk_counts, ppr_stats* stats, void* cuda_stream);

/*
 * High-precision queries without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that may not allocate
 * device memory themselves or through this library -- for example a plug-in
 * inside a server or database that gets a fixed memory budget from its host's
 * own allocator, or a process that has already reserved all free memory in a
 * caching pool.  ppr_sssp_query grows a per-graph workspace with cudaMalloc;
 * this call instead runs a simpler variant of the pull sweep (zero start,
 * every node pushed each pass) whose scratch is one 16 MiB array compiled into
 * the library, and it calls no allocation routine.
 *   src: host int32[k]; out_pi: DEVICE k x n float64 (caller-owned);
 *   out_sweeps: optional host int32[k] (passes run for each source).
 *   Result: ||pi_hat - pi||_1 <= lambda for every source, as ppr_sssp_query.
 * Limit: sources are solved k_tile at a time, k_tile = min(k, 8) rounded down
 * to 1, 2, 4 or 8.  n * k_tile * 24 bytes plus the residual sums,
 * (max_sweeps + 1) * k_tile * 8 bytes with max_sweeps =
 * 4 ceil(ln lambda / ln(1 - alpha)) + 64, must fit in the 16 MiB (about
 * 87,000 nodes at k_tile = 8, 690,000 at k_tile = 1 for alpha = 0.2); larger
 * graphs return PPR_ERR_ARG with a message, and so does an alpha so small that
 * max_sweeps would exceed 131072.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before capturing any stream on the device.  All calls share the one array
 * (it keeps the last call's contents; the call clears what must start at
 * zero), so calls that overlap on the GPU -- other threads, other streams --
 * race and must be serialised by the caller.  The graph's per-node scale
 * factors depend on alpha and are rewritten (on the call's stream) when a
 * call brings an alpha other than the last one used on that graph: calls with
 * different alphas on one graph must therefore be serialised against every
 * query entry point (ppr_sssp_query included), not only against each other.
 * The graph itself is allocated by ppr_graph_load as usual.  Errors:
 * PPR_ERR_ARG, PPR_ERR_NOT_CONVERGED, PPR_ERR_CUDA.
 */
ppr_status ppr_sssp_query_noalloc(ppr_graph* g, const int32_t* src, int32_t k, double alpha, double lambda,
                                  double* out_pi, int32_t* out_sweeps, void* cuda_stream);

/* Device bytes the workspace of a high-precision query of k sources needs
 * (k_tile as in ppr_query_opts, 0 = the width the query would pick: the
 * autotuned one of k's bucket, else the smallest power of two >= k up to 64),
 * for alpha = 0.2 and lambda = 1e-8 (other values change only the per-pass
 * residual sums, 512 bytes per pass), outputs in device or page-locked host
 * memory (pageable host outputs add k x n x 8 bytes of staging each).  The
 * library reuses the workspace across calls, so a server can admit a batch
 * when this fits in free memory plus what the graph already holds
 * (ppr_workspace_bytes); ppr_sssp_query applies the same test and refuses
 * with PPR_ERR_ADMIT before any launch.  -1 on bad arguments. */
int64_t ppr_query_state_bytes(const ppr_graph* g, int32_t k, int32_t k_tile);

/* Device bytes the graph's query workspace holds now (it grows to the largest
 * batch seen and is reused; ppr_free releases it).  -1 for a NULL graph. */
int64_t ppr_workspace_bytes(const ppr_graph* g);

/* Test hooks for the error paths, process-wide, off by default; no GPU fault
 * is involved.  PPR_INJECT_FREE_BYTES: admission tests see at most `value`
 * free device bytes (value < 0: off).  PPR_INJECT_ALLOC_FAIL: the value-th
 * workspace allocation from now on fails as out of memory, and the call that
 * made it returns PPR_ERR_OOM (value <= 0: off).  PPR_ERR_ARG for an unknown
 * hook. */
#define PPR_INJECT_FREE_BYTES 1
#define PPR_INJECT_ALLOC_FAIL 2
ppr_status ppr_inject(int32_t hook, int64_t value);

/* Self-test of the device conversions between the library's Q1.63 fixed-point
 * values (the exact reserve and residue of Sec. 4, Eq. 7) and FP32/FP64, which
 * the kernels do with integer instructions: `count` counter-generated inputs
 * (seed), each checked bit for bit against CUDA's conversion intrinsics.
 * out_mismatches (host, 7 entries) receives the mismatch counts of: Q1.63 ->
 * FP32, 64-bit integer -> FP32, Q1.63 -> FP64, signed Q1.63 -> FP32, FP32 ->
 * signed Q1.63 (these round to nearest even; |value| < 1), FP32 -> Q1.63 by
 * truncation (0 <= value < 2), and floor(integer x FP32 value) (value in
 * [0, 1]).  Synchronises the stream.
 * Errors: PPR_ERR_ARG (count < 0, NULL out_mismatches), PPR_ERR_CUDA. */
ppr_status ppr_selftest_fixconv(int64_t count, uint64_t seed, int64_t* out_mismatches, void* cuda_stream);

/*
 * Measure, on a calibration batch src[k], every tile width up to the smallest
 * power of two >= k (at most 64) combined with queue->sweep switch thresholds
 * of {0, 0.002, 0.02, 0.1} x m x k_tile frontier edges (Algorithm 3 fixes
 * scanThreshold = n/4 for a CPU), each timed with CUDA events on the stream,
 * and the three fastest again over three calls (best mean); then, for the
 * chosen one, the over-relaxation factor w of the
 * in-place correction passes over {1.05, 1.1, 1.15}, each judged by its mean
 * time over three calls (their pass counts vary from call to call; a factor
 * under which a call does not certify is skipped).
 * The fastest setting is written to *best (from *base, NULL = defaults),
 * its time to *best_ms (optional), and remembered in the graph for later HP
 * calls of a k of the same power-of-two bucket: the tile width and switch
 * for calls with k_tile = 0 / switch_edges = -1, w for every HP call (the
 * stats report it).  out_pi: device k x n float64 scratch for the calibration answers.
 * Widths whose workspace does not fit are skipped.  Errors as ppr_sssp_query,
 * and PPR_ERR_NOT_CONVERGED when no candidate certifies the calibration batch
 * within max_sweeps (nothing is remembered then).
 */
ppr_status ppr_autotune(ppr_graph* g, const int32_t* src, int32_t k, const ppr_query_opts* base, double* out_pi,
                        ppr_query_opts* best, double* best_ms, void* cuda_stream);

/*
 * SpeedPPR-Index (Sec. 6.2): SpeedPPR needs at most d_v walks from a node v,
 * so the endpoints of d_v alpha-walks per node (m int32 in all, independent
 * of eps) answer every approximate query.  The walk stored for the caller's
 * out-edge slot e (row_ptr[v] + k) uses Philox-4x32-10 with key (seed_lo,
 * seed_hi) and counter (e_lo, e_hi, t/2, 0x1D3A), words as in the walk phase.
 * ppr_sssp_query(..., PPR_APPROX) with flags PPR_FLAG_INDEX then reads, for
 * each v with r(v) > 0, the first W_v = min(ceil(r(v) W), d_v) stored
 * endpoints of v instead of walking.  Builds on the device (4 m bytes, kept
 * with the graph; a rebuild replaces it).  ppr_index_get copies the endpoints
 * to a host int32[m] in the caller's slot order and node ids; it blocks.
 * Errors: PPR_ERR_ARG (NULL graph or output, alpha outside (0, 1), or
 * ppr_index_get before any build), PPR_ERR_OOM (no room for the 4 m bytes),
 * PPR_ERR_NOT_CONVERGED (a stored walk longer than 2^16 steps), PPR_ERR_CUDA.
 * An indexed query on a graph without an index, or with one built for another
 * alpha, fails with PPR_ERR_ARG.
 */
ppr_status ppr_index_build(ppr_graph* g, uint64_t seed, double alpha, void* cuda_stream);
ppr_status ppr_index_get(const ppr_graph* g, int32_t* endpoints);

/* Release the graph and every device buffer it owns; NULL is allowed. */
void ppr_free(ppr_graph* g);

/* Message of the last error on the calling thread ("" if none). */
const char* ppr_last_error(void);

/* Graph sizes: n, m as loaded (0 for a NULL graph). */
int64_t ppr_graph_n(const ppr_graph* g);
int64_t ppr_graph_m(const ppr_graph* g);

/* ------------------------------------------------------------------------
 * Learned warm start.  The paper always starts from r = e_s; here a model
 * maps a two-step sketch of the source (reserve after two Power Iterations,
 * Eq. 5, plus the alive mass of Eq. 3 at step 2) projected by a fixed Gaussian
 * n x 128 matrix through an MLP 128 -> hidden -> hidden -> 64 (GELU) to
 * coefficients h, and returns x = max(0, S + U h) / sum (U: n x 64 basis).
 * ppr_sssp_query with opts->warm_start = model pushes the residual of x,
 * r = (alpha e_s + (1-alpha) x P - x) / alpha, to lambda exactly as it pushes
 * e_s from the zero start, so the l1 guarantee does not depend on the model.
 * Weights and U are FP32 masters with BF16 copies used by tensor-core GEMMs
 * (FP32 accumulation); training minimises the mean l1 error ||x - pi||_1
 * against exact vectors computed by the plain method, with Adam.
 * ------------------------------------------------------------------------ */
typedef struct ppr_model ppr_model;

typedef struct {
  int32_t feat_dim;  /* 128 */
  int32_t hidden;    /* hidden width, multiple of 16 (512) */
  int32_t rank;      /* basis rank, 64 */
  int32_t correction_passes; /* 0: x0 = max(0, S + U h)/sum replaces the zero start.
                                L > 0: the zero-start solve runs L passes, then the
                                model adds mu * max(0, U h)/sum, mu = 1 - sum(x) the
                                mass still missing (the residual's sum becomes 0) */
  uint64_t seed;     /* weight init and Gaussian feature matrix */
  float lr;          /* Adam step size (1e-3) */
  int32_t epochs;    /* epochs for ppr_model_train (20) */
  double alpha;      /* 0.2 */
  double lambda;     /* labels' l1 accuracy (1e-8) */
} ppr_model_opts;

void ppr_model_default_opts(ppr_model_opts* opts);

/* New model for graph g (init: W ~ N(0, 1/fan_in), b = 0, U = 0, so the
 * untrained model returns the sketch).  Errors: PPR_ERR_ARG, PPR_ERR_OOM. */
ppr_status ppr_model_create(ppr_graph* g, const ppr_model_opts* opts, ppr_model** out);

/* Train on n_src sources (host ids): exact labels from the plain HP method
 * (kept on the device, n x n_src FP32), then `epochs` passes of Adam over
 * batches of 64 sources in a shuffled order.  loss_per_epoch: optional host
 * array of `epochs` mean l1 losses.  Errors: PPR_ERR_ARG, PPR_ERR_ADMIT. */
ppr_status ppr_model_train(ppr_model* model, const int32_t* train_src, int32_t n_src, int32_t epochs, float lr,
                           uint64_t shuffle_seed, float* loss_per_epoch, void* cuda_stream);

/* One forward/backward over k <= 64 sources with labels (k x n float64, host
 * or device, caller's node order); lr > 0 also applies one Adam step.  loss
 * receives the mean l1 error of the batch.  Errors: PPR_ERR_ARG (NULL model
 * or labels, k outside 1..64, lr < 0, a source out of range), PPR_ERR_OOM,
 * PPR_ERR_CUDA. */
ppr_status ppr_model_train_step(ppr_model* model, const int32_t* src, int32_t k, const double* labels, float lr,
                                double* loss, void* cuda_stream);

/* The model's estimate x for k sources (k x n float64, host or device).
 * Errors: PPR_ERR_ARG (NULL model or output, k < 1, a source out of range),
 * PPR_ERR_OOM, PPR_ERR_CUDA. */
ppr_status ppr_model_estimate(ppr_model* model, const int32_t* src, int32_t k, double* out_x, void* cuda_stream);

/* Parameters and last gradients, flat float32 host arrays of
 * ppr_model_param_count entries (0 for a NULL model) in the order W1
 * (feat x hidden), b1, W2 (hidden x hidden), b2, W3 (hidden x rank), b3,
 * U (n x rank, caller's node order); either pointer of get_params may be
 * NULL.  set_params also refreshes the BF16 copies.  Errors: PPR_ERR_ARG
 * (NULL model, or NULL params for set_params), PPR_ERR_CUDA. */
int64_t ppr_model_param_count(const ppr_model* model);
ppr_status ppr_model_get_params(const ppr_model* model, float* params, float* grads);
ppr_status ppr_model_set_params(ppr_model* model, const float* params);

/* Checkpoint (parameters and Adam moments) to a binary file, and back; a
 * checkpoint loads only into a graph of the same n.  Errors: PPR_ERR_ARG
 * (NULL arguments, a file that cannot be opened, written, read or
 * recognised as a checkpoint for this graph), PPR_ERR_CUDA (save: a copy
 * from the device failed), PPR_ERR_OOM (load).  ppr_model_free accepts
 * NULL. */
ppr_status ppr_model_save(const ppr_model* model, const char* path);
ppr_status ppr_model_load(ppr_graph* g, const char* path, ppr_model** out);
void ppr_model_free(ppr_model* model);

#ifdef __cplusplus
}
#endif
#endif /* PPR_GB300_H */
