/*
 * FP64 CPU oracle for single-source Personalized PageRank (arXiv 2101.03652).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * statement of what the CUDA library computes.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header or constant table with the CUDA path.
 *
 * Graph: CSR with row_ptr int64[n+1], col_idx int32[m], out-degree
 * d_v = row_ptr[v+1]-row_ptr[v] >= 1 (no dead ends, Sec. 2).  The transition
 * matrix is P_v = A_v / d_v (Sec. 2).  Vectors are row vectors indexed by node.
 *
 * Functions and the passages they follow:
 *   orc_push_sequence   Algorithm 1 with a given push order (running example)
 *   orc_powitr          Power Iteration, Sec. 3.1 Eqs. 3-5, run as
 *                       Simultaneous Forward Push (Sec. 4.1, Eq. 7, r_max = 0)
 *   orc_fifo_fwdpush    First-In-First-Out Forward Push, Algorithm 2
 *   orc_fifo_refine     Algorithm 2's loop started from a given (pi, r): used for
 *                       SpeedPPR's refinement step (Algorithm 4, third step)
 *   orc_powerpush       Power Iteration with Forward Push, Algorithm 3
 *   orc_dense_solve     the linear system of Eq. 1 by Gaussian elimination
 *   orc_residual        r = (alpha e_s + (1-alpha) x P - x) / alpha, the push
 *                       residual of an arbitrary estimate x (invariant of Sec. 3.2)
 *   orc_speedppr_W      W of Eq. 8
 *   orc_walks           SpeedPPR's walk phase, Algorithm 4 (loop over v with r>0)
 *   orc_speedppr        Algorithm 4 end to end
 *   orc_philox4x32_10   Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
 *   orc_gaussian_rows   rows of the fixed random feature matrix of the learned
 *                       warm start (Box-Muller on Philox words)
 *   orc_build_walk_index, orc_index_walks
 *                       SpeedPPR-Index: d_v stored walks per node (Sec. 6.2)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_GRAPH -2
#define ORC_ERR_OOM -3
#define ORC_ERR_NOT_CONVERGED -4

typedef struct {
  int64_t iterations;      /* PowItr iterations / FIFO levels / dense scans */
  int64_t pushes;          /* push operations performed */
  int64_t edge_pushes;     /* sum of d_v over all push operations */
  int64_t edge_pushes_at_lambda; /* edge pushes when r_sum first <= lambda at a level end */
  int64_t fifo_pushes;     /* pushes done in the queue phase (Algorithm 3) */
  int64_t scans;           /* full sequential scans (Algorithm 3) */
  int64_t walks;           /* random walks performed (Algorithm 4) */
  int64_t walk_steps;      /* total moves over all walks */
  double r_sum;            /* final sum of residues (recomputed) */
  double W;                /* Eq. 8 */
} orc_stats;

/* Neumaier-compensated sum of r[0..n) */
static double sum_comp(const double* r, int64_t n) {
  double s = 0.0, c = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double t = s + r[i];
    if (fabs(s) >= fabs(r[i])) c += (s - t) + r[i];
    else c += (r[i] - t) + s;
    s = t;
  }
  return s + c;
}
static double abs_sum_comp(const double* r, int64_t n) {
  double s = 0.0, c = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double a = fabs(r[i]);
    double t = s + a;
    if (s >= a) c += (s - t) + a;
    else c += (a - t) + s;
    s = t;
  }
  return s + c;
}

/* The graph must satisfy Sec. 2's assumptions: every d_v >= 1; ids in range.
 * Rows sorted ascending without duplicates or self-loops (the generators'
 * cleaning) are also required so that the CSR is canonical. */
int orc_validate(int64_t n, const int64_t* rp, const int32_t* ci) {
  if (n < 1 || !rp || !ci || rp[0] != 0) return ORC_ERR_ARG;
  for (int64_t v = 0; v < n; ++v) {
    if (rp[v + 1] - rp[v] < 1) return ORC_ERR_GRAPH;
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
      if (ci[e] < 0 || ci[e] >= n || ci[e] == v) return ORC_ERR_GRAPH;
      if (e > rp[v] && ci[e] <= ci[e - 1]) return ORC_ERR_GRAPH;
    }
  }
  return ORC_OK;
}

/* One push operation on v (Sec. 3.2): pi(v) += alpha r(v); each out-neighbour
 * u gets (1-alpha) r(v) / d_v; then r(v) = 0.  Returns the residue pushed. */
static double push_one(int64_t v, const int64_t* rp, const int32_t* ci, double alpha, double* pi,
                       double* r) {
  double rv = r[v];
  int64_t d = rp[v + 1] - rp[v];
  pi[v] += alpha * rv;
  double share = (1.0 - alpha) * rv / (double)d;
  for (int64_t e = rp[v]; e < rp[v + 1]; ++e) r[ci[e]] += share;
  r[v] = 0.0;
  return rv;
}

/*
 * Algorithm 1 (FwdPush) with the "arbitrary" choice made explicit: starting
 * from pi = 0, r = e_s, push the nodes of order[0..count) in turn (Sec. 3.2).
 */
int orc_push_sequence(int64_t n, const int64_t* rp, const int32_t* ci, double alpha, int32_t s,
                      const int32_t* order, int64_t count, double* pi, double* r) {
  if (n < 1 || s < 0 || s >= n || !pi || !r || (count > 0 && !order)) return ORC_ERR_ARG;
  memset(pi, 0, sizeof(double) * (size_t)n);
  memset(r, 0, sizeof(double) * (size_t)n);
  r[s] = 1.0;
  for (int64_t i = 0; i < count; ++i) {
    if (order[i] < 0 || order[i] >= n) return ORC_ERR_ARG;
    push_one(order[i], rp, ci, alpha, pi, r);
  }
  return ORC_OK;
}

/*
 * Power Iteration (Sec. 3.1): gamma^(0) = e_s; each iteration sets
 * pi^(j+1) = pi^(j) + alpha gamma^(j) and gamma^(j+1) = (1-alpha) gamma^(j) P
 * (Eq. 3, Eq. 5), i.e. SimFwdPush with r_max = 0 (Sec. 4.1, Eq. 7).  Stops when
 * ||gamma||_1 <= lambda (the l1 error of Eq. 6).  Returns pi and r = gamma.
 */
int orc_powitr(int64_t n, const int64_t* rp, const int32_t* ci, double alpha, int32_t s, double lambda,
               int64_t max_iter, double* pi, double* r, orc_stats* st) {
  if (n < 1 || s < 0 || s >= n || !(alpha > 0 && alpha < 1) || !(lambda > 0) || !pi || !r)
    return ORC_ERR_ARG;
  double* nxt = (double*)calloc((size_t)n, sizeof(double));
  if (!nxt) return ORC_ERR_OOM;
  memset(pi, 0, sizeof(double) * (size_t)n);
  memset(r, 0, sizeof(double) * (size_t)n);
  r[s] = 1.0;
  int64_t j = 0, edges = 0;
  double rsum = 1.0;
  while (rsum > lambda) {
    if (j >= max_iter) { free(nxt); return ORC_ERR_NOT_CONVERGED; }
    memset(nxt, 0, sizeof(double) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) {
      if (r[v] == 0.0) continue;
      int64_t d = rp[v + 1] - rp[v];
      pi[v] += alpha * r[v];
      double share = (1.0 - alpha) * r[v] / (double)d;
      for (int64_t e = rp[v]; e < rp[v + 1]; ++e) nxt[ci[e]] += share;
      edges += d;
    }
    memcpy(r, nxt, sizeof(double) * (size_t)n);
    ++j;
    rsum = abs_sum_comp(r, n);
  }
  free(nxt);
  if (st) {
    memset(st, 0, sizeof(*st));
    st->iterations = j;
    st->edge_pushes = edges;
    st->r_sum = rsum;
  }
  return ORC_OK;
}

/*
 * Algorithm 2 (FIFO-FwdPush) with a first-in-first-out queue and a membership
 * flag for the test "u not in Q".  The queue holds at most n nodes because of
 * that test, so a ring of n slots suffices.  Level bookkeeping follows the
 * iterations S^(j) defined after Theorem 1: S^(0) = {s}, S^(j+1) = the nodes
 * appended while S^(j) is processed.
 */
typedef struct { int32_t* q; uint8_t* in; int64_t head, tail, cap; } ring;
static int ring_init(ring* R, int64_t n) {
  R->q = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  R->in = (uint8_t*)calloc((size_t)n, 1);
  R->head = R->tail = 0; R->cap = n;
  return (R->q && R->in) ? 0 : -1;
}
static void ring_free(ring* R) { free(R->q); free(R->in); }
static int64_t ring_size(const ring* R) { return R->tail - R->head; }
static void ring_push(ring* R, int32_t v) { R->q[R->tail % R->cap] = v; R->tail++; R->in[v] = 1; }
static int32_t ring_pop(ring* R) { int32_t v = R->q[R->head % R->cap]; R->head++; R->in[v] = 0; return v; }

/* The queue loop of Algorithm 2 from the current (pi, r) and queue.  The
 * incremental r_sum tracks the decrease alpha * r(v) of each push. */
static void fifo_loop(ring* Q, const int64_t* rp, const int32_t* ci, double alpha, double rmax,
                      double lambda, double* pi, double* r, double* rsum, orc_stats* st) {
  int64_t level_end = Q->tail;
  int reached = (*rsum <= lambda);
  while (ring_size(Q) > 0) {
    int32_t v = ring_pop(Q);
    double rv = r[v];
    int64_t d = rp[v + 1] - rp[v];
    pi[v] += alpha * rv;
    double share = (1.0 - alpha) * rv / (double)d;
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
      int32_t u = ci[e];
      r[u] += share;
      int64_t du = rp[u + 1] - rp[u];
      if (r[u] > (double)du * rmax && !Q->in[u]) ring_push(Q, u);
    }
    r[v] = 0.0;
    *rsum -= alpha * rv;
    st->pushes++;
    st->edge_pushes += d;
    if (Q->head == level_end) { /* end of iteration S^(j) */
      st->iterations++;
      level_end = Q->tail;
      if (!reached && *rsum <= lambda) { reached = 1; st->edge_pushes_at_lambda = st->edge_pushes; }
    }
  }
  if (!reached) st->edge_pushes_at_lambda = -1;
}

int orc_fifo_fwdpush(int64_t n, const int64_t* rp, const int32_t* ci, double alpha, int32_t s,
                     double rmax, double lambda, double* pi, double* r, orc_stats* st) {
  if (n < 1 || s < 0 || s >= n || !(alpha > 0 && alpha < 1) || !(rmax >= 0) || !pi || !r)
    return ORC_ERR_ARG;
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  ring Q;
  if (ring_init(&Q, n)) { ring_free(&Q); return ORC_ERR_OOM; }
  memset(pi, 0, sizeof(double) * (size_t)n);
  memset(r, 0, sizeof(double) * (size_t)n);
  r[s] = 1.0;
  ring_push(&Q, s);
  double rsum = 1.0;
  fifo_loop(&Q, rp, ci, alpha, rmax, lambda, pi, r, &rsum, st);
  ring_free(&Q);
  st->r_sum = sum_comp(r, n);
  return ORC_OK;
}

/* Algorithm 2's loop from a given state: the queue starts with every node that
 * is active w.r.t. rmax, in ascending id order (refinement of Algorithm 4). */
int orc_fifo_refine(int64_t n, const int64_t* rp, const int32_t* ci, double alpha, double rmax,
                    double* pi, double* r, orc_stats* st) {
  if (n < 1 || !(alpha > 0 && alpha < 1) || !(rmax >= 0) || !pi || !r) return ORC_ERR_ARG;
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  ring Q;
  if (ring_init(&Q, n)) { ring_free(&Q); return ORC_ERR_OOM; }
  for (int64_t v = 0; v < n; ++v)
    if (r[v] > (double)(rp[v + 1] - rp[v]) * rmax) ring_push(&Q, (int32_t)v);
  double rsum = sum_comp(r, n);
  fifo_loop(&Q, rp, ci, alpha, rmax, 0.0, pi, r, &rsum, st);
  ring_free(&Q);
  st->r_sum = sum_comp(r, n);
  return ORC_OK;
}

/*
 * Algorithm 3 (PowerPush).  epoch_num = 8 and scan_threshold = n/4 in the
 * paper; both are parameters here.  r_max = lambda/m for the queue phase.
 * The queue phase runs while Q is non-empty, |Q| <= scan_threshold and
 * r_sum > lambda.  Then, if r_sum > lambda, epochs i = 1..epoch_num use
 * r'_max = lambda^(i/epoch_num)/m and repeat full sequential scans in id order
 * (asynchronous pushes on the current residues) while r_sum > m r'_max.
 * r_sum is tracked incrementally in the queue phase and recomputed exactly
 * after each scan; a scan that pushes nothing ends its epoch (rounding only).
 */
int orc_powerpush(int64_t n, const int64_t* rp, const int32_t* ci, double alpha, int32_t s,
                  double lambda, int epoch_num, double scan_threshold, double* pi, double* r,
                  orc_stats* st) {
  if (n < 1 || s < 0 || s >= n || !(alpha > 0 && alpha < 1) || !(lambda > 0) || epoch_num < 1 || !pi ||
      !r)
    return ORC_ERR_ARG;
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  int64_t m = rp[n];
  double rmax = lambda / (double)m;
  ring Q;
  if (ring_init(&Q, n)) { ring_free(&Q); return ORC_ERR_OOM; }
  memset(pi, 0, sizeof(double) * (size_t)n);
  memset(r, 0, sizeof(double) * (size_t)n);
  r[s] = 1.0;
  ring_push(&Q, s);
  double rsum = 1.0;
  while (ring_size(&Q) > 0 && (double)ring_size(&Q) <= scan_threshold && rsum > lambda) {
    int32_t v = ring_pop(&Q);
    double rv = r[v];
    int64_t d = rp[v + 1] - rp[v];
    pi[v] += alpha * rv;
    double share = (1.0 - alpha) * rv / (double)d;
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
      int32_t u = ci[e];
      r[u] += share;
      if (!Q.in[u] && r[u] > (double)(rp[u + 1] - rp[u]) * rmax) ring_push(&Q, u);
    }
    r[v] = 0.0;
    rsum -= alpha * rv;
    st->pushes++;
    st->fifo_pushes++;
    st->edge_pushes += d;
  }
  ring_free(&Q);
  rsum = sum_comp(r, n);
  if (rsum > lambda) {
    for (int i = 1; i <= epoch_num; ++i) {
      double thr = pow(lambda, (double)i / (double)epoch_num); /* m * r'_max */
      double rmax_i = thr / (double)m;
      while (rsum > thr) {
        int64_t pushed = 0;
        for (int64_t v = 0; v < n; ++v) {
          int64_t d = rp[v + 1] - rp[v];
          if (r[v] > (double)d * rmax_i) {
            push_one(v, rp, ci, alpha, pi, r);
            ++pushed;
            st->edge_pushes += d;
          }
        }
        st->pushes += pushed;
        st->scans++;
        rsum = sum_comp(r, n);
        if (pushed == 0) break;
      }
    }
  }
  st->r_sum = rsum;
  return ORC_OK;
}

/*
 * Eq. 1: pi_s = alpha e_s + (1-alpha) pi_s P, i.e. (I - (1-alpha) P^T) pi^T =
 * alpha e_s^T.  Dense Gaussian elimination with partial pivoting; n small.
 */
int orc_dense_solve(int64_t n, const int64_t* rp, const int32_t* ci, double alpha, int32_t s,
                    double* pi) {
  if (n < 1 || n > 4096 || s < 0 || s >= n || !pi) return ORC_ERR_ARG;
  double* M = (double*)calloc((size_t)(n * n), sizeof(double));
  double* b = (double*)calloc((size_t)n, sizeof(double));
  if (!M || !b) { free(M); free(b); return ORC_ERR_OOM; }
  for (int64_t i = 0; i < n; ++i) M[i * n + i] = 1.0;
  for (int64_t v = 0; v < n; ++v) {
    double p = 1.0 / (double)(rp[v + 1] - rp[v]);
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) M[(int64_t)ci[e] * n + v] -= (1.0 - alpha) * p; /* (P^T)[u][v] */
  }
  b[s] = alpha;
  for (int64_t k = 0; k < n; ++k) {
    int64_t piv = k;
    for (int64_t i = k + 1; i < n; ++i)
      if (fabs(M[i * n + k]) > fabs(M[piv * n + k])) piv = i;
    if (piv != k) {
      for (int64_t j = 0; j < n; ++j) { double t = M[k * n + j]; M[k * n + j] = M[piv * n + j]; M[piv * n + j] = t; }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    double dkk = M[k * n + k];
    for (int64_t i = k + 1; i < n; ++i) {
      double f = M[i * n + k] / dkk;
      if (f == 0.0) continue;
      for (int64_t j = k; j < n; ++j) M[i * n + j] -= f * M[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double acc = b[i];
    for (int64_t j = i + 1; j < n; ++j) acc -= M[i * n + j] * pi[j];
    pi[i] = acc / M[i * n + i];
  }
  free(M); free(b);
  return ORC_OK;
}

/*
 * Push residual of an arbitrary estimate x: the r that keeps the invariant
 * pi_s = x + sum_v r(v) pi_v of Sec. 3.2, namely
 * r = (alpha e_s + (1-alpha) x P - x) / alpha.
 */
int orc_residual(int64_t n, const int64_t* rp, const int32_t* ci, double alpha, int32_t s,
                 const double* x, double* r) {
  if (n < 1 || s < 0 || s >= n || !x || !r) return ORC_ERR_ARG;
  double* xp = (double*)calloc((size_t)n, sizeof(double));
  if (!xp) return ORC_ERR_OOM;
  for (int64_t v = 0; v < n; ++v) {
    double share = x[v] / (double)(rp[v + 1] - rp[v]);
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) xp[ci[e]] += share;
  }
  for (int64_t u = 0; u < n; ++u) {
    double b = (u == s) ? alpha : 0.0;
    r[u] = (b + (1.0 - alpha) * xp[u] - x[u]) / alpha;
  }
  free(xp);
  return ORC_OK;
}

/* ------------------------------------------------------------- Philox-4x32-10 */
/* Salmon et al., SC'11: 10 rounds; round multipliers 0xD2511F53, 0xCD9E8D57;
 * key schedule adds the Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* --------------------------------------------------------------- SpeedPPR */
/* Eq. 8 with the natural logarithm: W = 2 (2 eps/3 + 2) ln n / (eps^2 mu). */
double orc_speedppr_W(int64_t n, double eps, double mu) {
  return 2.0 * (2.0 * eps / 3.0 + 2.0) * log((double)n) / (eps * eps * mu);
}

/*
 * The walk phase of Algorithm 4 for residue vector r: for each v with
 * r(v) > 0 (ascending v), W_v = ceil(r(v) * W) alpha-random walks start at v
 * (Sec. 2: at the current node the walk stops with probability alpha, else it
 * moves to a uniform out-neighbour); each walk that stops at u adds
 * r(v) / W_v to est(u) and 1 to counts(u).
 *
 * Random numbers (one fixed definition shared with the CUDA library by
 * specification, not by code): walk ids are the exclusive prefix sum of W_v
 * over ascending v.  Walk w at step t uses Philox-4x32-10 with
 * key = (seed_lo, seed_hi), counter = (w_lo, w_hi, t/2, source_index); words
 * 2(t%2) and 2(t%2)+1 are the stop word and the move word.  The walk stops at
 * the current node iff stop word < floor(alpha 2^32); otherwise it moves to
 * col_idx[row_ptr[v] + ((move word * d_v) >> 32)].  A walk longer than
 * max_steps moves is an error.
 */
int orc_walks(int64_t n, const int64_t* rp, const int32_t* ci, double alpha, const double* r, double W,
              uint64_t seed, uint32_t source_index, int64_t max_steps, uint32_t* counts, double* est,
              orc_stats* st) {
  if (n < 1 || !r || !counts || !est || !(W > 0) || !(alpha > 0 && alpha < 1)) return ORC_ERR_ARG;
  const uint32_t stop_below = (uint32_t)floor(alpha * 4294967296.0);
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  memset(counts, 0, sizeof(uint32_t) * (size_t)n);
  memset(est, 0, sizeof(double) * (size_t)n);
  uint64_t wid = 0;
  int64_t steps_total = 0;
  for (int64_t v = 0; v < n; ++v) {
    if (!(r[v] > 0.0)) continue;
    double prod = r[v] * W;
    uint64_t Wv = (uint64_t)ceil(prod);
    double inc = r[v] / (double)Wv;
    for (uint64_t k = 0; k < Wv; ++k, ++wid) {
      int64_t cur = v;
      uint32_t words[4];
      int64_t t = 0;
      for (;;) {
        if ((t & 1) == 0) {
          uint32_t ctr[4] = {(uint32_t)wid, (uint32_t)(wid >> 32), (uint32_t)(t >> 1), source_index};
          orc_philox4x32_10(ctr, key, words);
        }
        uint32_t stopw = words[2 * (t & 1)], movew = words[2 * (t & 1) + 1];
        if (stopw < stop_below) break;
        if (t >= max_steps) return ORC_ERR_NOT_CONVERGED;
        int64_t d = rp[cur + 1] - rp[cur];
        cur = ci[rp[cur] + (int64_t)(((uint64_t)movew * (uint64_t)d) >> 32)];
        ++t;
      }
      counts[cur] += 1;
      est[cur] += inc;
      steps_total += t;
    }
  }
  if (st) { st->walks = (int64_t)wid; st->walk_steps = steps_total; st->W = W; }
  return ORC_OK;
}

/*
 * Algorithm 4: W from Eq. 8; PowerPush with lambda = m / W; refinement with
 * r_max = 1/W until no node is active; walks from the remaining residue;
 * pi_out = reserve + walk estimates.  r_out (optional) receives the residue
 * the walks were launched from, counts (optional) the walk endpoints.
 */
int orc_speedppr(int64_t n, const int64_t* rp, const int32_t* ci, double alpha, int32_t s, double eps,
                 double mu, uint64_t seed, uint32_t source_index, double* pi_out, double* r_out,
                 uint32_t* counts, orc_stats* st) {
  if (n < 2 || s < 0 || s >= n || !(eps > 0) || !(mu > 0) || !pi_out) return ORC_ERR_ARG;
  orc_stats local;
  if (!st) st = &local;
  memset(st, 0, sizeof(*st));
  int64_t m = rp[n];
  double W = orc_speedppr_W(n, eps, mu);
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* est = (double*)malloc(sizeof(double) * (size_t)n);
  uint32_t* cnt = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  if (!r || !est || !cnt) { free(r); free(est); free(cnt); return ORC_ERR_OOM; }
  orc_stats a, b, c;
  int rc = orc_powerpush(n, rp, ci, alpha, s, (double)m / W, 8, (double)n / 4.0, pi_out, r, &a);
  if (rc == ORC_OK) rc = orc_fifo_refine(n, rp, ci, alpha, 1.0 / W, pi_out, r, &b);
  memset(&c, 0, sizeof(c));
  if (rc == ORC_OK) rc = orc_walks(n, rp, ci, alpha, r, W, seed, source_index, 1 << 16, cnt, est, &c);
  if (rc == ORC_OK) {
    if (r_out) memcpy(r_out, r, sizeof(double) * (size_t)n);
    if (counts) memcpy(counts, cnt, sizeof(uint32_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) pi_out[v] += est[v];
    st->pushes = a.pushes + b.pushes;
    st->edge_pushes = a.edge_pushes + b.edge_pushes;
    st->walks = c.walks;
    st->walk_steps = c.walk_steps;
    st->W = W;
    st->r_sum = sum_comp(r, n);
  }
  free(r); free(est); free(cnt);
  return rc;
}

/* ------------------------------------------------ warm-start feature matrix */
/*
 * Row u of the n x F feature matrix G used to project the two-step sketch:
 * entry (u, j) is a standard normal.  Philox-4x32-10 with key (seed_lo,
 * seed_hi) and counter (u, j/4, 0x47, 0) gives words w0..w3; (w0, w1) make
 * entries 4q, 4q+1 and (w2, w3) make 4q+2, 4q+3 by Box-Muller (Box & Muller,
 * 1958): u1 = (wa + 1) 2^-32 in (0, 1], u2 = wb 2^-32, radius
 * sqrt(-2 ln u1), angles 2 pi u2 (cosine first, then sine).  F % 4 == 0.
 * Writes rows u0 .. u0+count-1 into out (count x F, row-major).
 */
void orc_gaussian_rows(int64_t u0, int64_t count, int F, uint64_t seed, double* out) {
  const double two_pi = 6.283185307179586476925286766559;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t i = 0; i < count; ++i) {
    uint64_t u = (uint64_t)(u0 + i);
    for (int q = 0; q < F / 4; ++q) {
      uint32_t ctr[4] = {(uint32_t)u, (uint32_t)q, 0x47u, 0u};
      uint32_t w[4];
      orc_philox4x32_10(ctr, key, w);
      for (int p = 0; p < 2; ++p) {
        double u1 = ((double)w[2 * p] + 1.0) * (1.0 / 4294967296.0);
        double u2 = (double)w[2 * p + 1] * (1.0 / 4294967296.0);
        double rad = sqrt(-2.0 * log(u1));
        out[i * F + 4 * q + 2 * p] = rad * cos(two_pi * u2);
        out[i * F + 4 * q + 2 * p + 1] = rad * sin(two_pi * u2);
      }
    }
  }
}

/* ------------------------------------------------------------ SpeedPPR-Index */
/*
 * The index of Sec. 6.2 ("Improvements over FORA"): SpeedPPR needs at most
 * d_v walks from each node v, so d_v walks per node, m in total, answer every
 * eps.  Walk k of node v belongs to edge slot e = row_ptr[v] + k: it is the
 * alpha-walk of orc_walks with Philox counter (e_lo, e_hi, t/2, 0x1D3A) under
 * key (seed_lo, seed_hi).  index[e] receives its endpoint.
 */
int orc_build_walk_index(int64_t n, const int64_t* rp, const int32_t* ci, double alpha, uint64_t seed,
                         int64_t max_steps, int32_t* index) {
  if (n < 1 || !rp || !ci || !index || !(alpha > 0 && alpha < 1)) return ORC_ERR_ARG;
  const uint32_t stop_below = (uint32_t)floor(alpha * 4294967296.0);
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t v = 0; v < n; ++v) {
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
      int64_t cur = v;
      uint32_t words[4];
      for (int64_t t = 0;; ++t) {
        if ((t & 1) == 0) {
          uint32_t ctr[4] = {(uint32_t)e, (uint32_t)((uint64_t)e >> 32), (uint32_t)(t >> 1), 0x1D3Au};
          orc_philox4x32_10(ctr, key, words);
        }
        if (words[2 * (t & 1)] < stop_below) break;
        if (t >= max_steps) return ORC_ERR_NOT_CONVERGED;
        int64_t d = rp[cur + 1] - rp[cur];
        cur = ci[rp[cur] + (int64_t)(((uint64_t)words[2 * (t & 1) + 1] * (uint64_t)d) >> 32)];
      }
      index[e] = (int32_t)cur;
    }
  }
  return ORC_OK;
}

/*
 * Algorithm 4's walk phase read from the index: for each v with r(v) > 0,
 * W_v = ceil(r(v) W) (at most d_v after the refinement; capped at d_v so that
 * float rounding of the residue cannot ask for more walks than stored), and
 * the endpoints of v's first W_v index walks each add r(v)/W_v to est and 1
 * to counts.
 */
int orc_index_walks(int64_t n, const int64_t* rp, const int32_t* index, const double* r, double W,
                    uint32_t* counts, double* est, orc_stats* st) {
  if (n < 1 || !rp || !index || !r || !counts || !est || !(W > 0)) return ORC_ERR_ARG;
  memset(counts, 0, sizeof(uint32_t) * (size_t)n);
  memset(est, 0, sizeof(double) * (size_t)n);
  int64_t walks = 0;
  for (int64_t v = 0; v < n; ++v) {
    if (!(r[v] > 0.0)) continue;
    int64_t d = rp[v + 1] - rp[v];
    int64_t Wv = (int64_t)ceil(r[v] * W);
    if (Wv > d) Wv = d;
    double inc = r[v] / (double)Wv;
    for (int64_t k = 0; k < Wv; ++k) {
      int32_t u = index[rp[v] + k];
      counts[u] += 1;
      est[u] += inc;
    }
    walks += Wv;
  }
  if (st) { memset(st, 0, sizeof(*st)); st->walks = walks; st->W = W; }
  return ORC_OK;
}
