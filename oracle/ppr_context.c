/*
 * Context timing only -- not an oracle, and test/benchmark infrastructure.
 *
 * A multi-core FP64 power iteration (Sec. 3.1, Eqs. 3-5: pi += alpha r,
 * r <- (1-alpha) r P until sum r <= lambda), the residue propagated as a pull
 * over the transposed graph with the destination rows split across OpenMP
 * threads.  The benchmark times it beside the single-threaded oracle to state
 * what all of the host's cores do with the plain method; a CPU test checks it
 * against the oracle's PowItr.  It shares no code with the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int64_t n, m;
  int64_t* in_rp;  /* in-CSR row pointers (n + 1) */
  int32_t* in_ci;  /* in-neighbours */
  double* inv_d;   /* 1 / out-degree */
} ctx_graph;

int ctx_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void ctx_graph_free(ctx_graph* g) {
  if (!g) return;
  free(g->in_rp);
  free(g->in_ci);
  free(g->inv_d);
  free(g);
}

/* transpose of the out-CSR (row_ptr int64, col_idx int32); NULL on failure */
ctx_graph* ctx_graph_new(int64_t n, const int64_t* rp, const int32_t* ci) {
  if (n < 1 || !rp || !ci) return NULL;
  ctx_graph* g = (ctx_graph*)calloc(1, sizeof(ctx_graph));
  if (!g) return NULL;
  g->n = n;
  g->m = rp[n];
  g->in_rp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  g->in_ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->m > 0 ? g->m : 1));
  g->inv_d = (double*)malloc(sizeof(double) * (size_t)n);
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!g->in_rp || !g->in_ci || !g->inv_d || !fill) {
    free(fill);
    ctx_graph_free(g);
    return NULL;
  }
  for (int64_t e = 0; e < g->m; ++e) g->in_rp[ci[e] + 1]++;
  for (int64_t u = 0; u < n; ++u) g->in_rp[u + 1] += g->in_rp[u];
  memcpy(fill, g->in_rp, sizeof(int64_t) * (size_t)n);
  for (int64_t v = 0; v < n; ++v) {
    const int64_t d = rp[v + 1] - rp[v];
    g->inv_d[v] = d > 0 ? 1.0 / (double)d : 0.0;
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) g->in_ci[fill[ci[e]]++] = (int32_t)v;
  }
  free(fill);
  return g;
}

/* pi (n doubles) for source s; returns 0, or -1 on bad arguments / memory,
 * -4 when max_iter iterations did not reach sum r <= lambda */
int ctx_powitr(const ctx_graph* g, double alpha, int32_t s, double lambda, int64_t max_iter, double* pi,
               int64_t* iterations) {
  if (!g || !pi || s < 0 || s >= g->n || !(alpha > 0.0 && alpha < 1.0) || !(lambda > 0.0)) return -1;
  const int64_t n = g->n;
  double* r = (double*)calloc((size_t)n, sizeof(double));
  double* rn = (double*)malloc(sizeof(double) * (size_t)n);
  if (!r || !rn) {
    free(r);
    free(rn);
    return -1;
  }
  memset(pi, 0, sizeof(double) * (size_t)n);
  r[s] = 1.0;
  double rsum = 1.0;
  int64_t it = 0;
  while (rsum > lambda && it < max_iter) {
    double next = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : next)
    for (int64_t u = 0; u < n; ++u) {
      pi[u] += alpha * r[u];
      double acc = 0.0;
      for (int64_t e = g->in_rp[u]; e < g->in_rp[u + 1]; ++e) acc += r[g->in_ci[e]] * g->inv_d[g->in_ci[e]];
      rn[u] = (1.0 - alpha) * acc;
      next += rn[u];
    }
    double* t = r;
    r = rn;
    rn = t;
    rsum = next;
    ++it;
  }
  free(r);
  free(rn);
  if (iterations) *iterations = it;
  return rsum <= lambda ? 0 : -4;
}
