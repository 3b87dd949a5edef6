/*
 * Seeded synthetic graph and source generators.
 *
 * This module only builds INPUTS: it draws edges, removes self-loops and
 * duplicates, gives every sink one random out-edge, and lays the result out
 * as a CSR (row_ptr int64 [n+1], col_idx int32 [m], rows sorted by id,
 * neighbours ascending).  It holds none of the Personalized PageRank
 * arithmetic; both the FP64 oracle and the CUDA library consume its output.
 *
 * Stand-ins for the paper's SNAP datasets (Sec. 8, Table 2): the paper's
 * graphs are directed power-law graphs with isolated nodes removed; here the
 * shapes come from a directed Chung-Lu model and from R-MAT.
 *
 * Randomness is counter-based (SplitMix64 finaliser, Steele/Lea/Flood 2014)
 * so the output does not depend on the number of threads.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>
#include <unistd.h>

#define TAG_EDGE 1u
#define TAG_PERM_OUT 2u
#define TAG_PERM_IN 3u
#define TAG_SINK 4u
#define TAG_SRC 5u
#define TAG_RELABEL 6u

static inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
/* word #i of the stream named (seed, tag) */
static inline uint64_t rng_at(uint64_t seed, uint64_t tag, uint64_t i) {
  return mix64(mix64(mix64(seed) ^ (tag * 0xD1B54A32D192ED03ULL)) + i);
}
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, n) by multiply-shift */
static inline uint64_t below(uint64_t x, uint64_t n) {
  return (uint64_t)(((unsigned __int128)x * (unsigned __int128)n) >> 64);
}

static int pick_threads(int t) {
  if (t > 0) return t;
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  if (c < 1) c = 1;
  if (c > 64) c = 64;
  return (int)c;
}

/* ---------------------------------------------------------------- threads */
typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi, int tid);
typedef struct { range_fn fn; void* ctx; int64_t lo, hi; int tid; } range_job;
static void* range_tramp(void* p) {
  range_job* j = (range_job*)p;
  j->fn(j->ctx, j->lo, j->hi, j->tid);
  return NULL;
}
static void parallel_for(int threads, int64_t total, range_fn fn, void* ctx) {
  if (threads <= 1 || total < 4096) { fn(ctx, 0, total, 0); return; }
  pthread_t th[64];
  range_job jobs[64];
  for (int t = 0; t < threads; ++t) {
    jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].tid = t;
    jobs[t].lo = total * t / threads; jobs[t].hi = total * (t + 1) / threads;
    pthread_create(&th[t], NULL, range_tramp, &jobs[t]);
  }
  for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------- parallel LSD radix sort */
#define RBITS 11
#define RBUCKETS (1 << RBITS)
typedef struct {
  uint64_t *src, *dst; int64_t cnt; int shift; int threads;
  int64_t* hist; /* [threads][RBUCKETS] */
} radix_ctx;
static void radix_hist(void* p, int64_t lo, int64_t hi, int tid) {
  radix_ctx* c = (radix_ctx*)p;
  int64_t* h = c->hist + (int64_t)tid * RBUCKETS;
  memset(h, 0, sizeof(int64_t) * RBUCKETS);
  for (int64_t i = lo; i < hi; ++i) h[(c->src[i] >> c->shift) & (RBUCKETS - 1)]++;
}
static void radix_scatter(void* p, int64_t lo, int64_t hi, int tid) {
  radix_ctx* c = (radix_ctx*)p;
  int64_t* h = c->hist + (int64_t)tid * RBUCKETS;
  for (int64_t i = lo; i < hi; ++i) {
    uint64_t k = c->src[i];
    c->dst[h[(k >> c->shift) & (RBUCKETS - 1)]++] = k;
  }
}
/* sorts keys[0..cnt) ascending on the low `bits` bits; returns 0 or -1 (OOM) */
static int radix_sort(uint64_t* keys, int64_t cnt, int bits, int threads) {
  uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(cnt > 0 ? cnt : 1));
  int64_t* hist = (int64_t*)malloc(sizeof(int64_t) * RBUCKETS * (size_t)threads);
  if (!tmp || !hist) { free(tmp); free(hist); return -1; }
  radix_ctx c;
  c.cnt = cnt; c.threads = threads; c.hist = hist;
  uint64_t *a = keys, *b = tmp;
  int eff_threads = (threads <= 1 || cnt < 4096) ? 1 : threads;
  for (int shift = 0; shift < bits; shift += RBITS) {
    c.src = a; c.dst = b; c.shift = shift;
    parallel_for(eff_threads, cnt, radix_hist, &c);
    int64_t run = 0;
    for (int d = 0; d < RBUCKETS; ++d)
      for (int t = 0; t < eff_threads; ++t) {
        int64_t v = hist[(int64_t)t * RBUCKETS + d];
        hist[(int64_t)t * RBUCKETS + d] = run;
        run += v;
      }
    parallel_for(eff_threads, cnt, radix_scatter, &c);
    uint64_t* s = a; a = b; b = s;
  }
  if (a != keys) memcpy(keys, a, sizeof(uint64_t) * (size_t)cnt);
  free(tmp); free(hist);
  return 0;
}

static int bits_for(int64_t n) {
  int b = 1;
  while (((int64_t)1 << b) < n) ++b;
  return b;
}

/*
 * keys: (src << 32 | dst) pairs, self-loops already dropped.  Sorts, removes
 * duplicates, gives each sink one out-edge to a uniform node != itself
 * (stream TAG_SINK of `seed`, word v) and builds the CSR.  Frees keys.
 */
static int finish_csr(uint64_t* keys, int64_t cnt, int64_t n, uint64_t seed, int threads,
                      int64_t* m_out, int64_t** rp_out, int32_t** ci_out) {
  int bits = bits_for(n);
  if (radix_sort(keys, cnt, 32 + bits, threads)) { free(keys); return -1; }
  int64_t u = 0;
  for (int64_t i = 0; i < cnt; ++i)
    if (u == 0 || keys[i] != keys[u - 1]) keys[u++] = keys[i];
  int64_t* rp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!rp) { free(keys); return -1; }
  for (int64_t i = 0; i < u; ++i) rp[(keys[i] >> 32) + 1]++;
  int64_t sinks = 0;
  for (int64_t v = 0; v < n; ++v)
    if (rp[v + 1] == 0) { rp[v + 1] = 1; ++sinks; }
  for (int64_t v = 0; v < n; ++v) rp[v + 1] += rp[v];
  int64_t m = u + sinks;
  int32_t* ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  if (!ci) { free(keys); free(rp); return -1; }
  int64_t e = 0;
  for (int64_t v = 0; v < n; ++v) {
    int64_t w = rp[v];
    if (e < u && (int64_t)(keys[e] >> 32) == v) {
      while (e < u && (int64_t)(keys[e] >> 32) == v) ci[w++] = (int32_t)(keys[e++] & 0xffffffffu);
    } else {
      uint64_t t = below(rng_at(seed, TAG_SINK, (uint64_t)v), (uint64_t)(n - 1));
      if ((int64_t)t >= v) ++t;
      ci[w++] = (int32_t)t;
    }
  }
  free(keys);
  *m_out = m; *rp_out = rp; *ci_out = ci;
  return 0;
}

/* seeded Fisher-Yates permutation of [0, n) */
static int32_t* permutation(int64_t n, uint64_t seed, uint64_t tag) {
  int32_t* p = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!p) return NULL;
  for (int64_t i = 0; i < n; ++i) p[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    int64_t j = (int64_t)below(rng_at(seed, tag, (uint64_t)i), (uint64_t)(i + 1));
    int32_t t = p[i]; p[i] = p[j]; p[j] = t;
  }
  return p;
}

/* ---------------------------------------------------------------- Chung-Lu */
/*
 * Directed Chung-Lu: node weights w_i = (i+1)^(-1/(gamma-1)), assigned to
 * nodes through two independent seeded permutations (one for the out side,
 * one for the in side).  m_draws (source, target) pairs are drawn by
 * inverse-CDF sampling; self-loops and duplicates are dropped.
 */
typedef struct {
  int64_t n, draws; uint64_t seed; const double* cdf; const int32_t *pout, *pin;
  uint64_t* keys;
} cl_ctx;
static int64_t cdf_pick(const double* cdf, int64_t n, double x) {
  int64_t lo = 0, hi = n - 1; /* first i with cdf[i] > x */
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (cdf[mid] > x) hi = mid; else lo = mid + 1;
  }
  return lo;
}
static void cl_work(void* p, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  cl_ctx* c = (cl_ctx*)p;
  double total = c->cdf[c->n - 1];
  for (int64_t i = lo; i < hi; ++i) {
    double x = u01(rng_at(c->seed, TAG_EDGE, 2 * (uint64_t)i)) * total;
    double y = u01(rng_at(c->seed, TAG_EDGE, 2 * (uint64_t)i + 1)) * total;
    int64_t a = c->pout[cdf_pick(c->cdf, c->n, x)];
    int64_t b = c->pin[cdf_pick(c->cdf, c->n, y)];
    c->keys[i] = (a == b) ? UINT64_MAX : (((uint64_t)a << 32) | (uint64_t)b);
  }
}
static int64_t drop_marked(uint64_t* keys, int64_t cnt) {
  int64_t u = 0;
  for (int64_t i = 0; i < cnt; ++i)
    if (keys[i] != UINT64_MAX) keys[u++] = keys[i];
  return u;
}

int pg_chung_lu(int64_t n, int64_t m_draws, double gamma, uint64_t seed, int threads,
                int64_t* m_out, int64_t** rp_out, int32_t** ci_out) {
  if (n < 2 || n > 0x7fffffffLL || m_draws < 0 || !(gamma > 1.0)) return -2;
  threads = pick_threads(threads);
  double* cdf = (double*)malloc(sizeof(double) * (size_t)n);
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m_draws > 0 ? m_draws : 1));
  int32_t* pout = permutation(n, seed, TAG_PERM_OUT);
  int32_t* pin = permutation(n, seed, TAG_PERM_IN);
  if (!cdf || !keys || !pout || !pin) { free(cdf); free(keys); free(pout); free(pin); return -1; }
  double run = 0.0, ex = -1.0 / (gamma - 1.0);
  for (int64_t i = 0; i < n; ++i) { run += pow((double)(i + 1), ex); cdf[i] = run; }
  cl_ctx c = {n, m_draws, seed, cdf, pout, pin, keys};
  parallel_for(threads, m_draws, cl_work, &c);
  free(cdf); free(pout); free(pin);
  int64_t cnt = drop_marked(keys, m_draws);
  return finish_csr(keys, cnt, n, seed, threads, m_out, rp_out, ci_out);
}

/* ------------------------------------------------------------------- R-MAT */
/*
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004): each of ef * 2^scale edges picks
 * one quadrant per bit level with probabilities (a, b, c, 1-a-b-c), where
 * quadrant b sets the destination bit and c the source bit.  Level l uses a
 * 21-bit slice of word l/3 of the edge's stream, compared against thresholds
 * rounded to 21 bits.  Ids are then relabelled by a seeded permutation so id
 * order carries no locality, self-loops and duplicates are dropped and sinks
 * are patched.
 */
typedef struct {
  int scale; uint64_t seed; uint32_t ta, tab, tabc; const int32_t* perm; uint64_t* keys;
} rm_ctx;
static void rm_work(void* p, int64_t lo, int64_t hi, int tid) {
  (void)tid;
  rm_ctx* c = (rm_ctx*)p;
  uint64_t words = (uint64_t)(c->scale + 2) / 3;
  for (int64_t i = lo; i < hi; ++i) {
    uint64_t a = 0, b = 0, w = 0;
    for (int l = 0; l < c->scale; ++l) {
      if (l % 3 == 0) w = rng_at(c->seed, TAG_EDGE, (uint64_t)i * words + (uint64_t)(l / 3));
      uint32_t x = (uint32_t)((w >> (21 * (l % 3))) & 0x1fffffu);
      uint64_t sb = 0, db = 0;
      if (x < c->ta) { sb = 0; db = 0; }
      else if (x < c->tab) { sb = 0; db = 1; }
      else if (x < c->tabc) { sb = 1; db = 0; }
      else { sb = 1; db = 1; }
      a = (a << 1) | sb;
      b = (b << 1) | db;
    }
    int64_t s = c->perm[a], d = c->perm[b];
    c->keys[i] = (s == d) ? UINT64_MAX : (((uint64_t)s << 32) | (uint64_t)d);
  }
}

int pg_rmat(int scale, double edge_factor, double a, double b, double c, uint64_t seed,
            int threads, int64_t* m_out, int64_t** rp_out, int32_t** ci_out) {
  if (scale < 1 || scale > 30 || !(edge_factor > 0) || a < 0 || b < 0 || c < 0 || a + b + c > 1.0)
    return -2;
  threads = pick_threads(threads);
  int64_t n = (int64_t)1 << scale;
  int64_t draws = (int64_t)llround(edge_factor * (double)n);
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(draws > 0 ? draws : 1));
  int32_t* perm = permutation(n, seed, TAG_RELABEL);
  if (!keys || !perm) { free(keys); free(perm); return -1; }
  const double one = (double)(1u << 21);
  rm_ctx ctx;
  ctx.scale = scale; ctx.seed = seed; ctx.perm = perm; ctx.keys = keys;
  ctx.ta = (uint32_t)llround(a * one);
  ctx.tab = (uint32_t)llround((a + b) * one);
  ctx.tabc = (uint32_t)llround((a + b + c) * one);
  parallel_for(threads, draws, rm_work, &ctx);
  free(perm);
  int64_t cnt = drop_marked(keys, draws);
  return finish_csr(keys, cnt, n, seed, threads, m_out, rp_out, ci_out);
}

/* ----------------------------------------------------------------- sources */
/* k uniform random node ids in [0, n) (with replacement), stream TAG_SRC */
int pg_sources(int64_t n, int64_t k, uint64_t seed, int32_t* out) {
  if (n < 1 || k < 0 || !out) return -2;
  for (int64_t i = 0; i < k; ++i) out[i] = (int32_t)below(rng_at(seed, TAG_SRC, (uint64_t)i), (uint64_t)n);
  return 0;
}

/* ------------------------------------------------------- BFS subgraph */
/*
 * The first `count` nodes reached by a breadth-first search from `root`
 * (out-edges, neighbours in ascending id order), relabelled 0..count-1 in
 * visiting order, with the induced edges; sinks of the subgraph are patched
 * with the same rule as the generators.
 */
int pg_bfs_subgraph(int64_t n, const int64_t* rp, const int32_t* ci, int32_t root, int64_t count,
                    uint64_t seed, int64_t* n_out, int64_t* m_out, int64_t** rp_out,
                    int32_t** ci_out) {
  if (n < 1 || root < 0 || root >= n || count < 2) return -2;
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* label = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!order || !label) { free(order); free(label); return -1; }
  for (int64_t i = 0; i < n; ++i) label[i] = -1;
  int64_t head = 0, tail = 0;
  order[tail] = root; label[root] = (int32_t)tail; ++tail;
  while (head < tail && tail < count) {
    int32_t v = order[head++];
    for (int64_t e = rp[v]; e < rp[v + 1] && tail < count; ++e) {
      int32_t u = ci[e];
      if (label[u] < 0) { label[u] = (int32_t)tail; order[tail++] = u; }
    }
  }
  int64_t nn = tail;
  int64_t cap = 0;
  for (int64_t i = 0; i < nn; ++i) cap += rp[order[i] + 1] - rp[order[i]];
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(cap > 0 ? cap : 1));
  if (!keys) { free(order); free(label); return -1; }
  int64_t cnt = 0;
  for (int64_t i = 0; i < nn; ++i) {
    int32_t v = order[i];
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
      int32_t lu = label[ci[e]];
      if (lu >= 0 && lu != i) keys[cnt++] = ((uint64_t)i << 32) | (uint64_t)lu;
    }
  }
  free(order); free(label);
  *n_out = nn;
  return finish_csr(keys, cnt, nn, seed, 1, m_out, rp_out, ci_out);
}

void pg_free(void* p) { free(p); }
