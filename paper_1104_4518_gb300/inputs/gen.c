/*
 * Seeded synthetic graph inputs for the BFS library, its tests and its benchmark.
 *
 * This module only produces edge lists and root choices.  It holds none of the
 * traversal's arithmetic (no CSR construction, no levels, no parents), so that
 * the CPU oracle and the CUDA path can both consume the same inputs while
 * sharing no code of the method itself.
 *
 * Random numbers: every draw is the i-th output of the SplitMix64 generator
 * (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014) seeded with `seed`, i.e. mix64(seed + (i + 1) * GAMMA) with the
 * published constants, so draws are counter-based and can be computed in any
 * order by any number of threads.
 *
 * Graph families (Sec. 6 of the paper: R-MAT with skewed degrees, edgefactor 16,
 * random vertex relabelling as in Graph 500, Sec. 4.4):
 *   - R-MAT: for edge e and bit level l (most significant first) one uniform
 *     U = draw(e * scale + l) picks a quadrant: U < A -> (0,0), U < A+B -> (0,1),
 *     U < A+B+C -> (1,0), else (1,1).  No noise is added.
 *   - relabel: Fisher-Yates shuffle of 0..n-1 driven by a second seed, applied
 *     to both endpoints of every edge.
 *   - 3D 7-point grid N^3 (id = x + N*y + N*N*z), each undirected edge once.
 *   - Erdos-Renyi G(n, m): m uniform pairs (self-loops and repeats allowed; the
 *     CSR builders drop them).
 *   - roots: draws modulo n, rejected until the vertex has a non-loop edge and
 *     has not been chosen before.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define GEN_GAMMA 0x9e3779b97f4a7c15ULL

static inline uint64_t gen_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* i-th output (i >= 0) of SplitMix64 seeded with `seed`. */
uint64_t gen_splitmix64_at(uint64_t seed, uint64_t i) {
  return gen_mix64(seed + (i + 1) * GEN_GAMMA);
}

/* Uniform double in [0, 1) from the top 53 bits of a draw. */
static inline double gen_unit(uint64_t seed, uint64_t i) {
  return (double)(gen_splitmix64_at(seed, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* Uniform integer in [0, bound) by the multiply-high method (Lemire 2019). */
static inline uint64_t gen_below(uint64_t seed, uint64_t i, uint64_t bound) {
  unsigned __int128 p = (unsigned __int128)gen_splitmix64_at(seed, i) * bound;
  return (uint64_t)(p >> 64);
}

static int gen_threads(void) {
  long t = sysconf(_SC_NPROCESSORS_ONLN);
  return t < 1 ? 1 : (int)t;
}

/* ---------------- thread pool helper ---------------- */

typedef struct {
  void (*fn)(void* ctx, int64_t lo, int64_t hi);
  void* ctx;
  int64_t lo, hi;
} gen_job;

static void* gen_job_run(void* p) {
  gen_job* j = (gen_job*)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

static int gen_nthreads = 0;

void gen_set_threads(int t) { gen_nthreads = t; }

static void gen_parallel_for(int64_t count, void (*fn)(void*, int64_t, int64_t), void* ctx) {
  int t = gen_nthreads > 0 ? gen_nthreads : gen_threads();
  if (t > 256) t = 256;
  if (count < 65536 || t <= 1) {
    fn(ctx, 0, count);
    return;
  }
  pthread_t th[256];
  gen_job jobs[256];
  int started[256];
  for (int i = 0; i < t; ++i) {
    jobs[i].fn = fn;
    jobs[i].ctx = ctx;
    jobs[i].lo = count * i / t;
    jobs[i].hi = count * (i + 1) / t;
    started[i] = pthread_create(&th[i], NULL, gen_job_run, &jobs[i]) == 0;
    if (!started[i]) gen_job_run(&jobs[i]);
  }
  for (int i = 0; i < t; ++i)
    if (started[i]) pthread_join(th[i], NULL);
}

/* ---------------- R-MAT ---------------- */

typedef struct {
  int scale;
  uint64_t seed;
  double a, ab, abc;
  int32_t* src;
  int32_t* dst;
} rmat_ctx;

static void rmat_body(void* p, int64_t lo, int64_t hi) {
  rmat_ctx* c = (rmat_ctx*)p;
  for (int64_t e = lo; e < hi; ++e) {
    uint32_t u = 0, v = 0;
    for (int l = 0; l < c->scale; ++l) {
      double r = gen_unit(c->seed, (uint64_t)e * (uint64_t)c->scale + (uint64_t)l);
      uint32_t bit = 1u << (c->scale - 1 - l);
      if (r < c->a) {
      } else if (r < c->ab) {
        v |= bit;
      } else if (r < c->abc) {
        u |= bit;
      } else {
        u |= bit;
        v |= bit;
      }
    }
    c->src[e] = (int32_t)u;
    c->dst[e] = (int32_t)v;
  }
}

/* Fills src/dst[0..m) with R-MAT endpoints on 2^scale vertices (before relabel). */
int gen_rmat(int scale, int64_t m, double a, double b, double c, uint64_t seed,
             int32_t* src, int32_t* dst) {
  if (scale < 1 || scale > 30 || m < 0 || !src || !dst) return -1;
  rmat_ctx ctx = {scale, seed, a, a + b, a + b + c, src, dst};
  gen_parallel_for(m, rmat_body, &ctx);
  return 0;
}

/* Fisher-Yates permutation of 0..n-1: for i = n-1 .. 1 swap perm[i] with
 * perm[j], j = draw(n-1-i) mod (i+1). */
int gen_permutation(int32_t n, uint64_t seed, int32_t* perm) {
  if (n < 0 || !perm) return -1;
  for (int32_t i = 0; i < n; ++i) perm[i] = i;
  for (int32_t i = n - 1; i > 0; --i) {
    int32_t j = (int32_t)gen_below(seed, (uint64_t)(n - 1 - i), (uint64_t)i + 1);
    int32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
  return 0;
}

typedef struct {
  const int32_t* perm;
  int32_t* src;
  int32_t* dst;
} relabel_ctx;

static void relabel_body(void* p, int64_t lo, int64_t hi) {
  relabel_ctx* c = (relabel_ctx*)p;
  for (int64_t e = lo; e < hi; ++e) {
    c->src[e] = c->perm[c->src[e]];
    c->dst[e] = c->perm[c->dst[e]];
  }
}

/* Applies vertex relabelling perm to both endpoint arrays in place. */
int gen_apply_permutation(const int32_t* perm, int64_t m, int32_t* src, int32_t* dst) {
  if (m < 0 || !perm || !src || !dst) return -1;
  relabel_ctx ctx = {perm, src, dst};
  gen_parallel_for(m, relabel_body, &ctx);
  return 0;
}

/* ---------------- 3D grid ---------------- */

typedef struct {
  int32_t N;
  int32_t* src;
  int32_t* dst;
} grid_ctx;

static void grid_body(void* p, int64_t lo, int64_t hi) {
  grid_ctx* c = (grid_ctx*)p;
  int64_t N = c->N;
  int64_t per_dir = N * N * (N - 1);
  for (int64_t e = lo; e < hi; ++e) {
    int64_t dir = e / per_dir, r = e % per_dir;
    int64_t a = r % (N - 1), rest = r / (N - 1);  /* a: coordinate along dir, < N-1 */
    int64_t p1 = rest % N, p2 = rest / N;
    int64_t x, y, z;
    if (dir == 0) { x = a; y = p1; z = p2; }
    else if (dir == 1) { x = p1; y = a; z = p2; }
    else { x = p1; y = p2; z = a; }
    int64_t id = x + N * y + N * N * z;
    int64_t step = dir == 0 ? 1 : (dir == 1 ? N : N * N);
    c->src[e] = (int32_t)id;
    c->dst[e] = (int32_t)(id + step);
  }
}

/* Number of undirected edges of the N^3 7-point grid. */
int64_t gen_grid3d_edges(int32_t N) {
  if (N < 1) return 0;
  return 3LL * N * N * (N - 1);
}

int gen_grid3d(int32_t N, int32_t* src, int32_t* dst) {
  if (N < 1 || (int64_t)N * N * N > 2147483647LL || !src || !dst) return -1;
  grid_ctx ctx = {N, src, dst};
  gen_parallel_for(gen_grid3d_edges(N), grid_body, &ctx);
  return 0;
}

/* ---------------- Erdos-Renyi G(n, m) ---------------- */

typedef struct {
  int32_t n;
  uint64_t seed;
  int32_t* src;
  int32_t* dst;
} er_ctx;

static void er_body(void* p, int64_t lo, int64_t hi) {
  er_ctx* c = (er_ctx*)p;
  for (int64_t e = lo; e < hi; ++e) {
    c->src[e] = (int32_t)gen_below(c->seed, 2 * (uint64_t)e, (uint64_t)c->n);
    c->dst[e] = (int32_t)gen_below(c->seed, 2 * (uint64_t)e + 1, (uint64_t)c->n);
  }
}

int gen_er(int32_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst) {
  if (n < 1 || m < 0 || !src || !dst) return -1;
  er_ctx ctx = {n, seed, src, dst};
  gen_parallel_for(m, er_body, &ctx);
  return 0;
}

/* ---------------- roots ---------------- */

typedef struct {
  const int32_t* src;
  const int32_t* dst;
  uint8_t* has_edge;
} touch_ctx;

static void touch_body(void* p, int64_t lo, int64_t hi) {
  touch_ctx* c = (touch_ctx*)p;
  for (int64_t e = lo; e < hi; ++e) {
    int32_t u = c->src[e], v = c->dst[e];
    if (u != v) {
      __atomic_store_n(&c->has_edge[u], (uint8_t)1, __ATOMIC_RELAXED);
      __atomic_store_n(&c->has_edge[v], (uint8_t)1, __ATOMIC_RELAXED);
    }
  }
}

/* Marks has_edge[v] = 1 for every vertex with at least one non-loop edge. */
int gen_touched(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, uint8_t* has_edge) {
  if (n < 0 || m < 0 || !has_edge) return -1;
  memset(has_edge, 0, (size_t)n);
  touch_ctx ctx = {src, dst, has_edge};
  gen_parallel_for(m, touch_body, &ctx);
  return 0;
}

/* Picks k distinct roots with a non-loop edge.  Returns the number picked
 * (less than k only if fewer such vertices exist). */
int32_t gen_roots(const uint8_t* has_edge, int32_t n, int32_t k, uint64_t seed, int32_t* roots) {
  if (n < 1 || k < 0 || !has_edge || !roots) return -1;
  int64_t avail = 0;
  for (int32_t v = 0; v < n; ++v) avail += has_edge[v] != 0;
  if (avail < k) k = (int32_t)avail;
  int32_t got = 0;
  for (uint64_t i = 0; got < k; ++i) {
    int32_t c = (int32_t)gen_below(seed, i, (uint64_t)n);
    if (!has_edge[c]) continue;
    int dup = 0;
    for (int32_t j = 0; j < got; ++j) dup |= roots[j] == c;
    if (!dup) roots[got++] = c;
  }
  return got;
}
