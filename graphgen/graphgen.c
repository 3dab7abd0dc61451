/*
 * graphgen.c - seeded synthetic graph generators (host, C11 + pthreads).
 *
 * These generators produce the undirected int32 edge lists that BOTH the
 * CPU oracle and the CUDA path consume.  They hold none of the triangle
 * method's arithmetic: no orientation, no degree order, no intersection.
 * An edge list may contain self-loops and duplicate / reversed pairs; the
 * cleanup step of the method (and of the oracle) removes them.
 *
 * Random numbers: every draw is the splitmix64 output function (Steele, Lea
 * and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
 * applied to a counter, so draw k of stream s under seed is a pure function
 * of (seed, s, k) and the result does not depend on the thread count.
 *
 *   mix(z)     = splitmix64 finaliser
 *   key(seed,s)= mix(seed*G + C0) ^ mix(s + G)            (G = golden gamma)
 *   draw(key,k)= mix(key + (k+1)*G)
 *
 * Generators
 *   gg_er       uniform endpoint pairs in [0,n)          (Erdos-Renyi G(n,E))
 *   gg_rmat     recursive-matrix (R-MAT / Kronecker) edges with quadrant
 *               probabilities (a,b,c,d), no per-level noise, then a seeded
 *               Fisher-Yates relabelling of the 2^scale ids
 *   gg_chunglu  Chung-Lu: weight w_i ~ (i+1)^(-1/(gamma-1)) scaled so that the
 *               weights sum to n*d, capped at sqrt(n*d), n*d/2 endpoint pairs
 *               drawn with probability proportional to w (Vose alias table),
 *               then an optional seeded Fisher-Yates relabelling.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define GG_GOLDEN 0x9E3779B97F4A7C15ULL
#define GG_C0 0x632BE59BD9B4E019ULL

static inline uint64_t gg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static inline uint64_t gg_key(uint64_t seed, uint64_t stream) {
  return gg_mix(seed * GG_GOLDEN + GG_C0) ^ gg_mix(stream + GG_GOLDEN);
}
static inline uint64_t gg_draw(uint64_t key, uint64_t k) {
  return gg_mix(key + (k + 1) * GG_GOLDEN);
}
/* integer in [0, bound) from the high 32 bits of r (multiply-shift). */
static inline uint32_t gg_below(uint64_t r, uint32_t bound) {
  return (uint32_t)(((r >> 32) * (uint64_t)bound) >> 32);
}

uint64_t gg_splitmix64(uint64_t x) { return gg_mix(x + GG_GOLDEN); }
uint64_t gg_draw_pub(uint64_t seed, uint64_t stream, uint64_t k) {
  return gg_draw(gg_key(seed, stream), k);
}

static int gg_threads(int want) {
  if (want > 0) return want;
  long p = sysconf(_SC_NPROCESSORS_ONLN);
  if (p < 1) p = 1;
  if (p > 64) p = 64;
  return (int)p;
}

/* ---------------------------------------------------------------- parallel */
typedef struct gg_job gg_job;
typedef void (*gg_body)(const gg_job*, int64_t lo, int64_t hi);
struct gg_job {
  gg_body body;
  int64_t lo, hi;
  /* generator parameters */
  uint64_t seed;
  uint32_t n;
  int scale;
  uint64_t thr_a, thr_ab, thr_abc; /* R-MAT thresholds, scaled by 2^32 */
  const uint32_t* alias_thr;
  const uint32_t* alias_idx;
  const int32_t* perm; /* optional relabelling */
  int32_t* src;
  int32_t* dst;
};

static void* gg_thread_main(void* arg) {
  gg_job* j = (gg_job*)arg;
  j->body(j, j->lo, j->hi);
  return NULL;
}

static void gg_run(gg_job proto, int64_t count, int nthreads) {
  nthreads = gg_threads(nthreads);
  if (count < (int64_t)nthreads * 4096) nthreads = 1;
  if (nthreads == 1) {
    proto.body(&proto, 0, count);
    return;
  }
  pthread_t tid[64];
  gg_job jobs[64];
  int64_t chunk = (count + nthreads - 1) / nthreads;
  int started = 0;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = proto;
    jobs[t].lo = (int64_t)t * chunk;
    jobs[t].hi = jobs[t].lo + chunk < count ? jobs[t].lo + chunk : count;
    if (jobs[t].lo >= jobs[t].hi) break;
    if (pthread_create(&tid[t], NULL, gg_thread_main, &jobs[t]) != 0) {
      gg_thread_main(&jobs[t]);
      tid[t] = 0;
    }
    started = t + 1;
  }
  for (int t = 0; t < started; ++t)
    if (tid[t]) pthread_join(tid[t], NULL);
}

/* ------------------------------------------------------- Fisher-Yates perm */
/* perm[i] = image of id i; stream 2^63+1 of the seed is reserved for it. */
void gg_permutation(uint32_t n, uint64_t seed, int32_t* perm) {
  for (uint32_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  uint64_t key = gg_key(seed, 0x8000000000000001ULL);
  for (uint32_t i = n; i > 1; --i) {
    uint32_t j = gg_below(gg_draw(key, n - i), i);
    int32_t t = perm[i - 1];
    perm[i - 1] = perm[j];
    perm[j] = t;
  }
}

/* --------------------------------------------------------------------- ER */
static void er_body(const gg_job* j, int64_t lo, int64_t hi) {
  for (int64_t i = lo; i < hi; ++i) {
    uint64_t key = gg_key(j->seed, (uint64_t)i);
    j->src[i] = (int32_t)gg_below(gg_draw(key, 0), j->n);
    j->dst[i] = (int32_t)gg_below(gg_draw(key, 1), j->n);
  }
}

/* E uniform pairs in [0,n).  Returns 0 on success. */
int gg_er(uint32_t n, int64_t num_edges, uint64_t seed, int32_t* src, int32_t* dst,
          int nthreads) {
  if (n == 0 || n > 0x7fffffffu || num_edges < 0) return 1;
  gg_job p;
  memset(&p, 0, sizeof p);
  p.body = er_body;
  p.seed = seed;
  p.n = n;
  p.src = src;
  p.dst = dst;
  gg_run(p, num_edges, nthreads);
  return 0;
}

/* ------------------------------------------------------------------ R-MAT */
static void rmat_body(const gg_job* j, int64_t lo, int64_t hi) {
  for (int64_t i = lo; i < hi; ++i) {
    uint64_t key = gg_key(j->seed, (uint64_t)i);
    uint32_t u = 0, v = 0;
    uint64_t r = 0;
    for (int l = 0; l < j->scale; ++l) {
      uint64_t p;
      if ((l & 1) == 0) {
        r = gg_draw(key, (uint64_t)(l >> 1));
        p = r >> 32;
      } else {
        p = r & 0xffffffffULL;
      }
      uint32_t bu, bv;
      if (p < j->thr_a) {
        bu = 0; bv = 0;
      } else if (p < j->thr_ab) {
        bu = 0; bv = 1;
      } else if (p < j->thr_abc) {
        bu = 1; bv = 0;
      } else {
        bu = 1; bv = 1;
      }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    if (j->perm) {
      j->src[i] = j->perm[u];
      j->dst[i] = j->perm[v];
    } else {
      j->src[i] = (int32_t)u;
      j->dst[i] = (int32_t)v;
    }
  }
}

/* R-MAT with 2^scale vertices and num_edges generated (directed) pairs.
 * permute != 0 relabels ids with gg_permutation(2^scale, seed). */
int gg_rmat(int scale, int64_t num_edges, double a, double b, double c, uint64_t seed,
            int permute, int32_t* src, int32_t* dst, int nthreads) {
  if (scale < 1 || scale > 30 || num_edges < 0) return 1;
  if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return 1;
  uint32_t n = 1u << scale;
  int32_t* perm = NULL;
  if (permute) {
    perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!perm) return 2;
    gg_permutation(n, seed, perm);
  }
  gg_job p;
  memset(&p, 0, sizeof p);
  p.body = rmat_body;
  p.seed = seed;
  p.n = n;
  p.scale = scale;
  p.thr_a = (uint64_t)(a * 4294967296.0);
  p.thr_ab = (uint64_t)((a + b) * 4294967296.0);
  p.thr_abc = (uint64_t)((a + b + c) * 4294967296.0);
  p.perm = perm;
  p.src = src;
  p.dst = dst;
  gg_run(p, num_edges, nthreads);
  free(perm);
  return 0;
}

/* --------------------------------------------------------------- Chung-Lu */
static void cl_body(const gg_job* j, int64_t lo, int64_t hi) {
  for (int64_t i = lo; i < hi; ++i) {
    uint64_t key = gg_key(j->seed, (uint64_t)i);
    uint32_t end[2];
    for (int s = 0; s < 2; ++s) {
      uint64_t r = gg_draw(key, (uint64_t)s);
      uint32_t col = gg_below(r, j->n);
      uint32_t coin = (uint32_t)(r & 0xffffffffULL);
      end[s] = coin < j->alias_thr[col] ? col : j->alias_idx[col];
    }
    if (j->perm) {
      j->src[i] = j->perm[end[0]];
      j->dst[i] = j->perm[end[1]];
    } else {
      j->src[i] = (int32_t)end[0];
      j->dst[i] = (int32_t)end[1];
    }
  }
}

/* Number of endpoint pairs gg_chunglu draws for (n, mean_deg). */
int64_t gg_chunglu_num_edges(uint32_t n, double mean_deg) {
  return (int64_t)llround((double)n * mean_deg / 2.0);
}

/* Chung-Lu graph; src/dst must hold gg_chunglu_num_edges(n, mean_deg) pairs. */
int gg_chunglu(uint32_t n, double gamma, double mean_deg, uint64_t seed, int permute,
               int32_t* src, int32_t* dst, int nthreads) {
  if (n < 2 || n > 0x7fffffffu || gamma <= 1.0 || mean_deg <= 0) return 1;
  int64_t num_edges = gg_chunglu_num_edges(n, mean_deg);
  double* w = (double*)malloc((size_t)n * sizeof(double));
  uint32_t* thr = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  uint32_t* ali = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  uint32_t* small = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  uint32_t* large = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
  int32_t* perm = permute ? (int32_t*)malloc((size_t)n * sizeof(int32_t)) : NULL;
  if (!w || !thr || !ali || !small || !large || (permute && !perm)) {
    free(w); free(thr); free(ali); free(small); free(large); free(perm);
    return 2;
  }
  double ex = -1.0 / (gamma - 1.0), sum = 0.0;
  for (uint32_t i = 0; i < n; ++i) {
    w[i] = pow((double)i + 1.0, ex);
    sum += w[i];
  }
  double total = (double)n * mean_deg, cap = sqrt(total), sc = total / sum;
  sum = 0.0;
  for (uint32_t i = 0; i < n; ++i) {
    w[i] *= sc;
    if (w[i] > cap) w[i] = cap;
    sum += w[i];
  }
  /* Vose alias table over probabilities w_i / sum, scaled by n. */
  uint32_t ns = 0, nl = 0;
  for (uint32_t i = 0; i < n; ++i) {
    w[i] = w[i] * (double)n / sum;
    if (w[i] < 1.0) small[ns++] = i; else large[nl++] = i;
  }
  while (ns > 0 && nl > 0) {
    uint32_t s = small[--ns], l = large[--nl];
    double t = w[s] * 4294967296.0;
    thr[s] = t >= 4294967295.0 ? 0xffffffffu : (uint32_t)t;
    ali[s] = l;
    w[l] = (w[l] + w[s]) - 1.0;
    if (w[l] < 1.0) small[ns++] = l; else large[nl++] = l;
  }
  while (nl > 0) { uint32_t l = large[--nl]; thr[l] = 0xffffffffu; ali[l] = l; }
  while (ns > 0) { uint32_t s = small[--ns]; thr[s] = 0xffffffffu; ali[s] = s; }
  if (permute) gg_permutation(n, seed, perm);
  gg_job p;
  memset(&p, 0, sizeof p);
  p.body = cl_body;
  p.seed = seed;
  p.n = n;
  p.alias_thr = thr;
  p.alias_idx = ali;
  p.perm = perm;
  p.src = src;
  p.dst = dst;
  gg_run(p, num_edges, nthreads);
  free(w); free(thr); free(ali); free(small); free(large); free(perm);
  return 0;
}
