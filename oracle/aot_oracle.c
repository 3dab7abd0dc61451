/*
 * aot_oracle.c - ORACLE for the AOT triangle-listing hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path, and the CUDA path never
 * calls it.  Plain, slow, single-threaded C; every count is an exact uint64.
 *
 * What it computes and where the paper defines it:
 *
 *  og_new           Input cleanup.  The method takes an undirected SIMPLE
 *                   graph (Sec. 2.1, problem statement); real inputs are
 *                   "processed appropriately" (Sec. 4, datasets).  Reading:
 *                   drop self-loops, merge duplicate and reversed pairs,
 *                   reject ids outside [0,n).  Adjacency sorted by vertex id.
 *  og_count         The plain definition of the output (Sec. 2.1): every
 *                   3-clique {a,b,c} once.  Edge iterator (Sec. 2.2) over the
 *                   id order: for each edge a<b, merge N(a) and N(b) keeping
 *                   c>b.  T and t(v) = number of triangles containing v.
 *  og_vertex_count  t(v) for a single vertex: edges among N(v).
 *  og_eta           The global total order of Sec. 1 / Sec. 2.2: degree
 *                   non-increasing, ties by smaller id (footnote to the
 *                   correctness argument of Sec. 3.2).  ORDER_ASC is the
 *                   degree non-decreasing variant that Example 1 uses.
 *                   ORDER_DEGEN is the degeneracy order that kClist orients
 *                   by (Sec. 2.3, Algorithm 2), see og_degeneracy.
 *  og_degeneracy    Core decomposition by peeling, level by level: at level
 *                   k every round removes ALL remaining vertices of current
 *                   degree <= k at once (their neighbours lose a degree per
 *                   removed neighbour), and k rises to the smallest
 *                   remaining degree when no vertex of degree <= k is left.
 *                   round[v] = the round that removed v, level[v] = its k
 *                   (the core number).  The degeneracy order is (round, id):
 *                   every vertex has at most level[v] later neighbours.
 *  og_orient        Orientation (Algorithm 3, first step): <u,v> iff
 *                   eta(u) < eta(v); out-lists in eta order (the local order
 *                   of Sec. 3.2).  Reported in rank space (id -> eta rank).
 *  og_costs         Cost counters of the analysis in Sec. 3.2 and Example 1:
 *                   sum deg+(v) (kClist, Sec. 2.3), sum min{deg+(u),deg+(v)}
 *                   (AOT), sum deg+(u)+deg+(v) (CF, Sec. 2.2), and the walk
 *                   length W of Algorithm 3 with ties broken by id and the
 *                   walk of a negative edge clipped to the part of N+(x)
 *                   after the pivot.
 *  og_work          Per-pivot item counts and walk sums of Algorithm 3
 *                   (positive: out-neighbour v with key(v) < key(u); negative:
 *                   in-neighbour x with key(x) < key(u); key = (deg+, rank)).
 *  og_work_rule     The same for three charging rules: Algorithm 3 with the
 *                   clip (= og_work), Algorithm 3 as printed (a negative edge
 *                   walks all of N+(u)), and the charging of kClist / CF
 *                   (Sec. 2.2, 2.3: every edge <u,v> walks N+(v) from u).
 *  og_costs_noclip  W of Algorithm 3 as printed (no clip).
 *  og_list_canonical  Every triangle once as (x,y,z) with eta(x)<eta(y)<eta(z),
 *                   sorted lexicographically by (eta(x),eta(y),eta(z)), written
 *                   in original ids.
 *  og_stream_vertex_counts  t(v) for a few sampled v straight from a raw edge
 *                   list, without building a graph (for huge inputs).
 *
 * Parallel paths (OpenMP; for the full-size parity tests and the CPU
 * baseline).  The serial functions above stay the definition: a -m "not gpu"
 * test checks each parallel function against them, and every count is still
 * an exact uint64 (per-thread partial sums added at the end).
 *
 *  og_new_par       og_new with the per-vertex sort and dedup spread over
 *                   threads (same cleaned graph).
 *  og_count_par     T and t(v) by the edge iterator of Sec. 2.2 (Algorithm 1,
 *                   CF) over the degree-ASCENDING orientation: for every
 *                   oriented <u,v>, merge N+(u) with N+(v); each common w
 *                   closes {u,v,w} once.  Parallel over u.
 *  og_list_canonical_par  the canonical list of og_list_canonical, produced
 *                   directly in its order: for x in eta order, for y in N+(x)
 *                   ascending, the z of N+(y) (ascending) that are marked as
 *                   members of N+(x).  Two passes (count per x, then write at
 *                   the prefix offset), parallel over x.
 *  og_threads       the number of threads the parallel paths use.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OG_OK 0
#define OG_ERR_ARG 1
#define OG_ERR_RANGE 2
#define OG_ERR_NOMEM 3

#define OG_ORDER_DESC 0
#define OG_ORDER_ASC 1
#define OG_ORDER_DEGEN 2

typedef struct {
  int32_t n;
  int64_t m;    /* undirected edges */
  int64_t* off; /* n+1, into adj (2m entries) */
  int32_t* adj; /* neighbours of each vertex, ascending id */
} og_graph;

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

void og_free(og_graph* g) {
  if (!g) return;
  free(g->off);
  free(g->adj);
  free(g);
}

og_graph* og_new(int32_t n, int64_t num_edges, const int32_t* src, const int32_t* dst,
                 int* status) {
  *status = OG_OK;
  if (n < 0 || num_edges < 0) { *status = OG_ERR_ARG; return NULL; }
  for (int64_t i = 0; i < num_edges; ++i) {
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) {
      *status = OG_ERR_RANGE;
      return NULL;
    }
  }
  og_graph* g = (og_graph*)calloc(1, sizeof(og_graph));
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!g || !cnt) { free(g); free(cnt); *status = OG_ERR_NOMEM; return NULL; }
  g->n = n;
  /* both directions of every non-loop pair */
  for (int64_t i = 0; i < num_edges; ++i) {
    if (src[i] == dst[i]) continue;
    cnt[src[i]]++;
    cnt[dst[i]]++;
  }
  int64_t* off = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!off) { free(g); free(cnt); *status = OG_ERR_NOMEM; return NULL; }
  off[0] = 0;
  for (int32_t v = 0; v < n; ++v) off[v + 1] = off[v] + cnt[v];
  int32_t* adj = (int32_t*)malloc((size_t)(off[n] > 0 ? off[n] : 1) * sizeof(int32_t));
  if (!adj) { free(g); free(cnt); free(off); *status = OG_ERR_NOMEM; return NULL; }
  for (int32_t v = 0; v < n; ++v) cnt[v] = off[v];
  for (int64_t i = 0; i < num_edges; ++i) {
    int32_t a = src[i], b = dst[i];
    if (a == b) continue;
    adj[cnt[a]++] = b;
    adj[cnt[b]++] = a;
  }
  /* sort each list and drop repeated neighbours; compact in place */
  int64_t w = 0;
  for (int32_t v = 0; v < n; ++v) {
    int64_t lo = off[v], hi = off[v + 1];
    qsort(adj + lo, (size_t)(hi - lo), sizeof(int32_t), cmp_i32);
    int64_t start = w;
    for (int64_t k = lo; k < hi; ++k)
      if (k == lo || adj[k] != adj[k - 1]) adj[w++] = adj[k];
    off[v] = start;
  }
  off[n] = w;
  free(cnt);
  g->off = off;
  g->adj = adj;
  g->m = w / 2;
  return g;
}

int32_t og_n(const og_graph* g) { return g->n; }
int64_t og_m(const og_graph* g) { return g->m; }
void og_degrees(const og_graph* g, int32_t* deg) {
  for (int32_t v = 0; v < g->n; ++v) deg[v] = (int32_t)(g->off[v + 1] - g->off[v]);
}
/* Copy the cleaned graph: off[n+1], adj[2m]. */
void og_copy(const og_graph* g, int64_t* off, int32_t* adj) {
  memcpy(off, g->off, ((size_t)g->n + 1) * sizeof(int64_t));
  memcpy(adj, g->adj, (size_t)g->off[g->n] * sizeof(int32_t));
}

/* ------------------------------------------------------------- counting */
/* Triangles {a<b<c}: for each edge a<b, the common neighbours c>b. */
uint64_t og_count(const og_graph* g, uint64_t* t /* n or NULL */) {
  uint64_t total = 0;
  if (t) memset(t, 0, (size_t)g->n * sizeof(uint64_t));
  for (int32_t a = 0; a < g->n; ++a) {
    for (int64_t i = g->off[a]; i < g->off[a + 1]; ++i) {
      int32_t b = g->adj[i];
      if (b <= a) continue;
      int64_t p = g->off[a], pe = g->off[a + 1];
      int64_t q = g->off[b], qe = g->off[b + 1];
      while (p < pe && q < qe) {
        int32_t x = g->adj[p], y = g->adj[q];
        if (x < y) { ++p; continue; }
        if (y < x) { ++q; continue; }
        if (x > b) {
          ++total;
          if (t) { t[a]++; t[b]++; t[x]++; }
        }
        ++p; ++q;
      }
    }
  }
  return total;
}

static int og_has_edge(const og_graph* g, int32_t a, int32_t b) {
  int64_t lo = g->off[a], hi = g->off[a + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (g->adj[mid] < b) lo = mid + 1; else hi = mid;
  }
  return lo < g->off[a + 1] && g->adj[lo] == b;
}

/* t(v) = number of edges {x,y} with x,y in N(v). */
uint64_t og_vertex_count(const og_graph* g, int32_t v) {
  uint64_t c = 0;
  for (int64_t i = g->off[v]; i < g->off[v + 1]; ++i)
    for (int64_t j = i + 1; j < g->off[v + 1]; ++j)
      c += (uint64_t)og_has_edge(g, g->adj[i], g->adj[j]);
  return c;
}

int og_is_triangle(const og_graph* g, int32_t a, int32_t b, int32_t c) {
  if (a < 0 || b < 0 || c < 0 || a >= g->n || b >= g->n || c >= g->n) return 0;
  return og_has_edge(g, a, b) && og_has_edge(g, b, c) && og_has_edge(g, a, c);
}

/* ----------------------------------------------------------------- order */
static const og_graph* s_sort_g;
static int s_sort_order;
static int cmp_eta(const void* pa, const void* pb) {
  int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
  int64_t da = s_sort_g->off[a + 1] - s_sort_g->off[a];
  int64_t db = s_sort_g->off[b + 1] - s_sort_g->off[b];
  if (da != db) {
    if (s_sort_order == OG_ORDER_DESC) return da > db ? -1 : 1;
    return da < db ? -1 : 1;
  }
  return (a > b) - (a < b);
}

static int cmp_u64(const void* a, const void* b);

/* Peeling rounds and levels (see the header).  Returns OG_ERR_NOMEM or OG_OK. */
int og_degeneracy(const og_graph* g, int32_t* round, int32_t* level) {
  int32_t n = g->n;
  int64_t* deg = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  int32_t* rem = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t)); /* remaining vertices */
  int32_t* fr = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));  /* this round's removals */
  if (!deg || !rem || !fr) { free(deg); free(rem); free(fr); return OG_ERR_NOMEM; }
  int32_t nrem = n, r = 0;
  int64_t k = 0;
  for (int32_t v = 0; v < n; ++v) {
    deg[v] = g->off[v + 1] - g->off[v];
    rem[v] = v;
    round[v] = -1;
  }
  while (nrem > 0) {
    int32_t nf = 0, keep = 0;
    for (int32_t i = 0; i < nrem; ++i) {
      int32_t v = rem[i];
      if (deg[v] <= k) fr[nf++] = v;
      else rem[keep++] = v;
    }
    if (nf == 0) { /* next level: the smallest remaining degree */
      k = deg[rem[0]];
      for (int32_t i = 1; i < nrem; ++i)
        if (deg[rem[i]] < k) k = deg[rem[i]];
      continue;
    }
    for (int32_t i = 0; i < nf; ++i) {
      round[fr[i]] = r;
      level[fr[i]] = (int32_t)k;
    }
    for (int32_t i = 0; i < nf; ++i) {
      int32_t v = fr[i];
      for (int64_t j = g->off[v]; j < g->off[v + 1]; ++j)
        if (round[g->adj[j]] < 0) deg[g->adj[j]]--;
    }
    nrem = keep;
    ++r;
  }
  free(deg); free(rem); free(fr);
  return OG_OK;
}

/* perm by ascending (round, id) of og_degeneracy */
static int og_eta_degen(const og_graph* g, int32_t* rank, int32_t* perm) {
  int32_t n = g->n;
  int32_t* round = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t* level = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  uint64_t* key = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
  if (!round || !level || !key || og_degeneracy(g, round, level) != OG_OK) {
    free(round); free(level); free(key);
    return OG_ERR_NOMEM;
  }
  for (int32_t v = 0; v < n; ++v) key[v] = ((uint64_t)(uint32_t)round[v] << 32) | (uint32_t)v;
  qsort(key, (size_t)n, sizeof(uint64_t), cmp_u64);
  for (int32_t r = 0; r < n; ++r) {
    perm[r] = (int32_t)(uint32_t)key[r];
    rank[perm[r]] = r;
  }
  free(round); free(level); free(key);
  return OG_OK;
}

/* perm[r] = vertex at eta position r, rank[v] = eta position of v. */
void og_eta(const og_graph* g, int order, int32_t* rank, int32_t* perm) {
  if (order == OG_ORDER_DEGEN) {
    og_eta_degen(g, rank, perm);
    return;
  }
  for (int32_t v = 0; v < g->n; ++v) perm[v] = v;
  s_sort_g = g;
  s_sort_order = order;
  qsort(perm, (size_t)g->n, sizeof(int32_t), cmp_eta);
  for (int32_t r = 0; r < g->n; ++r) rank[perm[r]] = r;
}

/* Oriented out-CSR in rank space: out_off[n+1], out_adj[m] ascending. */
static int og_orient_alloc(const og_graph* g, int order, int32_t** rank_o, int32_t** perm_o,
                           int64_t** off_o, int32_t** adj_o) {
  int32_t n = g->n;
  int32_t* rank = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t* perm = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  int64_t* off = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  int32_t* adj = (int32_t*)malloc(((size_t)g->m + 1) * sizeof(int32_t));
  if (!rank || !perm || !off || !adj) {
    free(rank); free(perm); free(off); free(adj);
    return OG_ERR_NOMEM;
  }
  og_eta(g, order, rank, perm);
  off[0] = 0;
  for (int32_t r = 0; r < n; ++r) {
    int32_t v = perm[r];
    int64_t k = off[r];
    for (int64_t i = g->off[v]; i < g->off[v + 1]; ++i) {
      int32_t rr = rank[g->adj[i]];
      if (rr > r) adj[k++] = rr;
    }
    qsort(adj + off[r], (size_t)(k - off[r]), sizeof(int32_t), cmp_i32);
    off[r + 1] = k;
  }
  *rank_o = rank; *perm_o = perm; *off_o = off; *adj_o = adj;
  return OG_OK;
}

int og_orient(const og_graph* g, int order, int32_t* rank, int32_t* perm, int64_t* out_off,
              int32_t* out_adj) {
  int32_t *rk, *pm, *adj;
  int64_t* off;
  int st = og_orient_alloc(g, order, &rk, &pm, &off, &adj);
  if (st) return st;
  memcpy(rank, rk, (size_t)g->n * sizeof(int32_t));
  memcpy(perm, pm, (size_t)g->n * sizeof(int32_t));
  memcpy(out_off, off, ((size_t)g->n + 1) * sizeof(int64_t));
  memcpy(out_adj, adj, (size_t)g->m * sizeof(int32_t));
  free(rk); free(pm); free(off); free(adj);
  return OG_OK;
}

/* key(x) < key(y) with key = (deg+, rank): the footnote's tie rule. */
static int key_less(const int64_t* off, int32_t x, int32_t y) {
  int64_t dx = off[x + 1] - off[x], dy = off[y + 1] - off[y];
  return dx < dy || (dx == dy && x < y);
}

/* Number of entries of N+(u) that are greater than v (rank space). */
static int64_t suffix_after(const int64_t* off, const int32_t* adj, int32_t u, int32_t v) {
  int64_t lo = off[u], hi = off[u + 1];
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (adj[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return off[u + 1] - lo;
}

/* out[0] = sum deg+(v) over <u,v>          (kClist cost, Sec. 2.3)
 * out[1] = sum min{deg+(u), deg+(v)}        (AOT bound, Sec. 3.2)
 * out[2] = sum deg+(u) + deg+(v)            (CF merge cost, Sec. 2.2)
 * out[3] = W: walk length of Algorithm 3, negative walks clipped after v
 * out[4] = number of positive edges (key(v) < key(u)) */
int og_costs(const og_graph* g, int order, uint64_t* out) {
  int32_t *rk, *pm, *adj;
  int64_t* off;
  int st = og_orient_alloc(g, order, &rk, &pm, &off, &adj);
  if (st) return st;
  uint64_t kc = 0, mn = 0, cf = 0, w = 0, pos = 0;
  for (int32_t u = 0; u < g->n; ++u) {
    uint64_t du = (uint64_t)(off[u + 1] - off[u]);
    for (int64_t i = off[u]; i < off[u + 1]; ++i) {
      int32_t v = adj[i];
      uint64_t dv = (uint64_t)(off[v + 1] - off[v]);
      kc += dv;
      mn += du < dv ? du : dv;
      cf += du + dv;
      if (key_less(off, v, u)) {
        w += dv;
        pos++;
      } else {
        w += (uint64_t)suffix_after(off, adj, u, v);
      }
    }
  }
  out[0] = kc; out[1] = mn; out[2] = cf; out[3] = w; out[4] = pos;
  free(rk); free(pm); free(off); free(adj);
  return OG_OK;
}

/* Per pivot p (rank space): items[p] = number of positive + negative items,
 * walk[p] = their summed walk lengths, staged[p] = deg+(p) if items[p] > 0. */
int og_work(const og_graph* g, int order, uint32_t* items, uint64_t* walk) {
  int32_t *rk, *pm, *adj;
  int64_t* off;
  int st = og_orient_alloc(g, order, &rk, &pm, &off, &adj);
  if (st) return st;
  memset(items, 0, (size_t)g->n * sizeof(uint32_t));
  memset(walk, 0, (size_t)g->n * sizeof(uint64_t));
  for (int32_t u = 0; u < g->n; ++u) {
    for (int64_t i = off[u]; i < off[u + 1]; ++i) {
      int32_t v = adj[i];
      if (key_less(off, v, u)) { /* positive: pivot u walks N+(v) */
        items[u]++;
        walk[u] += (uint64_t)(off[v + 1] - off[v]);
      } else { /* negative: pivot v walks N+(u) after v */
        items[v]++;
        walk[v] += (uint64_t)suffix_after(off, adj, u, v);
      }
    }
  }
  free(rk); free(pm); free(off); free(adj);
  return OG_OK;
}

/* rule 0: Algorithm 3 with the clip; 1: without it; 2: every edge walks
 * N+(v) from its tail u. */
int og_work_rule(const og_graph* g, int order, int rule, uint32_t* items, uint64_t* walk) {
  if (rule < 0 || rule > 2) return OG_ERR_ARG;
  int32_t *rk, *pm, *adj;
  int64_t* off;
  int st = og_orient_alloc(g, order, &rk, &pm, &off, &adj);
  if (st) return st;
  memset(items, 0, (size_t)g->n * sizeof(uint32_t));
  memset(walk, 0, (size_t)g->n * sizeof(uint64_t));
  for (int32_t u = 0; u < g->n; ++u) {
    for (int64_t i = off[u]; i < off[u + 1]; ++i) {
      int32_t v = adj[i];
      if (rule == 2 || key_less(off, v, u)) { /* pivot u walks N+(v) */
        items[u]++;
        walk[u] += (uint64_t)(off[v + 1] - off[v]);
      } else if (rule == 0) { /* pivot v walks N+(u) after v */
        items[v]++;
        walk[v] += (uint64_t)suffix_after(off, adj, u, v);
      } else { /* pivot v walks all of N+(u) */
        items[v]++;
        walk[v] += (uint64_t)(off[u + 1] - off[u]);
      }
    }
  }
  free(rk); free(pm); free(off); free(adj);
  return OG_OK;
}

/* W of Algorithm 3 without the clip: positive edges walk deg+(v), negative
 * edges deg+(u). */
int og_costs_noclip(const og_graph* g, int order, uint64_t* out) {
  int32_t *rk, *pm, *adj;
  int64_t* off;
  int st = og_orient_alloc(g, order, &rk, &pm, &off, &adj);
  if (st) return st;
  uint64_t w = 0;
  for (int32_t u = 0; u < g->n; ++u) {
    uint64_t du = (uint64_t)(off[u + 1] - off[u]);
    for (int64_t i = off[u]; i < off[u + 1]; ++i) {
      int32_t v = adj[i];
      w += key_less(off, v, u) ? (uint64_t)(off[v + 1] - off[v]) : du;
    }
  }
  *out = w;
  free(rk); free(pm); free(off); free(adj);
  return OG_OK;
}

/* ----------------------------------------------------------------- listing */
static int cmp_tri(const void* pa, const void* pb) {
  const int32_t* a = (const int32_t*)pa;
  const int32_t* b = (const int32_t*)pb;
  for (int k = 0; k < 3; ++k)
    if (a[k] != b[k]) return (a[k] > b[k]) - (a[k] < b[k]);
  return 0;
}

static void sort3(int32_t* x) {
  int32_t t;
  if (x[0] > x[1]) { t = x[0]; x[0] = x[1]; x[1] = t; }
  if (x[1] > x[2]) { t = x[1]; x[1] = x[2]; x[2] = t; }
  if (x[0] > x[1]) { t = x[0]; x[0] = x[1]; x[1] = t; }
}

/* All triangles as id-sorted triples (a<b<c), lexicographic.  Returns T;
 * writes only if out != NULL and cap >= T. */
uint64_t og_list_ids(const og_graph* g, int32_t* out, uint64_t cap) {
  uint64_t total = og_count(g, NULL);
  if (!out || cap < total) return total;
  uint64_t k = 0;
  for (int32_t a = 0; a < g->n; ++a)
    for (int64_t i = g->off[a]; i < g->off[a + 1]; ++i) {
      int32_t b = g->adj[i];
      if (b <= a) continue;
      int64_t p = g->off[a], pe = g->off[a + 1], q = g->off[b], qe = g->off[b + 1];
      while (p < pe && q < qe) {
        int32_t x = g->adj[p], y = g->adj[q];
        if (x < y) { ++p; continue; }
        if (y < x) { ++q; continue; }
        if (x > b) { out[3 * k] = a; out[3 * k + 1] = b; out[3 * k + 2] = x; ++k; }
        ++p; ++q;
      }
    }
  return total;
}

/* Canonical form: (x,y,z) with eta(x)<eta(y)<eta(z), sorted by eta triple. */
uint64_t og_list_canonical(const og_graph* g, int order, int32_t* out, uint64_t cap) {
  uint64_t total = og_count(g, NULL);
  if (!out || cap < total) return total;
  og_list_ids(g, out, cap);
  int32_t* rank = (int32_t*)malloc(((size_t)g->n + 1) * sizeof(int32_t));
  int32_t* perm = (int32_t*)malloc(((size_t)g->n + 1) * sizeof(int32_t));
  if (!rank || !perm) { free(rank); free(perm); return (uint64_t)-1; }
  og_eta(g, order, rank, perm);
  for (uint64_t k = 0; k < total; ++k) {
    int32_t* t = out + 3 * k;
    t[0] = rank[t[0]]; t[1] = rank[t[1]]; t[2] = rank[t[2]];
    sort3(t);
  }
  qsort(out, (size_t)total, 3 * sizeof(int32_t), cmp_tri);
  for (uint64_t k = 0; k < 3 * total; ++k) out[k] = perm[out[k]];
  free(rank); free(perm);
  return total;
}

/* ------------------------------------------------------- streaming sample */
/* t(v) for K sampled vertices from a raw edge list (loops/duplicates allowed).
 * Two passes: collect N(v); then collect the distinct pairs {x,y} inside N(v).
 * Memory: one n-byte mark array per sampled vertex, reused. */
static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

int og_stream_vertex_counts(int32_t n, int64_t num_edges, const int32_t* src,
                            const int32_t* dst, int32_t k, const int32_t* verts,
                            uint64_t* out) {
  uint8_t* mark = (uint8_t*)calloc((size_t)n, 1);
  if (!mark) return OG_ERR_NOMEM;
  for (int32_t s = 0; s < k; ++s) {
    int32_t v = verts[s];
    memset(mark, 0, (size_t)n);
    for (int64_t i = 0; i < num_edges; ++i) {
      if (src[i] == v && dst[i] != v) mark[dst[i]] = 1;
      if (dst[i] == v && src[i] != v) mark[src[i]] = 1;
    }
    uint64_t cap = 1024, cnt = 0;
    uint64_t* pairs = (uint64_t*)malloc(cap * sizeof(uint64_t));
    if (!pairs) { free(mark); return OG_ERR_NOMEM; }
    for (int64_t i = 0; i < num_edges; ++i) {
      int32_t a = src[i], b = dst[i];
      if (a == b || !mark[a] || !mark[b]) continue;
      if (a > b) { int32_t t = a; a = b; b = t; }
      if (cnt == cap) {
        cap *= 2;
        uint64_t* np = (uint64_t*)realloc(pairs, cap * sizeof(uint64_t));
        if (!np) { free(pairs); free(mark); return OG_ERR_NOMEM; }
        pairs = np;
      }
      pairs[cnt++] = ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
    }
    qsort(pairs, (size_t)cnt, sizeof(uint64_t), cmp_u64);
    uint64_t distinct = 0;
    for (uint64_t i = 0; i < cnt; ++i)
      if (i == 0 || pairs[i] != pairs[i - 1]) distinct++;
    out[s] = distinct;
    free(pairs);
  }
  free(mark);
  return OG_OK;
}

/* ---------------------------------------------------------- parallel paths */
int og_threads(int threads) {
#ifdef _OPENMP
  return threads > 0 ? threads : omp_get_max_threads();
#else
  (void)threads;
  return 1;
#endif
}

og_graph* og_new_par(int32_t n, int64_t num_edges, const int32_t* src, const int32_t* dst,
                     int* status, int threads) {
  *status = OG_OK;
  if (n < 0 || num_edges < 0) { *status = OG_ERR_ARG; return NULL; }
  int bad = 0;
  int nt = og_threads(threads);
#pragma omp parallel for num_threads(nt) reduction(| : bad) schedule(static)
  for (int64_t i = 0; i < num_edges; ++i)
    bad |= (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n);
  if (bad) { *status = OG_ERR_RANGE; return NULL; }
  og_graph* g = (og_graph*)calloc(1, sizeof(og_graph));
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* off = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!g || !cnt || !off) { free(g); free(cnt); free(off); *status = OG_ERR_NOMEM; return NULL; }
  g->n = n;
  for (int64_t i = 0; i < num_edges; ++i) {
    if (src[i] == dst[i]) continue;
    cnt[src[i]]++;
    cnt[dst[i]]++;
  }
  off[0] = 0;
  for (int32_t v = 0; v < n; ++v) off[v + 1] = off[v] + cnt[v];
  int32_t* adj = (int32_t*)malloc((size_t)(off[n] > 0 ? off[n] : 1) * sizeof(int32_t));
  if (!adj) { free(g); free(cnt); free(off); *status = OG_ERR_NOMEM; return NULL; }
  for (int32_t v = 0; v < n; ++v) cnt[v] = off[v];
  for (int64_t i = 0; i < num_edges; ++i) {
    int32_t a = src[i], b = dst[i];
    if (a == b) continue;
    adj[cnt[a]++] = b;
    adj[cnt[b]++] = a;
  }
  /* sort each list and drop repeats inside its own range; cnt[v] = kept */
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1024)
  for (int32_t v = 0; v < n; ++v) {
    int64_t lo = off[v], hi = off[v + 1], w = lo;
    qsort(adj + lo, (size_t)(hi - lo), sizeof(int32_t), cmp_i32);
    for (int64_t k = lo; k < hi; ++k)
      if (k == lo || adj[k] != adj[k - 1]) adj[w++] = adj[k];
    cnt[v] = w - lo;
  }
  /* compact in place (left shifts only, in vertex order) */
  int64_t w = 0;
  for (int32_t v = 0; v < n; ++v) {
    int64_t lo = off[v];
    if (w != lo) memmove(adj + w, adj + lo, (size_t)cnt[v] * sizeof(int32_t));
    off[v] = w;
    w += cnt[v];
  }
  off[n] = w;
  free(cnt);
  g->off = off;
  g->adj = adj;
  g->m = w / 2;
  return g;
}

/* eta as in og_eta, through a thread-safe sort of (degree key, id) words */
static int og_eta_keys(const og_graph* g, int order, int32_t* rank, int32_t* perm) {
  if (order == OG_ORDER_DEGEN) return og_eta_degen(g, rank, perm);
  int32_t n = g->n;
  uint64_t* key = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
  if (!key) return OG_ERR_NOMEM;
  for (int32_t v = 0; v < n; ++v) {
    uint64_t d = (uint64_t)(g->off[v + 1] - g->off[v]);
    uint64_t k = order == OG_ORDER_DESC ? (0xffffffffull - d) : d;
    key[v] = (k << 32) | (uint32_t)v;
  }
  qsort(key, (size_t)n, sizeof(uint64_t), cmp_u64);
  for (int32_t r = 0; r < n; ++r) {
    perm[r] = (int32_t)(uint32_t)key[r];
    rank[perm[r]] = r;
  }
  free(key);
  return OG_OK;
}

/* Oriented out-CSR in rank space (same result as og_orient_alloc). */
static int og_orient_par(const og_graph* g, int order, int nt, int32_t** rank_o, int32_t** perm_o,
                         int64_t** off_o, int32_t** adj_o) {
  int32_t n = g->n;
  int32_t* rank = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t* perm = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  int64_t* off = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  int32_t* adj = (int32_t*)malloc(((size_t)g->m + 1) * sizeof(int32_t));
  if (!rank || !perm || !off || !adj || og_eta_keys(g, order, rank, perm) != OG_OK) {
    free(rank); free(perm); free(off); free(adj);
    return OG_ERR_NOMEM;
  }
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1024)
  for (int32_t r = 0; r < n; ++r) {
    int32_t v = perm[r];
    int64_t c = 0;
    for (int64_t i = g->off[v]; i < g->off[v + 1]; ++i) c += rank[g->adj[i]] > r;
    off[r + 1] = c;
  }
  off[0] = 0;
  for (int32_t r = 0; r < n; ++r) off[r + 1] += off[r];
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1024)
  for (int32_t r = 0; r < n; ++r) {
    int32_t v = perm[r];
    int64_t k = off[r];
    for (int64_t i = g->off[v]; i < g->off[v + 1]; ++i) {
      int32_t rr = rank[g->adj[i]];
      if (rr > r) adj[k++] = rr;
    }
    qsort(adj + off[r], (size_t)(k - off[r]), sizeof(int32_t), cmp_i32);
  }
  *rank_o = rank; *perm_o = perm; *off_o = off; *adj_o = adj;
  return OG_OK;
}

/* T, and t(v) (original ids) when t != NULL.  Returns (uint64_t)-1 when out
 * of memory. */
uint64_t og_count_par(const og_graph* g, uint64_t* t, int threads) {
  int nt = og_threads(threads);
  int32_t *rank, *perm, *adj;
  int64_t* off;
  if (og_orient_par(g, OG_ORDER_ASC, nt, &rank, &perm, &off, &adj) != OG_OK) return (uint64_t)-1;
  int32_t n = g->n;
  uint64_t* tl = NULL; /* one rank-space count array per thread */
  if (t) {
    tl = (uint64_t*)calloc((size_t)nt * ((size_t)n + 1), sizeof(uint64_t));
    if (!tl) { free(rank); free(perm); free(off); free(adj); return (uint64_t)-1; }
  }
  uint64_t total = 0;
#pragma omp parallel num_threads(nt) reduction(+ : total)
  {
#ifdef _OPENMP
    uint64_t* my = tl ? tl + (size_t)omp_get_thread_num() * ((size_t)n + 1) : NULL;
#else
    uint64_t* my = tl;
#endif
#pragma omp for schedule(dynamic, 64)
    for (int32_t u = 0; u < n; ++u) {
      for (int64_t i = off[u]; i < off[u + 1]; ++i) {
        int32_t v = adj[i];
        /* every entry of N+(v) is above v, so the merge starts after v in N+(u) */
        int64_t p = i + 1, pe = off[u + 1], q = off[v], qe = off[v + 1];
        uint64_t c = 0;
        while (p < pe && q < qe) {
          int32_t x = adj[p], y = adj[q];
          if (x < y) { ++p; continue; }
          if (y < x) { ++q; continue; }
          ++c;
          if (my) my[x]++;
          ++p; ++q;
        }
        total += c;
        if (my) { my[u] += c; my[v] += c; }
      }
    }
  }
  if (t) {
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int32_t r = 0; r < n; ++r) {
      uint64_t s = 0;
      for (int k = 0; k < nt; ++k) s += tl[(size_t)k * ((size_t)n + 1) + r];
      t[perm[r]] = s;
    }
    free(tl);
  }
  free(rank); free(perm); free(off); free(adj);
  return total;
}

/* Canonical list (see og_list_canonical).  Returns T; writes only if
 * out != NULL and cap >= T; (uint64_t)-1 when out of memory. */
uint64_t og_list_canonical_par(const og_graph* g, int order, int32_t* out, uint64_t cap,
                               int threads) {
  int nt = og_threads(threads);
  int32_t *rank, *perm, *adj;
  int64_t* off;
  if (og_orient_par(g, order, nt, &rank, &perm, &off, &adj) != OG_OK) return (uint64_t)-1;
  int32_t n = g->n;
  uint64_t* per = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
  uint8_t* marks = (uint8_t*)calloc((size_t)nt * ((size_t)n + 1), 1);
  if (!per || !marks) {
    free(per); free(marks); free(rank); free(perm); free(off); free(adj);
    return (uint64_t)-1;
  }
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      uint64_t run = 0;
      for (int32_t x = 0; x < n; ++x) { uint64_t c = per[x]; per[x] = run; run += c; }
      per[n] = run;
      if (!out || cap < run) break;
    }
#pragma omp parallel num_threads(nt)
    {
#ifdef _OPENMP
      uint8_t* mk = marks + (size_t)omp_get_thread_num() * ((size_t)n + 1);
#else
      uint8_t* mk = marks;
#endif
#pragma omp for schedule(dynamic, 64)
      for (int32_t x = 0; x < n; ++x) {
        for (int64_t i = off[x]; i < off[x + 1]; ++i) mk[adj[i]] = 1;
        uint64_t k = pass == 1 ? per[x] : 0;
        for (int64_t i = off[x]; i < off[x + 1]; ++i) {
          int32_t y = adj[i];
          for (int64_t j = off[y]; j < off[y + 1]; ++j) {
            int32_t z = adj[j];
            if (!mk[z]) continue;
            if (pass == 1) {
              out[3 * k] = perm[x];
              out[3 * k + 1] = perm[y];
              out[3 * k + 2] = perm[z];
            }
            ++k;
          }
        }
        if (pass == 0) per[x] = k;
        for (int64_t i = off[x]; i < off[x + 1]; ++i) mk[adj[i]] = 0;
      }
    }
  }
  uint64_t total = per[n];
  free(per); free(marks); free(rank); free(perm); free(off); free(adj);
  return total;
}
