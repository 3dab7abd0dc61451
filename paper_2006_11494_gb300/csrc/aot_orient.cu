// aot_orient.cu - orientation of an undirected edge list into the oriented
// out-CSR of Algorithm 3 (first step) and the per-pivot work items of its
// adaptive orientation (Sec. 3.1-3.2).
//
//  cleanup   key = (min << b) | max per non-loop pair, radix sort, unique
//            (the input is an undirected simple graph, Sec. 2.1)
//  degree    deg(v) over unique edges (warp-aggregated atomics)
//  eta       stable radix sort of ids by degree (non-increasing by default),
//            so ties keep the smaller id first (footnote of Sec. 3.2)
//  orient    relabel to eta rank, key = (min rank << b) | max rank, radix
//            sort: out-lists come out sorted by eta (the local order, Sec. 3.2)
//  items     edge <u,v>: positive item of pivot u walking N+(v) if
//            key(v) < key(u), else negative item of pivot v walking the part
//            of N+(u) after v; key = (deg+, rank)
//  bins      pivots with items, grouped by deg+ for the intersection kernels
#include "aot_internal.cuh"

namespace aot {

constexpr uint64_t INVALID_KEY = ~0ull;

__global__ void k_make_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            int64_t E, int32_t n, int bits, uint64_t* __restrict__ keys,
                            DevScalars* dev) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  int32_t a = src[i], b = dst[i];
  uint64_t k = INVALID_KEY;
  if (a < 0 || a >= n || b < 0 || b >= n) {
    atomicOr(&dev->err, DEVERR_RANGE);
  } else if (a != b) {
    uint32_t lo = (uint32_t)min(a, b), hi = (uint32_t)max(a, b);
    k = ((uint64_t)lo << bits) | hi;
  }
  keys[i] = k;
}

__global__ void k_unique_flags(const uint64_t* __restrict__ keys, int64_t E,
                               uint32_t* __restrict__ flags) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  uint64_t k = keys[i];
  flags[i] = (k != INVALID_KEY && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
}

// warp-aggregated atomicAdd of 1 to cnt[key]
__device__ __forceinline__ void agg_inc(uint32_t* cnt, uint32_t key, bool active) {
  unsigned grp = __match_any_sync(FULL, active ? key : 0xffffffffu);
  if (active && lane_id() == (unsigned)(__ffs(grp) - 1)) atomicAdd(&cnt[key], (uint32_t)__popc(grp));
}

__global__ void k_compact_unique(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ flags,
                                 const uint32_t* __restrict__ pos, int64_t E, int bits,
                                 uint64_t* __restrict__ ukeys, uint32_t* __restrict__ deg) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool act = i < E && flags[i];
  uint64_t k = act ? keys[i] : 0;
  if (act) ukeys[pos[i]] = k;
  uint32_t lo = (uint32_t)(k >> bits), hi = (uint32_t)(k & ((1ull << bits) - 1));
  agg_inc(deg, lo, act);
  agg_inc(deg, hi, act);
}

__global__ void k_eta_keys(const uint32_t* __restrict__ deg, int32_t n, int bits, bool desc,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ ids) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint32_t d = deg[v];
  keys[v] = desc ? (uint32_t)(((1ull << bits) - 1) - d) : d;
  ids[v] = (uint32_t)v;
}

// ---------------------------------------------- degeneracy order (peeling)
// The degeneracy order of kClist (Sec. 2.3, Algorithm 2), computed level by
// level: at level k each round removes every remaining vertex of current
// degree <= k at once, and k rises to the smallest remaining degree when
// none is left; eta = (round, id).  Every vertex then has at most its core
// number of later neighbours.
constexpr uint32_t UNSET = 0xffffffffu;

// both directions of every unique edge, at the cursors of a copy of the offsets
__global__ void k_sym_fill(const uint64_t* __restrict__ ukeys, int64_t m, int bits,
                           uint32_t* __restrict__ cursor, uint32_t* __restrict__ sadj) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint64_t k = ukeys[i];
  const uint32_t lo = (uint32_t)(k >> bits), hi = (uint32_t)(k & ((1ull << bits) - 1));
  sadj[atomicAdd(&cursor[lo], 1u)] = hi;
  sadj[atomicAdd(&cursor[hi], 1u)] = lo;
}

// warp-aggregated append of v to list[*cnt]
__device__ __forceinline__ void warp_append(bool in, uint32_t v, uint32_t* list, unsigned int* cnt) {
  const unsigned bal = __ballot_sync(FULL, in);
  if (!bal) return;
  const unsigned leader = (unsigned)(__ffs(bal) - 1);
  uint32_t base = 0;
  if (lane_id() == leader) base = atomicAdd(cnt, (unsigned)__popc(bal));
  base = __shfl_sync(FULL, base, leader);
  if (in) list[base + __popc(bal & lanemask_lt())] = v;
}

// the first frontier of level k: every remaining vertex of degree <= k
__global__ void k_peel_scan(const uint32_t* __restrict__ cur, const uint32_t* __restrict__ rnd,
                            int32_t n, uint32_t k, uint32_t* __restrict__ frontier, unsigned int* cnt) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = v < n && rnd[v] == UNSET && cur[v] <= k;
  warp_append(in, (uint32_t)v, frontier, cnt);
}

// the smallest degree of a remaining vertex
__global__ void k_peel_min(const uint32_t* __restrict__ cur, const uint32_t* __restrict__ rnd, int32_t n,
                           unsigned int* out) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t d = v < n && rnd[v] == UNSET ? cur[v] : UNSET;
  d = __reduce_min_sync(FULL, d);
  if (lane_id() == 0 && d != UNSET) atomicMin(out, d);
}

// One round, a warp per frontier vertex v: round[v] = r, and every remaining
// neighbour w loses one degree; the w whose degree drops from k+1 to k join
// the next frontier (exactly one decrement sees that step).  A neighbour in
// the same frontier may still read as remaining: its degree (already <= k)
// only drops further and it is never appended again.
__global__ void k_peel_round(const uint32_t* __restrict__ frontier, uint32_t nf, uint32_t r, uint32_t k,
                             const uint32_t* __restrict__ soff, const uint32_t* __restrict__ sadj,
                             uint32_t* __restrict__ cur, uint32_t* __restrict__ rnd,
                             uint32_t* __restrict__ next, unsigned int* ncnt) {
  const unsigned lane = lane_id();
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t f = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < nf; f += warps) {
    const uint32_t v = frontier[f];
    if (lane == 0) rnd[v] = r;
    const uint32_t b = soff[v], e = soff[v + 1];
    for (uint32_t i0 = b; i0 < e; i0 += 32) {
      const uint32_t i = i0 + lane;
      bool join = false;
      uint32_t w = 0;
      if (i < e) {
        w = sadj[i];
        if (rnd[w] == UNSET) join = atomicSub(&cur[w], 1u) == k + 1;
      }
      warp_append(join, w, next, ncnt);
    }
  }
}

__global__ void k_iota(uint32_t* __restrict__ a, int32_t n) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) a[v] = (uint32_t)v;
}

__global__ void k_rank_from_perm(const uint32_t* __restrict__ perm_sorted, int32_t n,
                                 const uint32_t* __restrict__ deg, int32_t* __restrict__ perm,
                                 int32_t* __restrict__ rank, uint32_t* __restrict__ degr) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  uint32_t v = perm_sorted[r];
  perm[r] = (int32_t)v;
  rank[v] = (int32_t)r;
  degr[r] = deg[v];
}

// Random local order (AOT-randomOrder of Sec. 4.2): the out-lists are sorted
// by a bijection h of the head rank on `bits`-bit words instead of the rank
// itself, h(x) = ((x ^ (x >> sh)) * mul) mod 2^bits with mul odd, so every
// list comes out in the same fixed pseudo-random order.  LocalOrder{0, 0}
// is the identity (the eta local order of Sec. 3.2).
struct LocalOrder {
  uint32_t mul, inv;  // odd multiplier and its inverse mod 2^bits (0: identity)
  int sh;
};
__device__ __forceinline__ uint32_t lo_hash(uint32_t x, const LocalOrder& o, uint32_t mask) {
  return o.mul ? ((x ^ (x >> o.sh)) * o.mul) & mask : x;
}
__device__ __forceinline__ uint32_t lo_unhash(uint32_t y, const LocalOrder& o, uint32_t mask, int bits) {
  if (!o.mul) return y;
  uint32_t x = (y * o.inv) & mask;  // undo the multiplication, then the xor-shift
  uint32_t r = x;
  for (int k = o.sh; k < bits; k += o.sh) r = x ^ (r >> o.sh);
  return r;
}

__global__ void k_relabel(const uint64_t* __restrict__ ukeys, int64_t m, int bits,
                          const int32_t* __restrict__ rank, LocalOrder lo_ord,
                          uint64_t* __restrict__ okeys) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint32_t mask = (uint32_t)((1ull << bits) - 1);
  uint64_t k = ukeys[i];
  uint32_t a = (uint32_t)rank[(uint32_t)(k >> bits)];
  uint32_t b = (uint32_t)rank[(uint32_t)(k & mask)];
  uint32_t lo = min(a, b), hi = max(a, b);
  okeys[i] = ((uint64_t)lo << bits) | lo_hash(hi, lo_ord, mask);
}

__global__ void k_split_csr(const uint64_t* __restrict__ okeys, int64_t m, int bits,
                            LocalOrder lo_ord, uint32_t* __restrict__ adj,
                            uint32_t* __restrict__ esrc, uint32_t* __restrict__ outdeg) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool act = i < m;
  uint64_t k = act ? okeys[i] : 0;
  uint32_t u = (uint32_t)(k >> bits);
  if (act) {
    const uint32_t mask = (uint32_t)((1ull << bits) - 1);
    adj[i] = lo_unhash((uint32_t)(k & mask), lo_ord, mask, bits);
    esrc[i] = u;
  }
  agg_inc(outdeg, u, act);
}

__global__ void k_max_outdeg(const uint32_t* __restrict__ outdeg, int32_t n, DevScalars* dev) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t d = v < n ? outdeg[v] : 0u;
  d = __reduce_max_sync(FULL, d);
  if (lane_id() == 0 && d) atomicMax(&dev->counters[0], d);
}

__device__ __forceinline__ bool key_less(uint32_t dx, uint32_t x, uint32_t dy, uint32_t y) {
  return dx < dy || (dx == dy && x < y);
}

// Work item rules (orientation flags):
//   RULE_AOT      Algorithm 3 with the suffix clip: a negative item walks
//                 only the part of N+(u) after v (eta-sorted lists)
//   RULE_NOCLIP   Algorithm 3 as printed: a negative item walks all of N+(u)
//   RULE_TAIL     no adaptive choice: every edge is an item of its tail u
//                 walking N+(v), the charging of Sec. 2.2 / Sec. 2.3 (with
//                 the probe route the work of kClist, Algorithm 2, with the
//                 merge route that of CF, Algorithm 1)
enum ItemRule { RULE_AOT = 0, RULE_NOCLIP = 1, RULE_TAIL = 2 };

// pivot of oriented edge e = <u,v> and its walk range
__device__ __forceinline__ void edge_item(int64_t e, const uint32_t* __restrict__ esrc,
                                          const uint32_t* __restrict__ adj,
                                          const uint32_t* __restrict__ off,
                                          const uint32_t* __restrict__ outdeg, int rule,
                                          uint32_t& pivot, uint32_t& vert, uint2& range) {
  uint32_t u = esrc[e], v = adj[e];
  uint32_t du = outdeg[u], dv = outdeg[v];
  if (rule == RULE_TAIL || key_less(dv, v, du, u)) {  // positive edge: pivot u walks N+(v)
    pivot = u;
    vert = v;
    range = make_uint2(off[v], off[v] + dv);
  } else {  // negative edge: pivot v walks N+(u) (after v with the clip)
    pivot = v;
    vert = u;
    range = make_uint2(rule == RULE_AOT ? (uint32_t)e + 1 : off[u], off[u] + du);
  }
}

// items per pivot, and posflag[e] = 1 for a positive edge (its pivot is its tail)
__global__ void k_item_count(const uint32_t* __restrict__ esrc, const uint32_t* __restrict__ adj,
                             const uint32_t* __restrict__ off, const uint32_t* __restrict__ outdeg,
                             int64_t m, int rule, uint32_t* __restrict__ items,
                             uint32_t* __restrict__ posflag) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool act = e < m;
  uint32_t p = 0, x;
  uint2 r;
  if (act) {
    edge_item(e, esrc, adj, off, outdeg, rule, p, x, r);
    posflag[e] = p == esrc[e] ? 1u : 0u;
  }
  agg_inc(items, p, act);
}

// Item slots.  A pivot's positive items come first, in out-list order (so
// sorted by the walked vertex): the slot of positive edge e of row u is its
// rank among the row's positive edges, from the exclusive scan pscan of the
// positive flags.  Negative items follow in arrival order (atomic cursor).
__global__ void k_item_fill(const uint32_t* __restrict__ esrc, const uint32_t* __restrict__ adj,
                            const uint32_t* __restrict__ off, const uint32_t* __restrict__ outdeg,
                            int64_t m, int rule, const uint32_t* __restrict__ wofs,
                            const uint32_t* __restrict__ pscan, uint32_t* __restrict__ cursor,
                            uint2* __restrict__ witem, uint32_t* __restrict__ wvert,
                            uint32_t* __restrict__ wedge) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool act = e < m;
  uint32_t p = 0, x = 0;
  uint2 r = make_uint2(0, 0);
  bool pos = false;
  if (act) {
    edge_item(e, esrc, adj, off, outdeg, rule, p, x, r);
    pos = p == esrc[e];
  }
  const bool neg = act && !pos;
  unsigned grp = __match_any_sync(FULL, neg ? p : 0xffffffffu);
  unsigned leader = (unsigned)(__ffs(grp) - 1);
  uint32_t base = 0;
  if (neg && lane_id() == leader) base = atomicAdd(&cursor[p], (uint32_t)__popc(grp));
  base = __shfl_sync(FULL, base, leader);
  if (act) {
    uint32_t slot;
    if (pos) {
      slot = wofs[p] + (pscan[e] - pscan[off[p]]);
    } else {
      const uint32_t npos = pscan[off[p + 1]] - pscan[off[p]];
      slot = wofs[p] + npos + base + (uint32_t)__popc(grp & lanemask_lt());
    }
    witem[slot] = r;
    wvert[slot] = x;
    wedge[slot] = (uint32_t)e;
  }
}

// Per pivot: walk[p] = summed walk length of its items, and the totals W,
// S += deg+(p) and merge work += items(p) deg+(p) (a merge of each item's
// walk with N+(p) reads deg+(p) more entries).  A thread sums a pivot of at
// most PW_SMALL items; larger pivots are listed for k_pivot_walk_big.
constexpr uint32_t PW_SMALL = 64;
__global__ void k_pivot_walk(const uint32_t* __restrict__ wofs, const uint2* __restrict__ witem,
                             const uint32_t* __restrict__ outdeg, int32_t n, uint64_t* __restrict__ walk,
                             uint32_t* __restrict__ big, DevScalars* dev) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t w = 0, st = 0, mw = 0;
  bool large = false;
  if (p < n) {
    const uint32_t b = wofs[p], e = wofs[p + 1];
    const uint64_t d = outdeg[p];
    if (e > b) {
      st = d;
      mw = (uint64_t)(e - b) * d;
    }
    large = e - b > PW_SMALL;
    if (!large) {
      for (uint32_t i = b; i < e; ++i) {
        const uint2 r = witem[i];
        w += r.y - r.x;
      }
      walk[p] = w;
    }
  }
  const unsigned bal = __ballot_sync(FULL, large);
  if (bal) {
    const unsigned leader = (unsigned)(__ffs(bal) - 1);
    uint32_t base = 0;
    if (lane_id() == leader) base = atomicAdd(&dev->counters[13], (unsigned)__popc(bal));
    base = __shfl_sync(FULL, base, leader);
    if (large) big[base + (uint32_t)__popc(bal & lanemask_lt())] = (uint32_t)p;
  }
  w = warp_sum(w);
  st = warp_sum(st);
  mw = warp_sum(mw);
  if (lane_id() == 0) {
    if (w) atomicAdd(&dev->total, (unsigned long long)w);
    if (st) atomicAdd(&dev->aux[0], (unsigned long long)st);
    if (mw) atomicAdd(&dev->aux[1], (unsigned long long)mw);
  }
}

// a warp per listed pivot (more than PW_SMALL items)
__global__ void k_pivot_walk_big(const uint32_t* __restrict__ wofs, const uint2* __restrict__ witem,
                                 const uint32_t* __restrict__ big, uint64_t* __restrict__ walk,
                                 DevScalars* dev) {
  const uint32_t nbig = dev->counters[13];
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  uint64_t tot = 0;
  for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nbig; k += warps) {
    const uint32_t p = big[k];
    const uint32_t b = wofs[p], e = wofs[p + 1];
    uint64_t w = 0;
    uint32_t i = b + lane_id();
    for (; i + 96 < e; i += 128) {  // four independent loads in flight per lane
      const uint2 r0 = witem[i], r1 = witem[i + 32], r2 = witem[i + 64], r3 = witem[i + 96];
      w += (uint64_t)(r0.y - r0.x) + (r1.y - r1.x) + (r2.y - r2.x) + (r3.y - r3.x);
    }
    for (; i < e; i += 32) {
      const uint2 r = witem[i];
      w += r.y - r.x;
    }
    w = warp_sum(w);
    if (lane_id() == 0) walk[p] = w;
    tot += w;
  }
  if (lane_id() == 0 && tot) atomicAdd(&dev->total, (unsigned long long)tot);
}

// --------------------------------------------------------------------- bins
__global__ void k_bin_flags(const uint32_t* __restrict__ items, const uint32_t* __restrict__ outdeg,
                            int32_t n, uint32_t warp_max, uint32_t cta_max, int bin,
                            uint32_t* __restrict__ flag) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  uint32_t d = outdeg[p];
  int b = d <= warp_max ? BIN_WARP : (d <= cta_max ? BIN_CTA : BIN_HUB);
  flag[p] = (items[p] > 0 && b == bin) ? 1u : 0u;
}

__global__ void k_bin_scatter(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                              int32_t n, uint32_t base, uint32_t* __restrict__ out) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  if (flag[p]) out[base + pos[p]] = (uint32_t)p;
}

__global__ void k_bin_stats(const uint32_t* __restrict__ items, const uint32_t* __restrict__ outdeg,
                            const uint64_t* __restrict__ walk, int32_t n, uint32_t warp_max,
                            uint32_t cta_max, DevScalars* dev) {
  __shared__ unsigned long long acc[4 * NUM_BINS];
  if (threadIdx.x < 4 * NUM_BINS) acc[threadIdx.x] = 0;
  __syncthreads();
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n && items[p] > 0) {
    uint32_t d = outdeg[p];
    int b = d <= warp_max ? BIN_WARP : (d <= cta_max ? BIN_CTA : BIN_HUB);
    atomicAdd(&acc[4 * b + 0], 1ull);
    atomicAdd(&acc[4 * b + 1], (unsigned long long)items[p]);
    atomicAdd(&acc[4 * b + 2], (unsigned long long)walk[p]);
    atomicAdd(&acc[4 * b + 3], (unsigned long long)d);
  }
  __syncthreads();
  if (threadIdx.x < 4 * NUM_BINS && acc[threadIdx.x]) atomicAdd(&dev->bins[threadIdx.x], acc[threadIdx.x]);
}

static inline unsigned grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return (unsigned)(g < 1 ? 1 : g);
}

aot_status bin_pivots(aot_graph* g, cudaStream_t s) {
  const int T = 256;
  uint32_t base = 0;
  for (int b = 0; b < NUM_BINS; ++b) {
    uint32_t cnt = 0;
    if (g->n > 0) {
      AOT_KERNEL("k_bin_flags", s)
        k_bin_flags<<<grid_for(g->n, T), T, 0, s>>>(g->items, g->outdeg, g->n,
                                                  g->tune.warp_max_outdeg,
                                                  g->tune.cta_max_outdeg, b, g->bin_flag);
      AOT_TRY(last_launch());
      AOT_TRY(scan_u32_u32(g->bin_flag, g->bin_pos, g->n, g->scan_tmp, s));
      AOT_KERNEL("k_bin_scatter", s)
        k_bin_scatter<<<grid_for(g->n, T), T, 0, s>>>(g->bin_flag, g->bin_pos, g->n, base,
                                                    g->bin_pivots);
      AOT_TRY(last_launch());
      AOT_CUDA(cudaMemcpyAsync(&cnt, g->bin_pos + g->n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
      AOT_CUDA(cudaStreamSynchronize(s));
    }
    g->bin_count[b] = cnt;
    base += cnt;
  }
  AOT_CUDA(cudaMemsetAsync(g->dev->bins, 0, sizeof(g->dev->bins), s));
  if (g->n > 0) {
    AOT_KERNEL("k_bin_stats", s)
      k_bin_stats<<<grid_for(g->n, T), T, 0, s>>>(g->items, g->outdeg, g->walk, g->n,
                                                  g->tune.warp_max_outdeg, g->tune.cta_max_outdeg,
                                                  g->dev);
    AOT_TRY(last_launch());
  }
  unsigned long long hb[4 * NUM_BINS];
  AOT_CUDA(cudaMemcpyAsync(hb, g->dev->bins, sizeof(hb), cudaMemcpyDeviceToHost, s));
  AOT_CUDA(cudaStreamSynchronize(s));
  for (int b = 0; b < NUM_BINS; ++b)
    for (int k = 0; k < 4; ++k) g->bin_stats[b][k] = hb[4 * b + k];
  g->binned_warp_max = g->tune.warp_max_outdeg;
  g->binned_cta_max = g->tune.cta_max_outdeg;
  return AOT_OK;
}

aot_status read_device_error(aot_graph* g, cudaStream_t s) {
  uint32_t err = 0;
  AOT_CUDA(cudaMemcpyAsync(&err, &g->dev->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  AOT_CUDA(cudaStreamSynchronize(s));
  if (err & DEVERR_RANGE) return AOT_ERR_VERTEX_RANGE;
  if (err & DEVERR_TIMEOUT) return AOT_ERR_TIMEOUT;
  if (err & DEVERR_CHECK) return AOT_ERR_DEVICE_CHECK;
  return AOT_OK;
}

// ---------------------------------------------------------------- workspace
struct OrientLayout {
  DevScalars* dev;
  uint64_t* keysA;
  uint64_t* keysB;
  uint32_t* flags;
  uint32_t* pos;
  uint32_t* deg;
  uint32_t* ek0; uint32_t* ek1; uint32_t* ev0; uint32_t* ev1;
  int32_t* perm; int32_t* rank; uint32_t* degr;
  uint32_t* off; uint32_t* adj; uint32_t* outdeg;
  uint32_t* wofs; uint32_t* items; uint64_t* walk;
  uint32_t* bin_pivots; uint32_t* bin_flag; uint32_t* bin_pos;
  uint32_t* hub_bitmap;
  uint32_t* hubinfo;
  uint64_t* tv;
  uint32_t* tcnt; uint64_t* toff;
  uint8_t* route; uint32_t* rprobe; uint2* eplist;
  void* tmp;
  size_t bytes;
};

static OrientLayout carve_orient(void* base, int64_t E, int32_t n, uint32_t flags, const Tuning& t) {
  OrientLayout L;
  Carve c(base);
  int64_t Es = E > 0 ? E : 1;
  int64_t ns = n > 0 ? n : 1;
  L.dev = c.take<DevScalars>(1);
  L.keysA = c.take<uint64_t>(Es);
  L.keysB = c.take<uint64_t>(Es);
  // flags and pos are dead once the work items exist; the staging-free item
  // list of the counting phase reuses them (8 (E+1) bytes)
  L.flags = c.take<uint32_t>(2 * (Es + 1));
  L.pos = L.flags + (Es + 1);
  L.deg = c.take<uint32_t>(ns);
  L.ek0 = c.take<uint32_t>(ns); L.ek1 = c.take<uint32_t>(ns);
  L.ev0 = c.take<uint32_t>(ns); L.ev1 = c.take<uint32_t>(ns);
  L.perm = c.take<int32_t>(ns); L.rank = c.take<int32_t>(ns); L.degr = c.take<uint32_t>(ns);
  L.off = c.take<uint32_t>(ns + 1);
  // padded: a warp's round of up to 256 entries that starts below m may read
  // up to 255 entries past it (the entries there are masked, never counted)
  L.adj = c.take<uint32_t>(Es + 256);
  L.outdeg = c.take<uint32_t>(ns);
  L.wofs = c.take<uint32_t>(ns + 1);
  L.items = c.take<uint32_t>(ns);
  L.walk = c.take<uint64_t>(ns);
  L.bin_pivots = c.take<uint32_t>(ns);
  L.bin_flag = c.take<uint32_t>(ns);
  L.bin_pos = c.take<uint32_t>(ns + 1);
  L.hub_bitmap = c.take<uint32_t>((size_t)t.hub_bitmaps * (size_t)((ns + 31) / 32));
  L.hubinfo = c.take<uint32_t>(4 * (size_t)ns);
  L.tv = c.take<uint64_t>(ns);
  L.tcnt = nullptr;
  L.toff = nullptr;
  if (!(flags & AOT_FLAG_NO_LIST)) {
    L.tcnt = c.take<uint32_t>(Es);
    L.toff = c.take<uint64_t>(Es + 1);
  }
  L.route = c.take<uint8_t>(Es);
  L.rprobe = c.take<uint32_t>(ns);
  L.eplist = reinterpret_cast<uint2*>(L.flags);
  int64_t big = Es > ns ? Es : ns;  // the eta sort and the pivot scans run over n
  size_t tb = radix_tmp_bytes(big);
  size_t sb = scan_tmp_bytes(big + 1);
  L.tmp = c.take<char>(tb > sb ? tb : sb);
  L.bytes = c.used();
  return L;
}

}  // namespace aot

using namespace aot;

namespace aot {
constexpr uint32_t ORIENT_FLAGS = AOT_ETA_DEG_ASC | AOT_FLAG_NO_LIST | AOT_FLAG_NO_CLIP |
                                  AOT_FLAG_LOCAL_RANDOM | AOT_FLAG_TAIL_PIVOT | AOT_ETA_DEGENERACY;
static bool flags_valid(uint32_t flags) {
  if (flags & ~ORIENT_FLAGS) return false;
  if ((flags & AOT_ETA_DEG_ASC) && (flags & AOT_ETA_DEGENERACY)) return false;  // one global order
  return true;
}
static int item_rule(uint32_t flags) {
  if (flags & AOT_FLAG_TAIL_PIVOT) return RULE_TAIL;
  if (flags & (AOT_FLAG_NO_CLIP | AOT_FLAG_LOCAL_RANDOM)) return RULE_NOCLIP;
  return RULE_AOT;
}
// the fixed pseudo-random local order of AOT_FLAG_LOCAL_RANDOM on `bits`-bit ranks
static LocalOrder local_order(uint32_t flags, int bits) {
  LocalOrder o{0u, 0u, 1};
  if (!(flags & AOT_FLAG_LOCAL_RANDOM)) return o;
  const uint32_t mask = bits >= 32 ? 0xffffffffu : (uint32_t)((1ull << bits) - 1);
  o.mul = (0x9E3779B9u & mask) | 1u;  // odd: a bijection mod 2^bits
  uint32_t inv = o.mul;               // Newton's iteration for the inverse mod 2^32
  for (int i = 0; i < 5; ++i) inv *= 2u - o.mul * inv;
  o.inv = inv & mask;
  o.sh = bits / 2 > 0 ? bits / 2 : 1;
  return o;
}
// Peeling rounds of the degeneracy order into L.ek0 (the eta sort keys).
// Scratch: the symmetric adjacency in the dead cleanup keys (2m words of the
// 8E bytes), its offsets in L.off and cursors in L.wofs, current degrees in
// L.bin_flag, two frontiers in L.hubinfo, counters in the device scalars;
// the later steps overwrite all of them.
static aot_status degeneracy_rounds(aot_graph* g, const OrientLayout& L, const uint64_t* ukeys,
                                    uint64_t* dead_keys, int64_t m, cudaStream_t s) {
  const int T = 256;
  const int32_t n = g->n;
  uint32_t* soff = L.off;
  uint32_t* cursor = L.wofs;
  uint32_t* sadj = reinterpret_cast<uint32_t*>(dead_keys);
  uint32_t* cur = L.bin_flag;
  uint32_t* rnd = L.ek0;
  uint32_t* fa = L.hubinfo;
  uint32_t* fb = L.hubinfo + n;
  unsigned int* cnt = &g->dev->counters[10];
  unsigned int* kmin = &g->dev->counters[11];
  AOT_TRY(scan_u32_u32(L.deg, soff, n, L.tmp, s));
  if (m > 0) {
    AOT_CUDA(cudaMemcpyAsync(cursor, soff, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    AOT_KERNEL("k_sym_fill", s)
      k_sym_fill<<<grid_for(m, T), T, 0, s>>>(ukeys, m, g->bits, cursor, sadj);
    AOT_TRY(last_launch());
  }
  AOT_CUDA(cudaMemcpyAsync(cur, L.deg, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
  AOT_CUDA(cudaMemsetAsync(rnd, 0xff, sizeof(uint32_t) * n, s));
  const int sms = sm_count();
  uint32_t k = 0, r = 0;
  int64_t remaining = n;
  while (remaining > 0) {
    unsigned int nf = 0;
    AOT_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned int), s));
    AOT_KERNEL("k_peel_scan", s)
      k_peel_scan<<<grid_for(n, T), T, 0, s>>>(cur, rnd, n, k, fa, cnt);
    AOT_TRY(last_launch());
    AOT_CUDA(cudaMemcpyAsync(&nf, cnt, sizeof(nf), cudaMemcpyDeviceToHost, s));
    AOT_CUDA(cudaStreamSynchronize(s));
    if (nf == 0) {  // next level: the smallest remaining degree
      unsigned int km = UNSET;
      AOT_CUDA(cudaMemsetAsync(kmin, 0xff, sizeof(unsigned int), s));
      AOT_KERNEL("k_peel_min", s)
        k_peel_min<<<grid_for(n, T), T, 0, s>>>(cur, rnd, n, kmin);
      AOT_TRY(last_launch());
      AOT_CUDA(cudaMemcpyAsync(&km, kmin, sizeof(km), cudaMemcpyDeviceToHost, s));
      AOT_CUDA(cudaStreamSynchronize(s));
      if (km == UNSET || km <= k) return AOT_ERR_DEVICE_CHECK;  // cannot happen: remaining > 0
      k = km;
      continue;
    }
    while (nf > 0) {
      unsigned int nn = 0;
      AOT_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned int), s));
      int64_t grid = ((int64_t)nf * 32 + T - 1) / T;
      if (grid > (int64_t)sms * 16) grid = (int64_t)sms * 16;
      AOT_KERNEL("k_peel_round", s)
        k_peel_round<<<(unsigned)grid, T, 0, s>>>(fa, nf, r, k, soff, sadj, cur, rnd, fb, cnt);
      AOT_TRY(last_launch());
      AOT_CUDA(cudaMemcpyAsync(&nn, cnt, sizeof(nn), cudaMemcpyDeviceToHost, s));
      AOT_CUDA(cudaStreamSynchronize(s));
      remaining -= nf;
      ++r;
      uint32_t* t = fa;
      fa = fb;
      fb = t;
      nf = nn;
    }
  }
  return AOT_OK;
}

}  // namespace aot

extern "C" aot_status aot_orient_workspace_size(int64_t num_edges, int32_t num_vertices,
                                                uint32_t flags, size_t* bytes) {
  if (!bytes || num_edges < 0 || num_vertices < 0) return AOT_ERR_INVALID_ARG;
  if (!flags_valid(flags)) return AOT_ERR_INVALID_ARG;
  if (num_edges >= (int64_t(1) << 40)) return AOT_ERR_OVERFLOW;
  Tuning t;
  *bytes = carve_orient(nullptr, num_edges, num_vertices, flags, t).bytes;
  return AOT_OK;
}

extern "C" aot_status aot_orient(const int32_t* d_src, const int32_t* d_dst, int64_t num_edges,
                                 int32_t num_vertices, uint32_t flags, void* d_workspace,
                                 size_t ws_bytes, aot_stream_t stream, aot_graph** out) {
  if (!out) return AOT_ERR_INVALID_ARG;
  *out = nullptr;
  if (num_edges < 0 || num_vertices < 0) return AOT_ERR_INVALID_ARG;
  if (num_edges > 0 && (!d_src || !d_dst)) return AOT_ERR_INVALID_ARG;
  if (!flags_valid(flags)) return AOT_ERR_INVALID_ARG;
  if (num_edges >= (int64_t(1) << 40)) return AOT_ERR_OVERFLOW;
  if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255)) return AOT_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Tuning tune = default_tuning();
  OrientLayout L = carve_orient(d_workspace, num_edges, num_vertices, flags, Tuning());
  if (ws_bytes < L.bytes) return AOT_ERR_WORKSPACE;
  if (num_edges > 0 && num_vertices == 0) return AOT_ERR_VERTEX_RANGE;

  aot_graph* g = new aot_graph();
  g->tune = tune;
  g->model = default_router();
  g->n = num_vertices;
  g->num_edges = num_edges;
  g->flags = flags;
  g->bits = num_vertices > 1 ? ceil_log2((uint64_t)num_vertices) : 1;
  g->dev = L.dev;
  g->perm = L.perm; g->rank = L.rank; g->degr = L.degr; g->off = L.off; g->outdeg = L.outdeg;
  g->wofs = L.wofs; g->items = L.items; g->walk = L.walk;
  g->bin_pivots = L.bin_pivots; g->bin_flag = L.bin_flag; g->bin_pos = L.bin_pos;
  g->hub_bitmap = L.hub_bitmap; g->hubinfo = L.hubinfo; g->tv = L.tv;
  g->tcnt = L.tcnt; g->toff = L.toff; g->has_list = !(flags & AOT_FLAG_NO_LIST);
  g->scan_tmp = L.tmp;
  g->route = L.route; g->rprobe = L.rprobe; g->eplist = L.eplist;
  g->adj = L.adj;
  auto fail = [&](aot_status st) { delete g; return st; };

  const int T = 256;
  const int32_t n = num_vertices;
  const int64_t E = num_edges;
  const int bits = g->bits;
  if (cudaMemsetAsync(L.dev, 0, sizeof(DevScalars), s) != cudaSuccess) return fail(AOT_ERR_CUDA);
  if (n > 0) {
    if (cudaMemsetAsync(L.deg, 0, sizeof(uint32_t) * n, s) != cudaSuccess ||
        cudaMemsetAsync(L.outdeg, 0, sizeof(uint32_t) * n, s) != cudaSuccess ||
        cudaMemsetAsync(L.items, 0, sizeof(uint32_t) * n, s) != cudaSuccess)
      return fail(AOT_ERR_CUDA);
  }
  // 1. cleanup: keys, sort, unique
  int64_t m = 0;
  uint64_t* sorted = L.keysA;
  uint64_t* other = L.keysB;
  if (E > 0) {
    AOT_KERNEL("k_make_keys", s)
      k_make_keys<<<grid_for(E, T), T, 0, s>>>(d_src, d_dst, E, n, bits, L.keysA, L.dev);
    if (last_launch()) return fail(AOT_ERR_CUDA);
    aot_status st = radix_sort_u64(L.keysA, L.keysB, E, 2 * bits, L.tmp, &L.dev->err, s, &sorted);
    if (st) return fail(st);
    other = sorted == L.keysA ? L.keysB : L.keysA;
    AOT_KERNEL("k_unique_flags", s)
      k_unique_flags<<<grid_for(E, T), T, 0, s>>>(sorted, E, L.flags);
    if (last_launch()) return fail(AOT_ERR_CUDA);
    st = scan_u32_u32(L.flags, L.pos, E, L.tmp, s);
    if (st) return fail(st);
    uint32_t mm = 0;
    if (cudaMemcpyAsync(&mm, L.pos + E, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
      return fail(AOT_ERR_CUDA);
    st = read_device_error(g, s);
    if (st) return fail(st);
    m = mm;
    AOT_KERNEL("k_compact_unique", s)
      k_compact_unique<<<grid_for(E, T), T, 0, s>>>(sorted, L.flags, L.pos, E, bits, other, L.deg);
    if (last_launch()) return fail(AOT_ERR_CUDA);
  }
  g->m = m;
  // 2. eta: stable sort of ids by degree key (or by peeling round)
  if (n > 0 && (flags & AOT_ETA_DEGENERACY)) {
    aot_status st = degeneracy_rounds(g, L, other, sorted, m, s);
    if (st) return fail(st);
    AOT_KERNEL("k_iota", s)
      k_iota<<<grid_for(n, T), T, 0, s>>>(L.ev0, n);
    if (last_launch()) return fail(AOT_ERR_CUDA);
  } else if (n > 0) {
    AOT_KERNEL("k_eta_keys", s)
      k_eta_keys<<<grid_for(n, T), T, 0, s>>>(L.deg, n, bits, !(flags & AOT_ETA_DEG_ASC), L.ek0,
                                            L.ev0);
    if (last_launch()) return fail(AOT_ERR_CUDA);
  }
  if (n > 0) {
    uint32_t *ko, *vo;
    aot_status st = radix_sort_u32_pairs(L.ek0, L.ek1, L.ev0, L.ev1, n, bits, L.tmp, &L.dev->err, s, &ko, &vo);
    if (st) return fail(st);
    AOT_KERNEL("k_rank_from_perm", s)
      k_rank_from_perm<<<grid_for(n, T), T, 0, s>>>(vo, n, L.deg, L.perm, L.rank, L.degr);
    if (last_launch()) return fail(AOT_ERR_CUDA);
  }
  // 3. orient: relabel, sort, split into out-CSR
  uint32_t* esrc = L.flags;  // the cleanup flags are dead now
  if (m > 0) {
    uint64_t* ukeys = other;
    uint64_t* okeys = sorted;  // reuse the other buffer
    AOT_KERNEL("k_relabel", s)
      k_relabel<<<grid_for(m, T), T, 0, s>>>(ukeys, m, bits, L.rank, local_order(flags, bits), okeys);
    if (last_launch()) return fail(AOT_ERR_CUDA);
    uint64_t* osorted;
    aot_status st = radix_sort_u64(okeys, ukeys, m, 2 * bits, L.tmp, &L.dev->err, s, &osorted);
    if (st) return fail(st);
    AOT_KERNEL("k_split_csr", s)
      k_split_csr<<<grid_for(m, T), T, 0, s>>>(osorted, m, bits, local_order(flags, bits), L.adj, esrc,
                                             L.outdeg);
    if (last_launch()) return fail(AOT_ERR_CUDA);
  }
  if (n > 0) {
    aot_status st = scan_u32_u32(L.outdeg, L.off, n, L.tmp, s);
    if (st) return fail(st);
    AOT_KERNEL("k_max_outdeg", s)
      k_max_outdeg<<<grid_for(n, T), T, 0, s>>>(L.outdeg, n, L.dev);
    if (last_launch()) return fail(AOT_ERR_CUDA);
  } else {
    if (cudaMemsetAsync(L.off, 0, sizeof(uint32_t), s)) return fail(AOT_ERR_CUDA);
  }
  // 4. work items (they overwrite the dead key buffers)
  g->witem = reinterpret_cast<uint2*>(L.keysA);
  g->wvert = reinterpret_cast<uint32_t*>(L.keysB);
  g->wedge = reinterpret_cast<uint32_t*>(L.keysB) + (E > 0 ? E : 1);
  // positive flags, then (in place) their exclusive scan: L.pos holds E + 1 >= m + 1 words
  uint32_t* pscan = L.pos;
  if (m > 0) {
    AOT_KERNEL("k_item_count", s)
      k_item_count<<<grid_for(m, T), T, 0, s>>>(esrc, L.adj, L.off, L.outdeg, m, item_rule(flags),
                                              L.items, pscan);
    if (last_launch()) return fail(AOT_ERR_CUDA);
    aot_status st = scan_u32_u32(pscan, pscan, m, L.tmp, s);
    if (st) return fail(st);
  }
  if (n > 0) {
    aot_status st = scan_u32_u32(L.items, L.wofs, n, L.tmp, s);
    if (st) return fail(st);
    if (cudaMemsetAsync(L.bin_flag, 0, sizeof(uint32_t) * n, s)) return fail(AOT_ERR_CUDA);
  } else {
    if (cudaMemsetAsync(L.wofs, 0, sizeof(uint32_t), s)) return fail(AOT_ERR_CUDA);
  }
  if (m > 0) {
    AOT_KERNEL("k_item_fill", s)
      k_item_fill<<<grid_for(m, T), T, 0, s>>>(esrc, L.adj, L.off, L.outdeg, m, item_rule(flags), L.wofs,
                                             pscan, L.bin_flag, g->witem, g->wvert, g->wedge);
    if (last_launch()) return fail(AOT_ERR_CUDA);
  }
  if (n > 0) {  // large-pivot list in bin_pos (n + 1 words, free until binning)
    AOT_KERNEL("k_pivot_walk", s)
      k_pivot_walk<<<grid_for(n, T), T, 0, s>>>(L.wofs, g->witem, L.outdeg, n, L.walk, L.bin_pos, L.dev);
    if (last_launch()) return fail(AOT_ERR_CUDA);
    AOT_KERNEL("k_pivot_walk_big", s)
      k_pivot_walk_big<<<(unsigned)(sm_count() * 8), T, 0, s>>>(L.wofs, g->witem, L.bin_pos, L.walk, L.dev);
    if (last_launch()) return fail(AOT_ERR_CUDA);
  }
  DevScalars hs;
  uint32_t npos = 0;  // the positive-flag scan's total
  if (cudaMemcpyAsync(&hs, L.dev, sizeof(DevScalars), cudaMemcpyDeviceToHost, s) ||
      (m > 0 && cudaMemcpyAsync(&npos, pscan + m, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) ||
      cudaStreamSynchronize(s))
    return fail(AOT_ERR_CUDA);
  g->positive = npos;
  if (hs.err) return fail(hs.err & DEVERR_RANGE ? AOT_ERR_VERTEX_RANGE : AOT_ERR_DEVICE_CHECK);
  g->W = hs.total;
  g->S = hs.aux[0];
  g->merge_work = hs.total + hs.aux[1];
  g->max_outdeg = (int32_t)hs.counters[0];
  // 5. bins
  aot_status st = bin_pivots(g, s);
  if (st) return fail(st);
  *out = g;
  return AOT_OK;
}
