// aot_count.cu - the walk-and-probe core of Algorithm 3 on the GPU.
//
// Every pivot p builds its index H over N+(p) once (Algorithm 3, index set-up
// per pivot; Sec. 3.2 stresses that each vertex builds H exactly once) and
// then walks its work items: for a positive item v the whole N+(v), for a
// negative item x the part of N+(x) after p; every walked w found in H closes
// the triangle (p,v,w) or (x,p,w) (Algorithm 3, output steps).
//
// GB300 mapping: pivots are binned by deg+(p).
//   BIN_WARP  deg+ <= warp_max: one warp per pivot, H = open-addressing hash
//             table in the warp's slice of shared memory
//   BIN_CTA   deg+ <= cta_max: one CTA per pivot, H in shared memory, the
//             CTA's warps split the pivot's items
//   BIN_HUB   larger: H = a global bitmap of n bits (L2 resident), several
//             hubs at a time, all CTAs split the hubs' items
// Inside a warp the items of a chunk (32 items) are flattened: lanes walk
// consecutive positions of the concatenated walk ranges (coalesced loads),
// find their item by a 5-step shuffle search over the exclusive prefix of
// walk lengths, probe H, and count with __ballot_sync/__popc.
// Work is handed out by per-bin atomic queues (persistent grids).
#include <vector>

#include "aot_internal.cuh"
#include "aot_kparams.cuh"

namespace aot {

constexpr int MAX_HUBS = 64;
struct HubGroup {
  int count;
  uint32_t words;                 // bitmap words per hub
  uint32_t* bitmap;
  uint32_t pivot[MAX_HUBS];
  uint32_t ib[MAX_HUBS];          // first item
  uint32_t ie[MAX_HUBS];          // end item
  uint32_t cbeg[MAX_HUBS + 1];    // prefix of 32-item chunks
};

__device__ __forceinline__ unsigned range_mask(int lo, int hi) {  // bits [lo, hi)
  unsigned a = lo >= 32 ? 0u : (lo <= 0 ? ~0u : (~0u << lo));
  unsigned b = hi >= 32 ? ~0u : (hi <= 0 ? 0u : ((1u << hi) - 1u));
  return a & b;
}

__device__ __forceinline__ int clamp_lane(int64_t x) {
  return x < -1 ? -1 : (x > 64 ? 64 : (int)x);
}

constexpr uint32_t LONG_ITEM = 64;  // items at least this long are walked by the whole warp

// One warp walks items [c, min(c+32, ie)) of pivot p.  probe(w, slot) tests
// H; on_w(w, slot) is called by every hitting lane (per-vertex counts of w).
// Long items are walked one at a time by all 32 lanes, four loads in flight
// per lane; the short ones are flattened: lanes take consecutive positions
// of their concatenated walk ranges and find their item by a shuffle search
// over the exclusive prefix of the lengths.  Returns this lane's hit count.
template <int MODE, class Probe, class OnW>
__device__ __forceinline__ uint32_t walk_chunk(const KParams& P, uint32_t p, uint32_t c,
                                               uint32_t ie, Probe probe, OnW on_w,
                                               uint32_t stage_share = 0) {
  const unsigned lane = lane_id();
  const uint32_t it = c + lane;
  const bool has = it < ie && (!P.route || P.route[it] == V_PROBE);
  uint2 r = has ? P.witem[it] : make_uint2(0u, 0u);
  uint32_t vert = 0, edge = 0;
  uint64_t tbase = 0;
  if (MODE != M_COUNT && has) vert = P.wvert[it];
  if (MODE >= M_LIST_COUNT && has) edge = P.wedge[it];
  uint2 ends = make_uint2(0u, 0u);  // listing: this lane's item's first two ids
  if (MODE == M_LIST_WRITE && has) {
    uint64_t a = P.toff[edge], b = P.toff[edge + 1];
    if (a == b || b <= P.cursor || a >= P.cursor + P.cap) r.y = r.x;  // nothing in the window
    tbase = a;
    if (r.x < r.y) ends = emit_ends(P, p, vert);
  }
  uint32_t len = r.y - r.x;
  uint32_t ihits = 0;  // hits of the item held by this lane
  uint32_t my = 0;     // hits found by this lane
  uint32_t mycyc = 0;  // M_TIMED: cycles of the item held by this lane

  // ---- long items: the whole warp, 4 x 32 entries per step
  unsigned longm = __ballot_sync(FULL, len >= LONG_ITEM);
  while (longm) {
    const int j = __ffs(longm) - 1;
    longm &= longm - 1;
    const long long t0 = MODE == M_TIMED ? clock64() : 0;
    const uint32_t x = __shfl_sync(FULL, r.x, j), y = __shfl_sync(FULL, r.y, j);
    uint2 ej = make_uint2(0u, 0u);
    uint64_t tb = 0;
    if (MODE == M_LIST_WRITE) {
      ej = make_uint2(__shfl_sync(FULL, ends.x, j), __shfl_sync(FULL, ends.y, j));
      tb = ((uint64_t)__shfl_sync(FULL, (uint32_t)(tbase >> 32), j) << 32) |
           __shfl_sync(FULL, (uint32_t)tbase, j);
    }
    uint32_t h = 0;  // hits of item j so far (warp-uniform)
    for (uint32_t k = x; k < y; k += 128) {
      uint32_t w[4], slot[4];
      bool hit[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t idx = k + u * 32 + lane;
        w[u] = idx < y ? __ldg(P.adj + idx) : EMPTY;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) hit[u] = w[u] != EMPTY && probe(w[u], slot[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned hm = __ballot_sync(FULL, hit[u]);
        if (hit[u]) {
          ++my;
          if (MODE == M_VERTEX) on_w(w[u], slot[u]);
          if (MODE == M_LIST_WRITE) emit(P, tb + h + (uint32_t)__popc(hm & lanemask_lt()), ej, w[u]);
        }
        h += (uint32_t)__popc(hm);
      }
    }
    if ((int)lane == j) {
      ihits = h;
      if (MODE == M_TIMED) mycyc = sat_cycles(clock64() - t0);
    }
  }
  if (len >= LONG_ITEM) len = 0;

  // ---- short items: flattened
  const long long ts0 = MODE == M_TIMED ? clock64() : 0;
  const uint32_t incl = warp_inclusive_scan(len);
  const uint32_t total = __shfl_sync(FULL, incl, 31);
  const uint32_t excl = incl - len;
  for (uint32_t q0 = 0; q0 < total; q0 += 32) {
    const uint32_t q = q0 + lane;
    const bool act = q < total;
    int j = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
      uint32_t e = __shfl_sync(FULL, excl, j + step);
      if (e <= q) j += step;
    }
    const uint32_t jx = __shfl_sync(FULL, r.x, j);
    const uint32_t je = __shfl_sync(FULL, excl, j);
    uint32_t w = 0, slot = 0;
    bool hit = false;
    if (act) {
      w = __ldg(P.adj + jx + (q - je));
      hit = probe(w, slot);
    }
    const unsigned hm = __ballot_sync(FULL, hit);
    if (MODE == M_LIST_WRITE) {
      const uint32_t prev = __shfl_sync(FULL, ihits, j);
      const unsigned peers = __match_any_sync(FULL, j);
      const uint32_t tb_lo = __shfl_sync(FULL, (uint32_t)tbase, j);
      const uint32_t tb_hi = __shfl_sync(FULL, (uint32_t)(tbase >> 32), j);
      const uint2 ej = make_uint2(__shfl_sync(FULL, ends.x, j), __shfl_sync(FULL, ends.y, j));
      if (hit)
        emit(P, (((uint64_t)tb_hi << 32) | tb_lo) + prev + (uint32_t)__popc(hm & peers & lanemask_lt()),
             ej, w);
    }
    if (MODE != M_COUNT) {
      const int64_t lo = (int64_t)excl - (int64_t)q0, hi = (int64_t)incl - (int64_t)q0;
      ihits += (uint32_t)__popc(hm & range_mask(clamp_lane(lo), clamp_lane(hi)));
    }
    if (hit) {
      ++my;
      if (MODE == M_VERTEX) on_w(w, slot);
    }
  }
  if (MODE == M_VERTEX && has && ihits) atomicAdd((unsigned long long*)&P.tv[vert], (unsigned long long)ihits);
  if (MODE == M_LIST_COUNT && has) P.tcnt[edge] = ihits;
  if (MODE == M_TIMED) {
    // a short item gets the flattened phase's time in proportion to its length
    const long long tshort = clock64() - ts0;
    if (has && len > 0 && total > 0) mycyc = sat_cycles((long long)((double)tshort * len / total));
    if (has) P.cyc[edge] = mycyc + stage_share;
  }
  return my;
}

// ------------------------------------------------------------ warp kernel
constexpr int WARP_TS = 128;  // slots per warp table of the warp bin (deg+ <= 64)

// A warp per pivot, its hash table (ts_max slots, plus as many hit counters
// in per-vertex mode) in the warp's share of dynamic shared memory; pivots
// come from queue q.  Used
// for the warp bin and, with cta_threads = 32, for the CTA bin: no CTA-wide
// barrier, so a pivot with long items holds up only its own warp.
// words of a warp's shared memory: table, hit counters (per-vertex mode) and
// the prefilter of 8 ts_max bits
template <int MODE>
__host__ __device__ constexpr size_t warp_pivot_words(uint32_t ts_max) {
  return (size_t)(MODE == M_VERTEX ? 2 : 1) * ts_max + ts_max / 4;
}

// prefilter bit of w among 2^fbits: the high bits of a second multiplicative
// hash (independent of the table slot, which takes the low bits)
__device__ __forceinline__ uint32_t filter_bit(uint32_t w, int fbits) {
  return (w * 0x85EBCA6Bu) >> (32 - fbits);
}

template <int MODE>
__global__ void __launch_bounds__(256) k_warp_pivots(KParams P, uint32_t ts_max, int q) {
  extern __shared__ uint32_t wp_sm[];
  const unsigned lane = lane_id(), wid = threadIdx.x >> 5;
  uint32_t* tab = wp_sm + (size_t)wid * warp_pivot_words<MODE>(ts_max);
  uint32_t* cnt = tab + ts_max;  // per-vertex mode only
  // prefilter: 8 ts bits, one set for every entry of N+(p);
  // a probe whose bit is clear misses without touching the table
  uint32_t* filt = tab + (MODE == M_VERTEX ? 2 : 1) * ts_max;
  uint64_t found = 0;
  while (true) {
    uint32_t idx = 0;
    if (lane == 0) idx = atomicAdd(&P.dev->counters[q], 1u);
    idx = __shfl_sync(FULL, idx, 0);
    if (idx >= P.num_pivots) break;
    const uint32_t p = P.pivots[idx];
    if (P.rprobe && P.rprobe[p] == 0) continue;  // every item of p takes another route
    if (MODE == M_LIST_WRITE && !list_window_overlaps(P, P.wofs[p], P.wofs[p + 1])) continue;
    const uint32_t b = P.off[p], d = P.off[p + 1] - b;
    const long long tst0 = MODE == M_TIMED ? clock64() : 0;
    uint32_t ts = 32;
    int fbits = 8;  // log2 of the prefilter bits, 8 ts
    while (ts < 2 * d) {
      ts <<= 1;
      ++fbits;
    }
    const uint32_t mask = ts - 1;
    for (uint32_t i = lane; i < ts; i += 32) {
      tab[i] = EMPTY;
      if (MODE == M_VERTEX) cnt[i] = 0;
    }
    for (uint32_t i = lane; i < ts / 4; i += 32) filt[i] = 0;
    __syncwarp();
    for (uint32_t i = lane; i < d; i += 32) {
      uint32_t w = P.adj[b + i], s = hash_slot(w, mask);
      while (atomicCAS(&tab[s], EMPTY, w) != EMPTY) s = (s + 1) & mask;
      const uint32_t f = filter_bit(w, fbits);
      atomicOr(&filt[f >> 5], 1u << (f & 31));
    }
    __syncwarp();
    const uint32_t stage_share = MODE == M_TIMED
        ? sat_cycles((clock64() - tst0) / (long long)max(1u, P.wofs[p + 1] - P.wofs[p])) : 0u;
    auto probe = [&](uint32_t w, uint32_t& slot) -> bool {
      const uint32_t f = filter_bit(w, fbits);
      if (!((filt[f >> 5] >> (f & 31)) & 1u)) return false;
      uint32_t s = hash_slot(w, mask);
      while (true) {
        uint32_t k = tab[s];
        if (k == w) { slot = s; return true; }
        if (k == EMPTY) return false;
        s = (s + 1) & mask;
      }
    };
    auto on_w = [&](uint32_t, uint32_t slot) { atomicAdd(&cnt[slot], 1u); };
    const uint32_t ib = P.wofs[p], ie = P.wofs[p + 1];
    uint32_t ph = 0;
    for (uint32_t c = ib; c < ie; c += 32) ph += walk_chunk<MODE>(P, p, c, ie, probe, on_w, stage_share);
    if (MODE == M_VERTEX) {
      __syncwarp();
      for (uint32_t i = lane; i < ts; i += 32)
        if (cnt[i]) atomicAdd((unsigned long long*)&P.tv[tab[i]], (unsigned long long)cnt[i]);
      uint32_t tot = warp_sum(ph);
      if (lane == 0 && tot) atomicAdd((unsigned long long*)&P.tv[p], (unsigned long long)tot);
    }
    found += ph;
    __syncwarp();
  }
  found = warp_sum(found);
  if (lane == 0 && found) atomicAdd(&P.dev->total, (unsigned long long)found);
}

// ------------------------------------------------------------- CTA kernel
template <int MODE>
__global__ void __launch_bounds__(1024, 1) k_cta_pivots(KParams P, uint32_t ts_max) {
  extern __shared__ uint32_t cta_sm[];
  uint32_t* tab = cta_sm;
  uint32_t* cnt = cta_sm + ts_max;
  __shared__ uint32_t s_idx;
  __shared__ unsigned long long s_hits;
  const unsigned lane = lane_id(), wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint64_t found = 0;
  while (true) {
    if (threadIdx.x == 0) {
      s_idx = atomicAdd(&P.dev->counters[Q_CTA], 1u);
      s_hits = 0;
    }
    __syncthreads();
    const uint32_t idx = s_idx;
    if (idx >= P.num_pivots) break;
    const uint32_t p = P.pivots[idx];
    if ((P.rprobe && P.rprobe[p] == 0) ||  // every item of p takes another route
        (MODE == M_LIST_WRITE && !list_window_overlaps(P, P.wofs[p], P.wofs[p + 1]))) {
      __syncthreads();
      continue;
    }
    const uint32_t b = P.off[p], d = P.off[p + 1] - b;
    const long long tst0 = MODE == M_TIMED ? clock64() : 0;
    uint32_t ts = 64;
    while (ts < 2 * d) ts <<= 1;
    const uint32_t mask = ts - 1;
    for (uint32_t i = threadIdx.x; i < ts; i += blockDim.x) {
      tab[i] = EMPTY;
      if (MODE == M_VERTEX) cnt[i] = 0;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) {
      uint32_t w = P.adj[b + i], s = hash_slot(w, mask);
      while (atomicCAS(&tab[s], EMPTY, w) != EMPTY) s = (s + 1) & mask;
    }
    __syncthreads();
    // the block's staging time, spread over the pivot's items (all warps waited for it)
    const uint32_t stage_share = MODE == M_TIMED
        ? sat_cycles((clock64() - tst0) * (long long)nw / (long long)max(1u, P.wofs[p + 1] - P.wofs[p])) : 0u;
    auto probe = [&](uint32_t w, uint32_t& slot) -> bool {
      uint32_t s = hash_slot(w, mask);
      while (true) {
        uint32_t k = tab[s];
        if (k == w) { slot = s; return true; }
        if (k == EMPTY) return false;
        s = (s + 1) & mask;
      }
    };
    auto on_w = [&](uint32_t, uint32_t slot) { atomicAdd(&cnt[slot], 1u); };
    const uint32_t ib = P.wofs[p], ie = P.wofs[p + 1];
    uint32_t ph = 0;
    for (uint32_t c = ib + 32 * wid; c < ie; c += 32 * nw) ph += walk_chunk<MODE>(P, p, c, ie, probe, on_w, stage_share);
    found += ph;
    if (MODE == M_VERTEX) {
      uint32_t tot = warp_sum(ph);
      if (lane == 0 && tot) atomicAdd(&s_hits, (unsigned long long)tot);
    }
    __syncthreads();
    if (MODE == M_VERTEX) {
      for (uint32_t i = threadIdx.x; i < ts; i += blockDim.x)
        if (cnt[i]) atomicAdd((unsigned long long*)&P.tv[tab[i]], (unsigned long long)cnt[i]);
      if (threadIdx.x == 0 && s_hits) atomicAdd((unsigned long long*)&P.tv[p], s_hits);
    }
    __syncthreads();
  }
  found = warp_sum(found);
  if (lane == 0 && found) atomicAdd(&P.dev->total, (unsigned long long)found);
}

// ------------------------------------------------------------- hub kernels
__global__ void k_hub_bits(HubGroup G, const uint32_t* __restrict__ off,
                           const uint32_t* __restrict__ adj, bool set) {
  const int b = blockIdx.y;
  const uint32_t p = G.pivot[b];
  const uint32_t beg = off[p], end = off[p + 1];
  uint32_t* bm = G.bitmap + (size_t)b * G.words;
  for (uint32_t i = beg + blockIdx.x * blockDim.x + threadIdx.x; i < end; i += gridDim.x * blockDim.x) {
    uint32_t w = adj[i];
    if (set) atomicOr(&bm[w >> 5], 1u << (w & 31));
    else bm[w >> 5] = 0u;
  }
}

template <int MODE>
__global__ void __launch_bounds__(256) k_hub_walk(KParams P, HubGroup G) {
  const unsigned lane = lane_id();
  const uint32_t nchunks = G.cbeg[G.count];
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  uint64_t found = 0;
  for (uint32_t ch = gw; ch < nchunks; ch += nwarps) {
    int b = 0;
    while (b + 1 < G.count && G.cbeg[b + 1] <= ch) ++b;
    const uint32_t p = G.pivot[b];
    const uint32_t* bm = G.bitmap + (size_t)b * G.words;
    const uint32_t c = G.ib[b] + 32 * (ch - G.cbeg[b]);
    auto probe = [&](uint32_t w, uint32_t&) -> bool { return (__ldcg(bm + (w >> 5)) >> (w & 31)) & 1u; };
    auto on_w = [&](uint32_t w, uint32_t) { atomicAdd((unsigned long long*)&P.tv[w], 1ull); };
    uint32_t ph = walk_chunk<MODE>(P, p, c, G.ie[b], probe, on_w);
    found += ph;
    if (MODE == M_VERTEX) {
      uint32_t tot = warp_sum(ph);
      if (lane == 0 && tot) atomicAdd((unsigned long long*)&P.tv[p], (unsigned long long)tot);
    }
  }
  found = warp_sum(found);
  if (lane == 0 && found) atomicAdd(&P.dev->total, (unsigned long long)found);
}

// ------------------------------------------------ segmented bitmap kernel
// Pivots with a large deg+ (beyond the shared-memory hash tables): H is a
// bitmap over eta ranks, held in shared memory one segment of SEG_BITS ranks
// at a time.  A CTA owns (pivot, block of up to SEG_ITEMS items) and sweeps
// the pivot's rank range [min N+(p), max N+(p)] segment by segment: it sets
// the bits of N+(p) in the segment, every warp advances its items' cursors
// through the entries below the segment end (out-lists are sorted by eta, so
// each walked entry is visited exactly once over all segments), then clears
// the bits.  Items keep cursor, end, next walked value and hit count in
// shared memory, so one item's hits come out in ascending w order (the
// listing order).  Items shorter than seg_long entries are walked by one
// thread each, longer ones by a warp in rounds of 128 entries (256 while at
// least seg_wide entries remain).  Each pivot's segment bounds (positions in
// N+(p)) are precomputed once per call by k_seg_bounds.
constexpr int SEG_THREADS = 1024;
constexpr uint32_t SEG_ITEMS = 1536;

constexpr uint32_t SEG_BITS_MAX = 1536u * 1024u;  // 192 KB of bitmap at most
constexpr uint32_t NONE = 0xffffffffu;
// bitmap + a zero guard word (answers every probe past the bitmap) and three
// pad words + per item: cursor, end, next walked value, hits; list of long
// items; long flags
constexpr size_t seg_smem_bytes(uint32_t seg_bits) {
  return (size_t)(seg_bits / 32 + 4) * 4 + 5 * (size_t)SEG_ITEMS * 4 + SEG_ITEMS;
}

// first index in [lo, hi) with a[idx] >= key (a sorted); all 32 lanes call it
__device__ __forceinline__ uint32_t warp_lower_bound(const uint32_t* __restrict__ a, uint32_t lo,
                                                     uint32_t hi, uint32_t key) {
  const unsigned lane = lane_id();
  while (hi - lo > 32) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t idx = lo + lane * step;
    const bool less = idx < hi && a[idx] < key;
    const int c = __popc(__ballot_sync(FULL, less));
    if (c == 0) return lo;
    const uint32_t nlo = lo + (uint32_t)(c - 1) * step + 1;
    const uint32_t nhi = min(hi, lo + (uint32_t)c * step);
    lo = nlo;
    hi = nhi;
  }
  const uint32_t idx = lo + lane;
  const bool less = idx < hi && a[idx] < key;
  return lo + (uint32_t)__popc(__ballot_sync(FULL, less));
}

// first index in [lo, hi) where less(idx) is false (less holds on a prefix);
// all 32 lanes call it
template <class Less>
__device__ __forceinline__ uint32_t warp_partition(uint32_t lo, uint32_t hi, Less less) {
  const unsigned lane = lane_id();
  while (hi - lo > 32) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t idx = lo + lane * step;
    const bool l = idx < hi && less(idx);
    const int c = __popc(__ballot_sync(FULL, l));
    if (c == 0) return lo;
    const uint32_t nlo = lo + (uint32_t)(c - 1) * step + 1;
    const uint32_t nhi = min(hi, lo + (uint32_t)c * step);
    lo = nlo;
    hi = nhi;
  }
  const uint32_t idx = lo + lane;
  const bool l = idx < hi && less(idx);
  return lo + (uint32_t)__popc(__ballot_sync(FULL, l));
}

constexpr uint32_t SEG_MAXB = 512;  // segment bounds of one pivot held in shared memory

// Work groups of the hub pivots, a warp per pivot.  A pivot's positive items
// come first, sorted by their walked vertex v (larger rank than the pivot),
// then its negative items (walked vertex of smaller rank).  With G >= 2
// groups, groups 0 .. G-2 hold the positive items by the tile of v's
// out-list, tile(v) = off[v] >> tile_bits (the out-lists of one tile fill
// 2^tile_bits consecutive adjacency entries; the last tile group also takes
// every later tile), and group G-1 the negative items; G = 1 is one group of
// all items.  Group g of hub h spans items [bound(g), bound(g+1)) with
// bound(0) = wofs[p], bound(G) = wofs[p+1] and the inner bounds in
// ist[(g-1) nh + h]; it takes ceil(size / SEG_ITEMS) tasks (tcnt[g nh + h]).
// Groups are laid out tile-major, so the task queue hands out every pivot's
// items of tile 0 first, then tile 1, ...: blocks that run at the same time
// walk the same out-lists, which stay in L2.
// Also: nbound[h] = segments + 1 of the pivot's rank range [min N+(p),
// max N+(p)] in segments of seg_bits.
__device__ __forceinline__ uint32_t group_bound(const uint32_t* ist, const uint32_t* wofs, uint32_t p,
                                                uint32_t h, uint32_t nh, uint32_t G, uint32_t g) {
  return g == 0 ? wofs[p] : (g == G ? wofs[p + 1] : ist[(size_t)(g - 1) * nh + h]);
}

__global__ void k_seg_groups(const uint32_t* __restrict__ pivots, uint32_t nh,
                             const uint32_t* __restrict__ wofs, const uint32_t* __restrict__ wvert,
                             const uint32_t* __restrict__ off, const uint32_t* __restrict__ adj,
                             uint32_t G, int tile_bits, uint32_t seg_bits,
                             uint32_t* __restrict__ ist, uint32_t* __restrict__ tcnt,
                             uint32_t* __restrict__ nbound) {
  const unsigned lane = lane_id();
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t h = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < nh; h += warps) {
    const uint32_t p = pivots[h];
    const uint32_t b = wofs[p], e = wofs[p + 1];
    if (G >= 2) {
      const uint32_t pe = warp_partition(b, e, [&](uint32_t i) { return wvert[i] > p; });
      for (uint32_t g = 1; g + 1 < G; ++g) {
        const uint32_t x = warp_partition(b, pe, [&](uint32_t i) {
          return (off[wvert[i]] >> tile_bits) < g;
        });
        if (lane == 0) ist[(size_t)(g - 1) * nh + h] = x;
      }
      if (lane == 0) ist[(size_t)(G - 2) * nh + h] = pe;
    }
    __syncwarp();
    for (uint32_t g = lane; g < G; g += 32) {
      const uint32_t a = group_bound(ist, wofs, p, h, nh, G, g);
      const uint32_t z = group_bound(ist, wofs, p, h, nh, G, g + 1);
      tcnt[(size_t)g * nh + h] = (z - a + SEG_ITEMS - 1) / SEG_ITEMS;
    }
    if (lane == 0) {
      const uint32_t lo = adj[off[p]], hi = adj[off[p + 1] - 1] + 1;  // hubs have deg+ > 0
      nbound[h] = (hi - lo + seg_bits - 1) / seg_bits + 1;
    }
  }
}

// Segment bounds of every hub pivot, a warp per pivot: bound s is the first
// position of N+(p) holding a rank >= min N+(p) + s * seg_bits (bound 0 is the
// list start, the last one its end).  Written only when they all fit in cap.
__global__ void k_seg_bounds(const uint32_t* __restrict__ pivots, uint32_t nh,
                             const uint32_t* __restrict__ off, const uint32_t* __restrict__ adj,
                             uint32_t seg_bits, const uint32_t* __restrict__ bofs, uint32_t* __restrict__ bnd,
                             uint64_t cap) {
  if ((uint64_t)bofs[nh] > cap) return;
  const unsigned lane = lane_id();
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t h = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < nh; h += warps) {
    const uint32_t p = pivots[h];
    const uint32_t pbeg = off[p], pend = off[p + 1];
    const uint32_t lo = adj[pbeg];
    const uint32_t nb = bofs[h + 1] - bofs[h];  // segments + 1
    uint32_t* out = bnd + bofs[h];
    uint32_t pc = pbeg;
    if (lane == 0) out[0] = pbeg;
    for (uint32_t sgm = 1; sgm + 1 < nb; ++sgm) {
      pc = warp_lower_bound(adj, pc, pend, lo + sgm * seg_bits);
      if (lane == 0) out[sgm] = pc;
    }
    if (lane == 0) out[nb - 1] = pend;
  }
}


// Hits of one round: per-lane count, and in per-vertex and listing modes the
// third vertices (listing ranks follow the warp's lane order).
template <int MODE, int E>
__device__ __forceinline__ void seg_count_hits(const KParams& P, unsigned hits, const uint32_t (&e)[E],
                                               uint32_t& lane_hits, uint32_t& hk, uint2 ends,
                                               uint64_t tb) {
  const uint32_t c = (uint32_t)__popc(hits);
  lane_hits += c;
  if (MODE == M_VERTEX) {
#pragma unroll
    for (int j = 0; j < E; ++j)
      if (hits & (1u << j)) atomicAdd((unsigned long long*)&P.tv[e[j]], 1ull);
  }
  if (MODE == M_LIST_WRITE) {
    const uint32_t incl = warp_inclusive_scan(c);
    uint64_t r = tb + hk + (incl - c);
#pragma unroll
    for (int j = 0; j < E; ++j)
      if (hits & (1u << j)) emit(P, r++, ends, e[j]);
    hk += __shfl_sync(FULL, incl, 31);
  }
}

// Takes the warp's next long item that has entries in the segment (nextv below
// segHi) from the task's shared list; k = NONE when the list is done.
// In a segment after the first, a long item with fewer than `tail` entries
// left is walked by a thread instead (tail = 0: never).
__device__ __forceinline__ bool tail_by_thread(uint32_t remaining, bool later_seg, uint32_t tail) {
  return later_seg && remaining < tail;
}

__device__ __forceinline__ void seg_next_visit(const uint32_t* longs, uint32_t nlong, uint32_t* next,
                                               const uint32_t* nextv, const uint32_t* cur,
                                               const uint32_t* endp, uint32_t segHi, bool later_seg,
                                               uint32_t tail, uint32_t& k, uint32_t& x, uint32_t& y) {
  const unsigned lane = lane_id();
  while (true) {
    uint32_t g = 0;
    if (lane == 0) g = atomicAdd(next, 1u);
    g = __shfl_sync(FULL, g, 0);
    if (g >= nlong) {
      k = NONE;
      x = y = 0;
      return;
    }
    k = longs[g];
    // else nothing of this item in the segment, or a thread walks it
    if (nextv[k] < segHi && !tail_by_thread(endp[k] - cur[k], later_seg, tail)) break;
  }
  x = cur[k];
  y = endp[k];
}

// Membership in the segment [segLo, segLo + 32 words) of N+(p): bit
// b = w - segLo of the shared-memory bitmap.  Entries below segLo wrap to a
// huge b, and every b past the bitmap reads the zero guard word, so a probe
// needs no range test.
struct BitProbe {
  const uint32_t* bm;
  uint32_t segLo, words;
  __device__ __forceinline__ bool operator()(uint32_t w) const {
    const uint32_t b = w - segLo;
    const uint32_t word = bm[min(b >> 5, words)];
    return (__funnelshift_r(word, word, b) & 1u) != 0u;
  }
};

// Membership in the pivot's tail, the entries of N+(p) past its first
// segment: a two-choice cuckoo table of 2^bits shared-memory slots holding
// rank + 1 (0: empty).  Rank w sits in slot h(w) or in h(w) ^ d(w), with
// h(w) = (w * 0x9E3779B1) >> (32 - bits) (Fibonacci hashing) and
// d(w) = ((w * 0x85EBCA77) >> (32 - bits)) | 1 (odd, so the two slots differ
// and each one is the other XOR d(w)).  A probe reads both slots: no loop, no
// divergence.  Entries outside the visit (which the walks mask) may probe as
// hits.
__device__ __forceinline__ uint32_t tail_slot(uint32_t w, uint32_t shift) { return (w * 0x9E3779B1u) >> shift; }
__device__ __forceinline__ uint32_t tail_step(uint32_t w, uint32_t shift) {
  return ((w * 0x85EBCA77u) >> shift) | 1u;
}
struct TailProbe {
  const uint32_t* tab;
  uint32_t shift;
  __device__ __forceinline__ bool operator()(uint32_t w) const {
    const uint32_t h = tail_slot(w, shift);
    const uint32_t a = tab[h], b = tab[h ^ tail_step(w, shift)];
    return (a == w + 1u) | (b == w + 1u);
  }
};
// Insertions that displace more keys than this give up (the table is then
// left for the segment sweep).
constexpr uint32_t TAIL_KICKS = 64;

// One warp advances one item through the segment [segLo, segHi) in rounds of
// 32 E entries: lane L holds the E entries at base + E L .. + E - 1 (E / 4
// 128-bit loads, base = x rounded down to a multiple of E).  An entry w is a
// hit iff it lies in [x, stop) and probe(w) holds (every entry of the round
// is probed: BitProbe and TailProbe take any value).  The visit ends at stop,
// the first index >= x holding an entry >= segHi, or y.  Lists are eta-sorted,
// so a vote on each lane's last entry tells whether stop lies in this round;
// the vote comes before the next round's load (no round past the visit's end
// is loaded), and only the final round computes stop, masks the entries from
// stop on (and, at y, the next list's entries) and returns the entry at stop
// in next_val (NONE at y).  Only lane 0 of the first round can hold entries
// below x.  The adjacency array is padded so that a round starting below y
// never reads past the allocation.
// x: cursor (updated), hk: hits of the item so far (updated).
template <int MODE, int E, class Probe>
__device__ __forceinline__ void seg_walk_item(const KParams& P, const Probe& probe, uint32_t segHi,
                                              uint32_t& x, uint32_t y,
                                              uint32_t& hk, uint2 ends, uint64_t tb,
                                              uint64_t& found, uint32_t& next_val) {
  static_assert(E == 4 || E == 8, "four or eight entries per lane");
  constexpr unsigned ALL = (1u << E) - 1u;
  constexpr uint32_t R = 32 * E;  // entries per round
  const unsigned lane = lane_id();
  uint32_t lane_hits = 0;
  next_val = NONE;
  if (x >= y) return;
  uint32_t base = x & ~(uint32_t)(E - 1);
  const uint4* src = reinterpret_cast<const uint4*>(P.adj + base) + (E / 4) * lane;
  unsigned head = lane == 0 ? (ALL << (x & (E - 1))) & ALL : ALL;  // entries >= x
  uint4 nxt[E / 4];
#pragma unroll
  for (int q = 0; q < E / 4; ++q) nxt[q] = __ldg(src + q);

  while (true) {
    uint32_t e[E];
#pragma unroll
    for (int q = 0; q < E / 4; ++q) {
      e[4 * q] = nxt[q].x;
      e[4 * q + 1] = nxt[q].y;
      e[4 * q + 2] = nxt[q].z;
      e[4 * q + 3] = nxt[q].w;
    }
    const bool tail = base + R >= y;                                 // warp-uniform: this round reaches y
    const bool fin = __any_sync(FULL, e[E - 1] >= segHi) || tail;   // warp-uniform: the visit ends here
    if (!fin) {  // the next round, only when the visit goes on
#pragma unroll
      for (int q = 0; q < E / 4; ++q) nxt[q] = __ldg(src + 8 * E + q);
    }
    unsigned hits = 0;
#pragma unroll
    for (int j = 0; j < E; ++j) hits |= (unsigned)probe(e[j]) << j;
    hits &= head;
    uint32_t stop = NONE;
    if (fin) {
      const uint32_t idx0 = base + E * lane;
      // entries below segHi, and those below x, are passed over
      unsigned below = ~head & ALL;
#pragma unroll
      for (int j = 0; j < E; ++j) below |= (unsigned)(e[j] < segHi) << j;
      const uint32_t j = (uint32_t)__ffs(~below) - 1u;  // 0..E
      stop = min(__reduce_min_sync(FULL, j < E ? idx0 + j : NONE), y);
      const uint32_t keep = idx0 < stop ? min(stop - idx0, (uint32_t)E) : 0u;
      hits &= (1u << keep) - 1u;
      const uint32_t rel = stop - base;  // 0..R
      const uint32_t rj = rel & (E - 1);
      uint32_t at = e[0];
#pragma unroll
      for (int q = 1; q < E; ++q)
        if (rj == (uint32_t)q) at = e[q];
      const uint32_t val = __shfl_sync(FULL, at, (rel / E) & 31u);
      next_val = stop < y ? val : NONE;
    }
    seg_count_hits<MODE, E>(P, hits, e, lane_hits, hk, ends, tb);
    if (fin) {
      x = stop;
      break;
    }
    head = ALL;
    base += R;
    src += 8 * E;
  }
  found += lane_hits;
  if (MODE != M_COUNT && MODE != M_LIST_WRITE) hk += __reduce_add_sync(FULL, lane_hits);
}

// One thread advances one short item through the segment [segLo, segHi)
// (hits: probe(w)): eight entries per step from two aligned 128-bit loads (base = x rounded
// down to a multiple of 4; the entries below x are passed over), stopping at
// the item's end y or at the first entry >= segHi, whose value is returned in
// nv.  Hits come out in order (listing ranks hk + i).  The padded adjacency
// array keeps the loads inside the allocation.
template <int MODE, class Probe>
__device__ __forceinline__ void seg_walk_short(const KParams& P, const Probe& probe, uint32_t segHi,
                                               uint32_t& x, uint32_t y, uint32_t& nv, uint32_t& hk,
                                               uint2 ends, uint64_t tb, uint64_t& found) {
  nv = NONE;
  while (x < y) {
    const uint32_t b0 = x & ~3u;
    const uint4* q = reinterpret_cast<const uint4*>(P.adj + b0);
    const uint4 lo = __ldg(q), hi = __ldg(q + 1);
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
    const uint32_t j0 = x & 3u;
    uint32_t nx = b0 + 8;  // the cursor after these eight, unless the visit stops
    bool stop = false;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (stop || (uint32_t)j < j0) continue;
      const uint32_t idx = b0 + j;
      if (idx >= y) {  // the item's end
        stop = true;
        nx = y;
        continue;
      }
      if (w[j] >= segHi) {  // the segment's end: resume here in a later segment
        stop = true;
        nx = idx;
        nv = w[j];
        continue;
      }
      if (probe(w[j])) {
        ++found;
        if (MODE == M_VERTEX) atomicAdd((unsigned long long*)&P.tv[w[j]], 1ull);
        if (MODE == M_LIST_WRITE) emit(P, tb + hk, ends, w[j]);
        ++hk;
      }
    }
    x = nx;
    if (stop) break;
  }
  if (x >= y) nv = NONE;
}

// Tasks: task_ofs[k] (k = g nh + h, K = G nh of them, plus the total) is the
// first task of work group g of hub h, whose items are [bound(g), bound(g+1))
// (k_seg_groups).
template <int MODE>
__global__ void __launch_bounds__(SEG_THREADS, 1) k_seg_pivots(KParams P, const uint32_t* __restrict__ task_ofs,
                                                               const uint32_t* __restrict__ ist,
                                                               uint32_t nh, uint32_t G, uint32_t seg_bits,
                                                               uint32_t seg_long, uint32_t seg_wide,
                                                               uint32_t seg_tail, uint32_t seg_hash,
                                                               const uint32_t* __restrict__ bofs,
                                                               const uint32_t* __restrict__ bnd,
                                                               uint64_t bcap) {
  extern __shared__ uint32_t seg_sm[];
  const uint32_t seg_words = seg_bits / 32;
  uint32_t* bm = seg_sm;
  uint32_t* cur = bm + seg_words + 4;
  uint32_t* endp = cur + SEG_ITEMS;
  uint32_t* nextv = endp + SEG_ITEMS;
  uint32_t* ih = nextv + SEG_ITEMS;
  uint32_t* longs = ih + SEG_ITEMS;                              // long items of the task
  uint8_t* islong = reinterpret_cast<uint8_t*>(longs + SEG_ITEMS);
  __shared__ uint32_t s_task, s_grp, s_pe, s_next, s_nlong;
  __shared__ uint32_t s_bound[SEG_MAXB];  // this pivot's segment bounds (when they fit)
  __shared__ unsigned long long s_hits, s_stage;
  __shared__ uint32_t s_tfail;
  const unsigned lane = lane_id(), wid = threadIdx.x >> 5;
  const uint32_t K = G * nh;
  const uint32_t ntasks = task_ofs[K];
  const bool have_bounds = bnd != nullptr && (uint64_t)bofs[nh] <= bcap;
  // the tail table takes the bitmap's words: 2^tbits slots (two-choice
  // cuckoo tables fill up to about half; a fuller one fails to build)
  const uint32_t tbits = 31u - (uint32_t)__clz(seg_words);
  const uint32_t tslots = 1u << tbits, tshift = 32u - tbits;
  const uint32_t hcap = min(seg_hash, tslots);
  for (uint32_t i = threadIdx.x; i <= seg_words; i += blockDim.x) bm[i] = 0;  // + guard word
  uint64_t found = 0;
  while (true) {
    if (threadIdx.x == 0) {
      s_task = atomicAdd(&P.dev->counters[Q_SEG], 1u);
      s_hits = 0;
      s_stage = 0;
      s_tfail = 0;
      s_nlong = 0;
    }
    __syncthreads();
    const uint32_t task = s_task;
    if (task >= ntasks) break;
    if (wid == 0) {  // largest k with task_ofs[k] <= task (32-ary search)
      uint32_t lo = 0, hi = K;
      while (hi - lo > 1) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t idx = lo + lane * step;
        const bool le = idx < hi && task_ofs[idx] <= task;
        const int c = __popc(__ballot_sync(FULL, le));
        const uint32_t nlo = lo + (uint32_t)(c - 1) * step;
        const uint32_t nhi = min(hi, lo + (uint32_t)c * step);
        lo = nlo;
        hi = nhi;
      }
      if (lane == 0) s_grp = lo;
    }
    __syncthreads();
    const uint32_t kg = s_grp;
    const uint32_t h = kg % nh, grp = kg / nh;
    const uint32_t p = P.pivots[h];
    if (P.rprobe && P.rprobe[p] == 0) {  // every item of p takes another route
      __syncthreads();
      continue;
    }
    // the pivot's list and its segment bounds (read while the items load)
    const uint32_t pbeg = P.off[p], pend = P.off[p + 1];
    const uint32_t nb = have_bounds ? bofs[h + 1] - bofs[h] : 0u;
    const bool use_bounds = nb != 0 && nb <= SEG_MAXB;
    if (use_bounds)
      for (uint32_t t = threadIdx.x; t < nb; t += blockDim.x) s_bound[t] = bnd[bofs[h] + t];
    const uint32_t i0 = group_bound(ist, P.wofs, p, h, nh, G, grp) + (task - task_ofs[kg]) * SEG_ITEMS;
    const uint32_t i1 = min(i0 + SEG_ITEMS, group_bound(ist, P.wofs, p, h, nh, G, grp + 1));
    if (MODE == M_LIST_WRITE && !list_window_overlaps(P, i0, i1)) {  // nothing of this task in the window
      __syncthreads();
      continue;
    }
    const uint32_t nk = i1 - i0;
    int live = 0;  // does any item of this task walk anything?
    for (uint32_t k = threadIdx.x; k < nk; k += blockDim.x) {
      uint2 r = P.witem[i0 + k];
      const bool mine = !P.route || P.route[i0 + k] == V_PROBE;
      if (!mine) r.y = r.x;
      if (MODE == M_LIST_WRITE) {
        const uint32_t e = P.wedge[i0 + k];
        const uint64_t a = P.toff[e], b = P.toff[e + 1];
        if (a == b || b <= P.cursor || a >= P.cursor + P.cap) r.y = r.x;
      }
      cur[k] = r.x;
      endp[k] = r.y;
      nextv[k] = r.x < r.y ? P.adj[r.x] : NONE;
      ih[k] = mine ? 0u : NONE;  // NONE: the item belongs to another route
      live |= r.x < r.y;
      const bool lg = r.y - r.x >= seg_long;  // long items are walked warp-wide
      islong[k] = lg;
      if (lg) longs[atomicAdd(&s_nlong, 1u)] = k;
    }
    if (!__syncthreads_or(live)) {  // nothing to walk: results only (zero hits)
      if (MODE == M_LIST_COUNT || MODE == M_TIMED)
        for (uint32_t k = threadIdx.x; k < nk; k += blockDim.x)
          if (ih[k] != NONE) {
            if (MODE == M_LIST_COUNT) P.tcnt[P.wedge[i0 + k]] = 0;
            else P.cyc[P.wedge[i0 + k]] = 0;
          }
      __syncthreads();
      continue;
    }
    const uint32_t lo_rank = P.adj[pbeg], hi_rank = P.adj[pend - 1] + 1;
    uint32_t pc = pbeg;
    __syncthreads();
    // every item with entries in [.., segHi) advances through the segment,
    // short ones a thread each, long ones a warp each
    auto visit = [&](const auto& probe, uint32_t segHi, bool later_seg) {
      for (uint32_t k = threadIdx.x; k < nk; k += blockDim.x) {
        if ((islong[k] && !tail_by_thread(endp[k] - cur[k], later_seg, seg_tail)) || nextv[k] >= segHi)
          continue;
        uint32_t x = cur[k], hk = ih[k], nv;
        uint2 ends = make_uint2(0u, 0u);
        uint64_t tb = 0;
        if (MODE == M_LIST_WRITE) {
          ends = emit_ends(P, p, P.wvert[i0 + k]);
          tb = P.toff[P.wedge[i0 + k]];
        }
        const long long tv0 = MODE == M_TIMED ? clock64() : 0;
        seg_walk_short<MODE>(P, probe, segHi, x, endp[k], nv, hk, ends, tb, found);
        if (MODE == M_TIMED) hk = ih[k] + sat_cycles(clock64() - tv0);  // ih holds cycles here
        cur[k] = x;
        nextv[k] = nv;
        ih[k] = hk;
      }
      const uint32_t nlong = s_nlong;
      while (true) {
        uint32_t k, x, y;
        seg_next_visit(longs, nlong, &s_next, nextv, cur, endp, segHi, later_seg, seg_tail, k, x, y);
        if (k == NONE) break;
        uint32_t hk = ih[k], nv;
        uint2 ends = make_uint2(0u, 0u);
        uint64_t tb = 0;
        if (MODE == M_LIST_WRITE) {
          ends = emit_ends(P, p, P.wvert[i0 + k]);
          tb = P.toff[P.wedge[i0 + k]];
        }
        const long long tv0 = MODE == M_TIMED ? clock64() : 0;
        if (y - x >= seg_wide)  // long remaining list: rounds of 256 entries
          seg_walk_item<MODE, 8>(P, probe, segHi, x, y, hk, ends, tb, found, nv);
        else
          seg_walk_item<MODE, 4>(P, probe, segHi, x, y, hk, ends, tb, found, nv);
        if (MODE == M_TIMED) hk = ih[k] + sat_cycles(clock64() - tv0);  // ih holds cycles here
        __syncwarp();
        if (lane == 0) {
          cur[k] = x;
          nextv[k] = nv;
          ih[k] = hk;
        }
        __syncwarp();
      }
    };
    uint32_t sgm = 0;
    bool tail_ok = true;  // block-uniform: may the tail table be tried?
    for (uint32_t segLo = lo_rank; segLo < hi_rank; segLo += seg_bits, ++sgm) {
      uint32_t segHi = min(segLo + seg_bits, hi_rank);
      // after the first segment, a pivot whose entries left fit the tail
      // table takes all its later segments in one pass over a hash of them
      bool hashed = tail_ok && sgm > 0 && segHi < hi_rank && pend - pc <= hcap;
      const long long tset0 = MODE == M_TIMED ? clock64() : 0;
      if (hashed) {
        for (uint32_t k = pc + threadIdx.x; k < pend; k += blockDim.x) {
          uint32_t key = P.adj[k] + 1u;  // distinct keys
          uint32_t h = tail_slot(key - 1u, tshift);
          uint32_t i = 0;
          for (; i < TAIL_KICKS; ++i) {
            key = atomicExch(&bm[h], key);  // place it, taking what was there
            if (key == 0u) break;
            h ^= tail_step(key - 1u, tshift);  // the displaced key's other slot
          }
          if (i == TAIL_KICKS) s_tfail = 1u;  // a key is out of the table
        }
        __syncthreads();
        if (s_tfail) {  // sweep the segments instead
          for (uint32_t i = threadIdx.x; i < tslots; i += blockDim.x) bm[i] = 0u;
          hashed = tail_ok = false;
        } else {
          segHi = hi_rank;
        }
      }
      if (!hashed && !use_bounds && wid == 0) {
        const uint32_t pe = warp_lower_bound(P.adj, pc, pend, segHi);
        if (lane == 0) s_pe = pe;
      }
      if (threadIdx.x == 0) s_next = 0;
      __syncthreads();
      const uint32_t pe = hashed ? pend : use_bounds ? s_bound[sgm + 1] : s_pe;
      if (pe > pc) {
        if (!hashed) {
          for (uint32_t k = pc + threadIdx.x; k < pe; k += blockDim.x) {
            const uint32_t b = P.adj[k] - segLo;
            atomicOr(&bm[b >> 5], 1u << (b & 31));
          }
          __syncthreads();
        }
        if (MODE == M_TIMED && threadIdx.x == 0) s_stage += (unsigned long long)(clock64() - tset0) * (blockDim.x >> 5);
        if (hashed)
          visit(TailProbe{bm, tshift}, segHi, true);
        else
          visit(BitProbe{bm, segLo, seg_words}, segHi, sgm > 0);
        __syncthreads();
        if (hashed) {
          for (uint32_t i = threadIdx.x; i < tslots; i += blockDim.x) bm[i] = 0u;
        } else {
          for (uint32_t k = pc + threadIdx.x; k < pe; k += blockDim.x) {
            const uint32_t b = P.adj[k] - segLo;
            bm[b >> 5] = 0u;
          }
        }
      }
      pc = pe;
      __syncthreads();
      if (hashed) break;
    }
    if (MODE == M_TIMED) {
      const unsigned long long sh = s_stage / (unsigned long long)max(1u, nk);
      const uint32_t share = sh > 0xffffffffull ? 0xffffffffu : (uint32_t)sh;
      for (uint32_t k = threadIdx.x; k < nk; k += blockDim.x)
        if (ih[k] != NONE) P.cyc[P.wedge[i0 + k]] = ih[k] + share;
    }
    if (MODE != M_COUNT && MODE != M_TIMED) {
      uint32_t th = 0;
      for (uint32_t k = threadIdx.x; k < nk; k += blockDim.x) {
        const uint32_t hk = ih[k];
        if (hk == NONE) continue;
        th += hk;
        if (MODE == M_VERTEX && hk) atomicAdd((unsigned long long*)&P.tv[P.wvert[i0 + k]], (unsigned long long)hk);
        if (MODE == M_LIST_COUNT) P.tcnt[P.wedge[i0 + k]] = hk;
      }
      if (MODE == M_VERTEX) {
        th = warp_sum(th);
        if (lane == 0 && th) atomicAdd(&s_hits, (unsigned long long)th);
        __syncthreads();
        if (threadIdx.x == 0 && s_hits) atomicAdd((unsigned long long*)&P.tv[p], s_hits);
      }
    }
    __syncthreads();
  }
  found = warp_sum(found);
  if (lane == 0 && found) atomicAdd(&P.dev->total, (unsigned long long)found);
}

__global__ void k_hub_info(const uint32_t* __restrict__ pivots, uint32_t nh,
                           const uint32_t* __restrict__ wofs, const uint32_t* __restrict__ off,
                           uint32_t* __restrict__ info) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nh) return;
  uint32_t p = pivots[i];
  info[4 * (size_t)i + 0] = p;
  info[4 * (size_t)i + 1] = wofs[p];
  info[4 * (size_t)i + 2] = wofs[p + 1];
  info[4 * (size_t)i + 3] = off[p + 1] - off[p];
}

// ------------------------------------------------------------------ driver
#define AOT_MODE_NAMES(k) {#k "/count", #k "/vertex", #k "/list_count", #k "/list_write", #k "/timed"}
static const char* const kWarpNames[5] = AOT_MODE_NAMES(k_warp_pivots);
static const char* const kCtaNames[5] = AOT_MODE_NAMES(k_cta_pivots);
static const char* const kHubNames[5] = AOT_MODE_NAMES(k_hub_walk);
static const char* const kSegNames[5] = AOT_MODE_NAMES(k_seg_pivots);
static const char* const kWarpCtaNames[5] = AOT_MODE_NAMES(k_warp_pivots_ctabin);  // the CTA bin a warp per pivot
template <int MODE>
static const char* mode_name(const char* base) {
  if (base[2] == 'w') return kWarpNames[MODE];
  if (base[2] == 'c') return kCtaNames[MODE];
  if (base[2] == 's') return kSegNames[MODE];
  return kHubNames[MODE];
}

template <int MODE>
static aot_status launch_bins(aot_graph* g, KParams P, cudaStream_t s) {
  const uint32_t nw = g->bin_count[BIN_WARP], nc = g->bin_count[BIN_CTA], nh = g->bin_count[BIN_HUB];
  const int sms = sm_count();
  // a warp per pivot with ts_max-slot tables; warps per CTA chosen (8, 4, 2
  // or 1) for the most resident warps
  auto launch_warps = [&](uint32_t count, uint32_t ts_max, int q, const char* name) -> aot_status {
    const size_t per_warp = warp_pivot_words<MODE>(ts_max) * sizeof(uint32_t);
    const size_t smem_cap = 227 * 1024;
    const size_t attr = per_warp * 8 < smem_cap ? per_warp * 8 : smem_cap;
    AOT_TRY(ensure_dyn_smem((const void*)k_warp_pivots<MODE>, attr));
    int warps_per_block = 1, per_sm = 0, best = -1;
    for (int w = 8; w >= 1; w >>= 1) {
      const size_t sm_bytes = (size_t)w * per_warp;
      if (sm_bytes > attr && sm_bytes > 48 * 1024) continue;
      int b = 0;
      AOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_warp_pivots<MODE>, 32 * w, sm_bytes));
      if (b * w > best) {
        best = b * w;
        warps_per_block = w;
        per_sm = b;
      }
    }
    const size_t smem = (size_t)warps_per_block * per_warp;
    int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int64_t need = ((int64_t)count + warps_per_block - 1) / warps_per_block;
    if (grid > need) grid = need;
    AOT_KERNEL(name, s)
      k_warp_pivots<MODE><<<(unsigned)grid, 32 * warps_per_block, smem, s>>>(P, ts_max, q);
    return last_launch();
  };
  if (nw) {
    P.pivots = g->bin_pivots;
    P.num_pivots = nw;
    AOT_TRY(launch_warps(nw, WARP_TS, Q_WARP, mode_name<MODE>("k_warp_pivots")));
  }
  uint32_t cta_ts = 64;  // table slots of the CTA bin: a power of two >= 2 cta_max
  while (cta_ts < 2 * g->binned_cta_max) cta_ts <<= 1;
  if (nc && g->tune.cta_threads == 32) {  // the CTA bin a warp per pivot
    P.pivots = g->bin_pivots + nw;
    P.num_pivots = nc;
    AOT_TRY(launch_warps(nc, cta_ts, Q_CTA, kWarpCtaNames[MODE]));
  } else if (nc) {
    P.pivots = g->bin_pivots + nw;
    P.num_pivots = nc;
    const uint32_t ts_max = cta_ts;
    size_t smem = (size_t)ts_max * 2 * sizeof(uint32_t);
    AOT_TRY(ensure_dyn_smem((const void*)k_cta_pivots<MODE>, smem));
    const int threads = g->tune.cta_threads;
    int per_sm = 0;
    AOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cta_pivots<MODE>, threads, smem));
    int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    if (grid > nc) grid = nc;
    AOT_KERNEL(mode_name<MODE>("k_cta_pivots"), s)
      k_cta_pivots<MODE><<<(unsigned)grid, threads, smem, s>>>(P, ts_max);
    AOT_TRY(last_launch());
  }
  // the segmented sweep needs eta-sorted out-lists: a random local order
  // takes the global bitmaps
  const int hub_mode = (g->flags & AOT_FLAG_LOCAL_RANDOM) ? 1 : g->tune.hub_mode;
  if (nh && hub_mode == 0) {
    // segmented shared-memory bitmap: tasks = (work group of a pivot, block
    // of SEG_ITEMS items), groups = tiles of the walked out-lists + negatives
    const uint32_t* dp = g->bin_pivots + nw + nc;
    const uint32_t seg_bits = g->tune.seg_bits;
    // hubinfo (4n words): inner group bounds ((G-1) nh) | task counts, then
    // offsets (G nh + 1) | bound counts (nh) | bound offsets (nh + 1) | segment
    // bounds (what is left: they are skipped when they do not fit).  G groups
    // need (2G + 1) nh + 2 <= 4n words; G = 1 always fits (nh <= n).
    const uint64_t n4 = 4 * (uint64_t)g->n;
    const int tb = (int)g->tune.tile_bits;
    const uint64_t gmax = ((n4 - 2) / nh - 1) / 2;
    uint64_t gw = tb ? (((uint64_t)g->m - 1) >> tb) + 2 : 1;  // tiles + the negative items
    if (gw > gmax) gw = gmax;
    if (gw < 2) gw = 1;
    const uint32_t G = (uint32_t)gw;
    const uint32_t K = G * nh;
    uint32_t* ist = g->hubinfo;
    uint32_t* task_ofs = ist + (size_t)(G - 1) * nh;
    uint32_t* nbound = task_ofs + K + 1;
    uint32_t* bofs = nbound + nh;
    uint32_t* bnd = bofs + nh + 1;
    const uint64_t used = (uint64_t)(bnd - g->hubinfo);
    // every pivot has at most ceil(n / seg_bits) segments: take the bounds only
    // when that many fit (this also keeps the 32-bit offsets exact)
    const uint64_t worst = (uint64_t)nh * (((uint64_t)g->n + seg_bits - 1) / seg_bits + 1);
    const uint64_t room = used < n4 ? n4 - used : 0;
    const uint64_t bcap = worst <= room && worst < 0xffffffffull ? room : 0;
    int64_t ggrid = ((int64_t)nh * 32 + 255) / 256;
    if (ggrid > (int64_t)sms * 8) ggrid = (int64_t)sms * 8;
    AOT_KERNEL("k_seg_groups", s)
      k_seg_groups<<<(unsigned)ggrid, 256, 0, s>>>(dp, nh, g->wofs, g->wvert, g->off, g->adj, G, tb,
                                                   seg_bits, ist, task_ofs, nbound);
    AOT_TRY(last_launch());
    AOT_TRY(scan_u32_u32(task_ofs, task_ofs, K, g->scan_tmp, s));
    if (bcap) {
      AOT_TRY(scan_u32_u32(nbound, bofs, nh, g->scan_tmp, s));
      int64_t bgrid = ((int64_t)nh * 32 + 255) / 256;
      if (bgrid > (int64_t)sms * 8) bgrid = (int64_t)sms * 8;
      AOT_KERNEL("k_seg_bounds", s)
        k_seg_bounds<<<(unsigned)bgrid, 256, 0, s>>>(dp, nh, g->off, g->adj, seg_bits, bofs, bnd, bcap);
      AOT_TRY(last_launch());
    }
    const size_t seg_smem = seg_smem_bytes(seg_bits);
    AOT_TRY(ensure_dyn_smem((const void*)k_seg_pivots<MODE>, seg_smem_bytes(SEG_BITS_MAX)));
    P.pivots = dp;
    P.num_pivots = nh;
    int per_sm = 0;
    const int seg_threads = g->tune.seg_threads;
    AOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_seg_pivots<MODE>, seg_threads, seg_smem));
    AOT_KERNEL(mode_name<MODE>("k_seg_pivots"), s)
      k_seg_pivots<MODE><<<(unsigned)(sms * (per_sm > 0 ? per_sm : 1)), seg_threads, seg_smem, s>>>(
          P, task_ofs, ist, nh, G, seg_bits, g->tune.seg_long, g->tune.seg_wide, g->tune.seg_tail, g->tune.seg_hash, bofs,
          bcap ? bnd : nullptr,
          bcap);
    AOT_TRY(last_launch());
  } else if (nh) {
    // hub descriptors on the host (hubs are few): pivot, first item, end item, deg+
    const uint32_t* dp = g->bin_pivots + nw + nc;
    AOT_KERNEL("k_hub_info", s)
      k_hub_info<<<(nh + 255) / 256, 256, 0, s>>>(dp, nh, g->wofs, g->off, g->hubinfo);
    AOT_TRY(last_launch());
    std::vector<uint32_t> hpv(4 * (size_t)nh);
    uint32_t* hp = hpv.data();
    AOT_CUDA(cudaMemcpyAsync(hp, g->hubinfo, sizeof(uint32_t) * 4 * nh, cudaMemcpyDeviceToHost, s));
    AOT_CUDA(cudaStreamSynchronize(s));
    const uint32_t words = (uint32_t)(((int64_t)g->n + 31) / 32);
    int per_group = g->tune.hub_bitmaps < MAX_HUBS ? g->tune.hub_bitmaps : MAX_HUBS;
    // the workspace starts uninitialised; every group clears the words it set
    AOT_CUDA(cudaMemsetAsync(g->hub_bitmap, 0, sizeof(uint32_t) * (size_t)words * per_group, s));
    for (uint32_t h0 = 0; h0 < nh; h0 += per_group) {
      HubGroup G;
      G.count = (int)((nh - h0) < (uint32_t)per_group ? (nh - h0) : (uint32_t)per_group);
      G.words = words;
      G.bitmap = g->hub_bitmap;
      G.cbeg[0] = 0;
      uint32_t maxdeg = 0;
      for (int b = 0; b < G.count; ++b) {
        const uint32_t* h = hp + 4 * (size_t)(h0 + b);
        G.pivot[b] = h[0];
        G.ib[b] = h[1];
        G.ie[b] = h[2];
        G.cbeg[b + 1] = G.cbeg[b] + (h[2] - h[1] + 31) / 32;
        if (h[3] > maxdeg) maxdeg = h[3];
      }
      dim3 sgrid((maxdeg + 255) / 256 < 64 ? (maxdeg + 255) / 256 : 64, G.count);
      if (sgrid.x == 0) sgrid.x = 1;
      AOT_KERNEL("k_hub_bits", s)
        k_hub_bits<<<sgrid, 256, 0, s>>>(G, g->off, g->adj, true);
      AOT_TRY(last_launch());
      int per_sm = 0;
      AOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hub_walk<MODE>, 256, 0));
      int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
      int64_t need = ((int64_t)G.cbeg[G.count] + 7) / 8;
      if (grid > need) grid = need;
      if (grid < 1) grid = 1;
      AOT_KERNEL(mode_name<MODE>("k_hub_walk"), s)
        k_hub_walk<MODE><<<(unsigned)grid, 256, 0, s>>>(P, G);
      AOT_TRY(last_launch());
      AOT_KERNEL("k_hub_bits", s)
        k_hub_bits<<<sgrid, 256, 0, s>>>(G, g->off, g->adj, false);
      AOT_TRY(last_launch());
    }
  }
  return AOT_OK;
}

static KParams base_params(aot_graph* g) {
  KParams P;
  P.off = g->off;
  P.adj = g->adj;
  P.wofs = g->wofs;
  P.witem = g->witem;
  P.wvert = g->wvert;
  P.wedge = g->wedge;
  P.pivots = nullptr;
  P.num_pivots = 0;
  P.tv = g->tv;
  P.tcnt = g->tcnt;
  P.toff = g->toff;
  P.perm = g->perm;
  P.out = nullptr;
  P.cursor = 0;
  P.cap = 0;
  P.dev = g->dev;
  P.route = g->routed ? g->route : nullptr;
  P.rprobe = g->routed ? g->rprobe : nullptr;
  P.cyc = nullptr;
  P.lblk = nullptr;
  return P;
}

static aot_status reset_scalars(aot_graph* g, cudaStream_t s) {
  AOT_CUDA(cudaMemsetAsync(&g->dev->total, 0, sizeof(unsigned long long), s));
  AOT_CUDA(cudaMemsetAsync(g->dev->counters + 1, 0, sizeof(unsigned int) * 14, s));
  return AOT_OK;
}

static aot_status check_route(aot_graph* g, aot_route route) {
  if (!g) return AOT_ERR_INVALID_ARG;
  if ((int)route < (int)AOT_ROUTE_PLAIN || (int)route > (int)AOT_ROUTE_RANDOM) return AOT_ERR_INVALID_ARG;
  // merge and binary search need eta-sorted out-lists
  if ((g->flags & AOT_FLAG_LOCAL_RANDOM) && route != AOT_ROUTE_PLAIN && route != AOT_ROUTE_PROBE)
    return AOT_ERR_INVALID_ARG;
  if (route == AOT_ROUTE_LEARNED && !g->model) return AOT_ERR_NOT_READY;
  if (g->max_outdeg >= (1 << 27)) return AOT_ERR_OVERFLOW;
  return AOT_OK;
}

// route the items, then run the pivot kernels and the staging-free kernel
template <int MODE>
static aot_status run_mode(aot_graph* g, aot_route route, KParams P, cudaStream_t s,
                           int sample_log2 = 0) {
  AOT_TRY(route_items(g, route, s, sample_log2));
  P.route = g->routed ? g->route : nullptr;
  P.rprobe = g->routed ? g->rprobe : nullptr;
  AOT_TRY(launch_bins<MODE>(g, P, s));
  return launch_ep<MODE>(g, P, s);
}

// Listing block ranges (see LIST_BLOCK): a CTA per block of work items.
__global__ void __launch_bounds__(256) k_list_blocks(const uint32_t* __restrict__ wedge,
                                                     const uint64_t* __restrict__ toff, uint32_t items,
                                                     uint32_t nblk, uint64_t* __restrict__ lblk) {
  __shared__ unsigned long long s_lo, s_hi;
  for (uint32_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    if (threadIdx.x == 0) {
      s_lo = ~0ull;
      s_hi = 0;
    }
    __syncthreads();
    unsigned long long lo = ~0ull, hi = 0;
    const uint32_t i0 = blk * LIST_BLOCK, i1 = min(i0 + LIST_BLOCK, items);
    for (uint32_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const uint32_t e = wedge[i];
      const unsigned long long a = toff[e], b = toff[e + 1];
      if (a < b) {
        lo = min(lo, a);
        hi = max(hi, b);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(FULL, lo, o));
      hi = max(hi, __shfl_xor_sync(FULL, hi, o));
    }
    if (lane_id() == 0) {
      atomicMin(&s_lo, lo);
      atomicMax(&s_hi, hi);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      lblk[2 * (size_t)blk] = s_lo;
      lblk[2 * (size_t)blk + 1] = s_hi;
    }
    __syncthreads();
  }
}

__global__ void k_gather_counts(const uint64_t* __restrict__ tv, const int32_t* __restrict__ rank,
                                int32_t n, uint64_t* __restrict__ out) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) out[v] = tv[rank[v]];
}

}  // namespace aot

using namespace aot;

extern "C" aot_status aot_count(aot_graph* g, aot_route route, uint64_t* h_total, aot_stream_t stream) {
  AOT_TRY(check_route(g, route));
  if (!h_total) return AOT_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  AOT_TRY(reset_scalars(g, s));
  if (g->m > 0) AOT_TRY(run_mode<M_COUNT>(g, route, base_params(g), s));
  unsigned long long t = 0;
  AOT_CUDA(cudaMemcpyAsync(&t, &g->dev->total, sizeof(t), cudaMemcpyDeviceToHost, s));
  AOT_CUDA(cudaStreamSynchronize(s));
  AOT_TRY(read_device_error(g, s));
  *h_total = t;
  return AOT_OK;
}

extern "C" aot_status aot_count_per_vertex(aot_graph* g, aot_route route, uint64_t* d_counts,
                                           uint64_t* h_total, aot_stream_t stream) {
  AOT_TRY(check_route(g, route));
  if (!d_counts && g->n > 0) return AOT_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  AOT_TRY(reset_scalars(g, s));
  if (g->n > 0) {
    AOT_CUDA(cudaMemsetAsync(g->tv, 0, sizeof(uint64_t) * g->n, s));
    if (g->m > 0) AOT_TRY(run_mode<M_VERTEX>(g, route, base_params(g), s));
    AOT_KERNEL("k_gather_counts", s)
      k_gather_counts<<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(g->tv, g->rank, g->n, d_counts);
    AOT_TRY(last_launch());
  }
  if (h_total) {
    unsigned long long t = 0;
    AOT_CUDA(cudaMemcpyAsync(&t, &g->dev->total, sizeof(t), cudaMemcpyDeviceToHost, s));
    AOT_CUDA(cudaStreamSynchronize(s));
    AOT_TRY(read_device_error(g, s));
    *h_total = t;
  }
  return AOT_OK;
}

extern "C" aot_status aot_graph_record_costs(aot_graph* g, int32_t variant, int32_t sample_log2,
                                             uint32_t* d_cycles, aot_stream_t stream) {
  if (!g || (g->m > 0 && !d_cycles) || variant < 0 || variant > 2) return AOT_ERR_INVALID_ARG;
  if (sample_log2 < 0 || sample_log2 > 30) return AOT_ERR_INVALID_ARG;
  if ((g->flags & AOT_FLAG_LOCAL_RANDOM) && variant != V_PROBE) return AOT_ERR_INVALID_ARG;
  if (g->max_outdeg >= (1 << 27)) return AOT_ERR_OVERFLOW;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (g->m == 0) return AOT_OK;
  AOT_CUDA(cudaMemsetAsync(d_cycles, 0, sizeof(uint32_t) * g->m, s));
  AOT_TRY(reset_scalars(g, s));
  const aot_route r = variant == V_PROBE ? AOT_ROUTE_PROBE : variant == V_MERGE ? AOT_ROUTE_MERGE : AOT_ROUTE_BSEARCH;
  KParams P = base_params(g);
  P.cyc = d_cycles;
  AOT_TRY(run_mode<M_TIMED>(g, r, P, s, variant == V_PROBE ? 0 : sample_log2));
  AOT_CUDA(cudaStreamSynchronize(s));
  return read_device_error(g, s);
}

extern "C" aot_status aot_list(aot_graph* g, aot_route route, uint64_t cursor, int32_t* d_out,
                               uint64_t cap, uint64_t* h_written, uint64_t* h_next, aot_stream_t stream) {
  AOT_TRY(check_route(g, route));
  if (!h_written || !h_next || (cap > 0 && !d_out)) return AOT_ERR_INVALID_ARG;
  if (g->flags & AOT_FLAG_LOCAL_RANDOM) return AOT_ERR_INVALID_ARG;  // no canonical order
  if (!g->has_list) return AOT_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!g->list_ready) {
    g->list_total = 0;
    if (g->m > 0) {
      AOT_TRY(reset_scalars(g, s));
      AOT_CUDA(cudaMemsetAsync(g->tcnt, 0, sizeof(uint32_t) * g->m, s));
      AOT_TRY(run_mode<M_LIST_COUNT>(g, route, base_params(g), s));
      AOT_TRY(scan_u32_u64(g->tcnt, g->toff, g->m, g->scan_tmp, s));
      // block ranges in tcnt's words, dead after the scan (a 256-byte piece
      // of at least 4 m bytes holds the 16 ceil(m / LIST_BLOCK) it needs)
      const uint64_t nblk = ((uint64_t)g->m + LIST_BLOCK - 1) / LIST_BLOCK;
      const uint64_t room = ((uint64_t)g->m * sizeof(uint32_t) + 255) & ~(uint64_t)255;
      g->lblk = nullptr;
      if (16 * nblk <= room) {
        g->lblk = reinterpret_cast<uint64_t*>(g->tcnt);
        unsigned grid = (unsigned)(nblk < (uint64_t)sm_count() * 16 ? nblk : (uint64_t)sm_count() * 16);
        AOT_KERNEL("k_list_blocks", s)
          k_list_blocks<<<grid, 256, 0, s>>>(g->wedge, g->toff, (uint32_t)g->m, (uint32_t)nblk, g->lblk);
        AOT_TRY(last_launch());
      }
      unsigned long long t = 0;
      AOT_CUDA(cudaMemcpyAsync(&t, g->toff + g->m, sizeof(t), cudaMemcpyDeviceToHost, s));
      AOT_CUDA(cudaStreamSynchronize(s));
      AOT_TRY(read_device_error(g, s));
      g->list_total = t;
    }
    g->list_ready = true;
  }
  const uint64_t T = g->list_total;
  if (cursor > T) return AOT_ERR_INVALID_ARG;
  uint64_t k = T - cursor < cap ? T - cursor : cap;
  if (k > 0) {
    KParams P = base_params(g);
    P.out = d_out;
    P.cursor = cursor;
    P.cap = k;
    P.lblk = g->lblk;
    AOT_TRY(reset_scalars(g, s));
    AOT_TRY(run_mode<M_LIST_WRITE>(g, route, P, s));
    AOT_CUDA(cudaStreamSynchronize(s));
    AOT_TRY(read_device_error(g, s));
  }
  *h_written = k;
  *h_next = cursor + k;
  return AOT_OK;
}

// ---------------------------------------------------------------- autotuner
// Coordinate search over the launch tuning of one graph: each candidate is
// binned and timed (CUDA events, best of reps) on the graph itself in the
// requested mode; the fastest tuning is kept on the graph and returned.
namespace aot {
static aot_status time_mode(aot_graph* g, int mode, int reps, cudaStream_t s, float* ms_out) {
  cudaEvent_t a, b;
  AOT_CUDA(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return AOT_ERR_CUDA;
  }
  float best = 3.0e38f;
  aot_status st = AOT_OK;
  for (int r = 0; r < reps && st == AOT_OK; ++r) {
    st = reset_scalars(g, s);
    if (st == AOT_OK && mode == 1) st = cudaMemsetAsync(g->tv, 0, sizeof(uint64_t) * g->n, s) ? AOT_ERR_CUDA : AOT_OK;
    if (st != AOT_OK) break;
    cudaEventRecord(a, s);
    st = mode == 1 ? run_mode<M_VERTEX>(g, AOT_ROUTE_PLAIN, base_params(g), s)
                   : run_mode<M_COUNT>(g, AOT_ROUTE_PLAIN, base_params(g), s);
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) st = AOT_ERR_CUDA;
    float ms = 0.f;
    if (st == AOT_OK && cudaEventElapsedTime(&ms, a, b) == cudaSuccess && ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms_out = best;
  return st;
}
}  // namespace aot

extern "C" aot_status aot_tune(aot_graph* g, int32_t mode, int32_t reps, aot_tuning* best_out,
                               float* h_best_ms, aot_stream_t stream) {
  if (!g || mode < 0 || mode > 1 || reps < 1 || reps > 100) return AOT_ERR_INVALID_ARG;
  if (g->max_outdeg >= (1 << 27)) return AOT_ERR_OVERFLOW;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  aot_tuning cur;
  AOT_TRY(aot_graph_get_tuning(g, &cur));
  float best_ms = 0.f;
  if (g->m > 0) {
    AOT_TRY(time_mode(g, mode, reps, s, &best_ms));
    auto trial = [&](aot_tuning cand) -> aot_status {
      if (aot_graph_set_tuning(g, &cand, stream) != AOT_OK) return AOT_OK;  // skip invalid candidates
      float ms = 0.f;
      AOT_TRY(time_mode(g, mode, reps, s, &ms));
      if (ms < 0.99f * best_ms) {  // a candidate must win by 1 %: near ties keep the current tuning
        best_ms = ms;
        cur = cand;
      }
      return AOT_OK;
    };
    const uint32_t ctas[] = {64, 256, 512, 1024, 2048, 4096};
    for (uint32_t c : ctas) {
      aot_tuning t = cur;
      t.cta_max_outdeg = c;
      t.warp_max_outdeg = c < t.warp_max_outdeg ? c : t.warp_max_outdeg;
      AOT_TRY(trial(t));
    }
    const int threads[] = {32, 256, 512, 1024};  // 32: the CTA bin a warp per pivot
    for (int th : threads) {
      aot_tuning t = cur;
      t.cta_threads = th;
      AOT_TRY(trial(t));
    }
    const uint32_t warps[] = {16, 32, 64};
    for (uint32_t w : warps) {
      aot_tuning t = cur;
      t.warp_max_outdeg = w <= t.cta_max_outdeg ? w : t.cta_max_outdeg;
      AOT_TRY(trial(t));
    }
    const uint32_t longs[] = {64u, 128u, 256u, 512u};
    for (uint32_t sl : longs) {
      aot_tuning t = cur;
      t.seg_long = sl;
      AOT_TRY(trial(t));
    }
    const uint32_t wides[] = {256u, 512u, 1024u, 4096u};
    for (uint32_t sw : wides) {
      aot_tuning t = cur;
      t.seg_wide = sw;
      AOT_TRY(trial(t));
    }
    // segment width, the hashed tail pass and the later segments' per-thread
    // threshold interact: search them jointly
    // (1310720 ranks keep the kernel's shared memory within a 196 KB carveout,
    // leaving 60 KB of L1 for the walked lists)
    const uint32_t segs[] = {1310720u, 1048576u, 1572864u};
    const uint32_t hashes[] = {12288u, 0u};
    const uint32_t tails[] = {64u, 128u, 192u, 256u};
    for (uint32_t sh : hashes)
      for (uint32_t sb : segs)
        for (uint32_t st : tails) {
          aot_tuning t = cur;
          t.seg_bits = sb;
          t.seg_hash = sh;
          t.seg_tail = st;
          AOT_TRY(trial(t));
        }
    {  // two CTAs of 512 threads per SM need segments of at most 576 K ranks
      const uint32_t segs2[] = {524288u, 589824u};
      for (uint32_t sb : segs2) {
        aot_tuning t = cur;
        t.seg_threads = 512;
        t.seg_bits = sb;
        AOT_TRY(trial(t));
      }
    }
    const uint32_t tiles[] = {0u, 21u, 22u, 23u, 24u, 25u};
    for (uint32_t tb : tiles) {
      aot_tuning t = cur;
      t.tile_bits = tb;
      AOT_TRY(trial(t));
    }
    AOT_TRY(aot_graph_set_tuning(g, &cur, stream));
  }
  if (best_out) *best_out = cur;
  if (h_best_ms) *h_best_ms = best_ms;
  return AOT_OK;
}
