// aot_route.cu - routing of work items to intersection variants, and the
// two variants that need no pivot index.
//
// Every work item of Algorithm 3 (pivot p, walked range R of an out-list,
// walked vertex v) finds the same triangles whichever way the intersection
// N+(p) & R is computed, so a route can only change speed, never the output:
//   V_PROBE    the pivot-grouped index probe (aot_count.cu kernels)
//   V_MERGE    warp merge: R is cut into 32 parts, each lane merges its part
//              with N+(p) from a binary-searched start (merge path)
//   V_BSEARCH  every walked entry is binary-searched in N+(p)
// A route array holds one variant byte per item; rprobe[p] counts the probe
// items of each pivot (pivots with none skip index staging) and eplist holds
// (item, pivot) of every merge / binary-search item.
#include "aot_internal.cuh"
#include "aot_kparams.cuh"

namespace aot {

// -------------------------------------------------------------- route fill
// variant >= 0: every item takes it (only items whose hash has its low
// sample_log2 bits zero when sample_log2 > 0; the others are skipped);
// variant < 0: a random variant per item.  Hash: splitmix64 of (seed, item).
__global__ void k_route_fill(uint8_t* __restrict__ route, int64_t m, int variant, uint64_t seed,
                             int sample_log2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  uint8_t v = (uint8_t)variant;
  if (variant < 0) v = (uint8_t)(z % 3);
  else if (sample_log2 > 0 && (z & ((1ull << sample_log2) - 1)) != 0) v = V_SKIP;
  route[i] = v;
}

// warp per pivot: probe items per pivot; merge / bsearch items appended to eplist
__global__ void k_route_lists(const uint32_t* __restrict__ wofs, int32_t n,
                              const uint8_t* __restrict__ route, uint32_t* __restrict__ rprobe,
                              uint2* __restrict__ eplist, DevScalars* dev) {
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (p >= n) return;
  const unsigned lane = lane_id();
  const uint32_t b = wofs[p], e = wofs[p + 1];
  uint32_t probes = 0;
  for (uint32_t c = b; c < e; c += 32) {
    const uint32_t it = c + lane;
    const bool has = it < e;
    const uint8_t v = has ? route[it] : (uint8_t)V_PROBE;
    const bool ep = has && (v == V_MERGE || v == V_BSEARCH);
    probes += (uint32_t)__popc(__ballot_sync(FULL, has && v == V_PROBE));
    const unsigned em = __ballot_sync(FULL, ep);
    if (em) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(&dev->counters[Q_EPLIST], (uint32_t)__popc(em));
      base = __shfl_sync(FULL, base, 0);
      if (ep) eplist[base + __popc(em & lanemask_lt())] = make_uint2(it, (uint32_t)p);
    }
  }
  if (lane == 0) rprobe[p] = probes;
}

// ------------------------------------------------------- staging-free variants
__device__ __forceinline__ uint32_t lower_bound_g(const uint32_t* __restrict__ a, uint32_t lo,
                                                  uint32_t hi, uint32_t key) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(a + mid) < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <int MODE>
__device__ __forceinline__ void ep_hit(const KParams& P, uint32_t w) {
  if (MODE == M_VERTEX) atomicAdd((unsigned long long*)&P.tv[w], 1ull);
}

// warp per (item, pivot) of eplist; grid-stride over the list
template <int MODE>
__global__ void __launch_bounds__(256) k_items_ep(KParams P, const uint2* __restrict__ eplist,
                                                 const uint8_t* __restrict__ route) {
  const unsigned lane = lane_id();
  const uint32_t count = P.dev->counters[Q_EPLIST];
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  uint64_t found = 0;
  for (uint32_t li = gw; li < count; li += nwarps) {
    const long long t0 = MODE == M_TIMED ? clock64() : 0;
    const uint2 ent = eplist[li];
    const uint32_t it = ent.x, p = ent.y;
    const uint2 r = P.witem[it];
    uint32_t x = r.x;
    const uint32_t y = r.y;
    uint32_t vert = 0, edge = 0;
    uint64_t tb = 0;
    if (MODE != M_COUNT) vert = P.wvert[it];
    if (MODE >= M_LIST_COUNT) edge = P.wedge[it];  // list modes and M_TIMED
    if (MODE == M_LIST_WRITE) {
      const uint64_t a = P.toff[edge], b = P.toff[edge + 1];
      if (a == b || b <= P.cursor || a >= P.cursor + P.cap) continue;
      tb = a;
    }
    const uint32_t pb = P.off[p], pe = P.off[p + 1];
    const uint2 ends = MODE == M_LIST_WRITE ? emit_ends(P, p, vert) : make_uint2(0u, 0u);
    uint32_t h = 0;  // hits of this item (warp-uniform after reductions)
    if (x < y && pb < pe) {
      if (route[it] == V_BSEARCH) {
        // only the part of N+(p) between the first and last walked entry can match
        const uint32_t lo = lower_bound_g(P.adj, pb, pe, __ldg(P.adj + x));
        for (uint32_t k0 = x; k0 < y; k0 += 32) {
          const uint32_t k = k0 + lane;
          bool hit = false;
          uint32_t w = 0;
          if (k < y) {
            w = __ldg(P.adj + k);
            const uint32_t pos = lower_bound_g(P.adj, lo, pe, w);
            hit = pos < pe && __ldg(P.adj + pos) == w;
          }
          const unsigned hm = __ballot_sync(FULL, hit);
          if (hit) {
            ep_hit<MODE>(P, w);
            if (MODE == M_LIST_WRITE) emit(P, tb + h + (uint32_t)__popc(hm & lanemask_lt()), ends, w);
          }
          h += (uint32_t)__popc(hm);
        }
      } else {
        // merge path: lane L merges its part of R with N+(p)
        const uint32_t len = y - x;
        const uint32_t part = (len + 31) / 32;
        const uint32_t a0 = x + min(len, lane * part), a1 = x + min(len, (lane + 1) * part);
        uint32_t c = 0;
        if (a0 < a1) {
          uint32_t bpos = lower_bound_g(P.adj, pb, pe, __ldg(P.adj + a0));
          for (uint32_t a = a0; a < a1 && bpos < pe; ++a) {
            const uint32_t av = __ldg(P.adj + a);
            uint32_t bv = __ldg(P.adj + bpos);
            while (bv < av && ++bpos < pe) bv = __ldg(P.adj + bpos);
            if (bpos < pe && bv == av) {
              ++c;
              if (MODE != M_LIST_WRITE) ep_hit<MODE>(P, av);
            }
          }
        }
        const uint32_t incl = warp_inclusive_scan(c);
        if (MODE == M_LIST_WRITE && c) {  // second pass: write in order
          uint64_t idx = tb + (incl - c);
          uint32_t bpos = lower_bound_g(P.adj, pb, pe, __ldg(P.adj + a0));
          for (uint32_t a = a0; a < a1 && bpos < pe; ++a) {
            const uint32_t av = __ldg(P.adj + a);
            uint32_t bv = __ldg(P.adj + bpos);
            while (bv < av && ++bpos < pe) bv = __ldg(P.adj + bpos);
            if (bpos < pe && bv == av) emit(P, idx++, ends, av);
          }
        }
        h = __shfl_sync(FULL, incl, 31);
      }
    }
    if (lane == 0) {
      found += h;
      if (MODE == M_VERTEX && h) {
        atomicAdd((unsigned long long*)&P.tv[vert], (unsigned long long)h);
        atomicAdd((unsigned long long*)&P.tv[p], (unsigned long long)h);
      }
      if (MODE == M_LIST_COUNT) P.tcnt[edge] = h;
      if (MODE == M_TIMED) P.cyc[edge] = sat_cycles(clock64() - t0);
    }
  }
  if (lane == 0 && found) atomicAdd(&P.dev->total, (unsigned long long)found);
}

// ------------------------------------------------------------------ driver
#define AOT_EP_NAMES {"k_items_ep/count", "k_items_ep/vertex", "k_items_ep/list_count", "k_items_ep/list_write", "k_items_ep/timed"}
static const char* const kEpNames[5] = AOT_EP_NAMES;

aot_status route_items(aot_graph* g, aot_route route, cudaStream_t s, int sample_log2) {
  g->routed = false;
  if (route == AOT_ROUTE_PLAIN || route == AOT_ROUTE_PROBE) return AOT_OK;
  if (g->m == 0) return AOT_OK;
  const int T = 256;
  const unsigned grid_m = (unsigned)((g->m + T - 1) / T);
  if (route == AOT_ROUTE_LEARNED) {
    AOT_TRY(learned_routes(g, s));
  } else {
    const int variant = route == AOT_ROUTE_MERGE ? V_MERGE
                        : route == AOT_ROUTE_BSEARCH ? V_BSEARCH : -1;
    AOT_KERNEL("k_route_fill", s)
      k_route_fill<<<grid_m, T, 0, s>>>(g->route, g->m, variant, 0x5EED5EEDull, sample_log2);
    AOT_TRY(last_launch());
  }
  AOT_CUDA(cudaMemsetAsync(&g->dev->counters[Q_EPLIST], 0, sizeof(unsigned int), s));
  AOT_KERNEL("k_route_lists", s)
    k_route_lists<<<(unsigned)(((int64_t)g->n * 32 + T - 1) / T), T, 0, s>>>(
        g->wofs, g->n, g->route, g->rprobe, g->eplist, g->dev);
  AOT_TRY(last_launch());
  g->routed = true;
  return AOT_OK;
}

template <int MODE>
aot_status launch_ep(aot_graph* g, const KParams& P, cudaStream_t s) {
  if (!g->routed) return AOT_OK;
  int dev = 0, sms = 1, per_sm = 1;
  AOT_CUDA(cudaGetDevice(&dev));
  AOT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  AOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_items_ep<MODE>, 256, 0));
  AOT_KERNEL(kEpNames[MODE], s)
    k_items_ep<MODE><<<(unsigned)(sms * (per_sm > 0 ? per_sm : 1)), 256, 0, s>>>(P, g->eplist, g->route);
  return last_launch();
}

template aot_status launch_ep<M_COUNT>(aot_graph*, const KParams&, cudaStream_t);
template aot_status launch_ep<M_VERTEX>(aot_graph*, const KParams&, cudaStream_t);
template aot_status launch_ep<M_LIST_COUNT>(aot_graph*, const KParams&, cudaStream_t);
template aot_status launch_ep<M_LIST_WRITE>(aot_graph*, const KParams&, cudaStream_t);
template aot_status launch_ep<M_TIMED>(aot_graph*, const KParams&, cudaStream_t);

}  // namespace aot
