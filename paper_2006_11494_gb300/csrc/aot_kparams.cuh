// aot_kparams.cuh - parameters shared by the intersection kernels of
// aot_count.cu (pivot-index probes) and aot_route.cu (staging-free variants).
#pragma once
#include "aot_internal.cuh"

namespace aot {

enum Mode { M_COUNT = 0, M_VERTEX = 1, M_LIST_COUNT = 2, M_LIST_WRITE = 3 };
enum Queue { Q_WARP = 1, Q_CTA = 2, Q_HUB = 3, Q_SEG = 4, Q_EPLIST = 5 };

struct KParams {
  const uint32_t* off;
  const uint32_t* adj;
  const uint32_t* wofs;
  const uint2* witem;
  const uint32_t* wvert;
  const uint32_t* wedge;
  const uint32_t* pivots;  // this bin's pivots
  uint32_t num_pivots;
  uint64_t* tv;            // per-vertex counts (rank space)
  uint32_t* tcnt;          // triangles per oriented edge
  const uint64_t* toff;    // exclusive offsets per oriented edge
  const int32_t* perm;
  int32_t* out;
  uint64_t cursor, cap;    // listing window [cursor, cursor + cap)
  DevScalars* dev;
  const uint8_t* route;    // variant per item (nullptr: every item probes)
  const uint32_t* rprobe;  // probe items per pivot (nullptr: all items)
};

// Listing output: triangle number idx, if it falls in the window, as
// (x, y, w) in original ids with eta(x) < eta(y) < eta(w).
__device__ __forceinline__ void emit(const KParams& P, uint64_t idx, uint32_t p, uint32_t v,
                                     uint32_t w) {
  if (idx >= P.cursor && idx < P.cursor + P.cap) {
    int32_t* o = P.out + 3 * (idx - P.cursor);
    o[0] = P.perm[p < v ? p : v];
    o[1] = P.perm[p < v ? v : p];
    o[2] = P.perm[w];
  }
}

template <int MODE>
aot_status launch_ep(aot_graph* g, const KParams& P, cudaStream_t s);
aot_status route_items(aot_graph* g, aot_route route, cudaStream_t s);

}  // namespace aot
