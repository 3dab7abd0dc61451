// aot_kparams.cuh - parameters shared by the intersection kernels of
// aot_count.cu (pivot-index probes) and aot_route.cu (staging-free variants).
#pragma once
#include "aot_internal.cuh"

namespace aot {

// M_TIMED counts like M_COUNT and also records per-edge cycles into cyc[]
enum Mode { M_COUNT = 0, M_VERTEX = 1, M_LIST_COUNT = 2, M_LIST_WRITE = 3, M_TIMED = 4 };
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
  uint32_t* cyc;           // M_TIMED: cycles per oriented edge
  const uint32_t* rprobe;  // probe items per pivot (nullptr: all items)
  const uint64_t* lblk;    // listing: output range per block of LIST_BLOCK items (nullptr: none)
};

// Work items per listing block: lblk[2 b] and lblk[2 b + 1] are the smallest
// first and the largest end triangle number of the items
// [b LIST_BLOCK, (b + 1) LIST_BLOCK) that have a triangle ([2^64 - 1, 0) when
// none has).  Items are stored pivot by pivot in rank order, a pivot's
// positive items in out-list order, so a block's range is narrow.
constexpr uint32_t LIST_BLOCK = 1536;

// Can any item of [i0, i1) write a triangle of the listing window?  (Always
// true without block ranges; a conservative test otherwise.)
__device__ __forceinline__ bool list_window_overlaps(const KParams& P, uint32_t i0, uint32_t i1) {
  if (!P.lblk) return true;
  if (i0 >= i1) return false;
  const uint64_t w0 = P.cursor, w1 = P.cursor + P.cap;
  for (uint32_t b = i0 / LIST_BLOCK; b <= (i1 - 1) / LIST_BLOCK; ++b)
    if (P.lblk[2 * (size_t)b + 1] > w0 && P.lblk[2 * (size_t)b] < w1) return true;
  return false;
}

// Listing output: triangle number idx, if it falls in the window, as
// (x, y, w) in original ids with eta(x) < eta(y) < eta(w).  (x, y) are the
// item's pivot and walked vertex, the same for all its triangles:
// emit_ends gives them once per item.
__device__ __forceinline__ uint2 emit_ends(const KParams& P, uint32_t p, uint32_t v) {
  return make_uint2((uint32_t)P.perm[p < v ? p : v], (uint32_t)P.perm[p < v ? v : p]);
}
__device__ __forceinline__ void emit(const KParams& P, uint64_t idx, uint2 ends, uint32_t w) {
  if (idx >= P.cursor && idx < P.cursor + P.cap) {
    int32_t* o = P.out + 3 * (idx - P.cursor);
    o[0] = (int32_t)ends.x;
    o[1] = (int32_t)ends.y;
    o[2] = P.perm[w];
  }
}

__device__ __forceinline__ uint32_t sat_cycles(long long c) {
  return c <= 0 ? 0u : (c >= 0xffffffffll ? 0xffffffffu : (uint32_t)c);
}

template <int MODE>
aot_status launch_ep(aot_graph* g, const KParams& P, cudaStream_t s);
aot_status route_items(aot_graph* g, aot_route route, cudaStream_t s, int sample_log2 = 0);

}  // namespace aot
