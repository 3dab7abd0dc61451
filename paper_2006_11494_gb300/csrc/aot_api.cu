// aot_api.cu - small C-ABI entry points: status strings, graph facts, export,
// destroy.  The heavy entry points live next to their kernels.
#include "aot_internal.cuh"

#include <map>
#include <mutex>
#include <utility>

using namespace aot;

namespace aot {
static std::mutex g_attr_mu;
static std::map<std::pair<int, const void*>, size_t> g_attr_set;  // (device, kernel) -> bytes
static std::map<int, int> g_sms;                                    // device -> SM count

aot_status ensure_dyn_smem(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return AOT_OK;  // the default limit
  int dev = 0;
  AOT_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_attr_mu);
  size_t& cur = g_attr_set[std::make_pair(dev, func)];
  if (cur >= bytes) return AOT_OK;
  AOT_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
  return AOT_OK;
}

static std::map<std::pair<int, const void*>, bool> g_carveout;  // (device, kernel) set

aot_status prefer_max_smem(const void* func) {
  int dev = 0;
  AOT_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_attr_mu);
  bool& done = g_carveout[std::make_pair(dev, func)];
  if (done) return AOT_OK;
  AOT_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared));
  done = true;
  return AOT_OK;
}

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  int& sms = g_sms[dev];
  if (sms <= 0) {
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  }
  return sms;
}

static std::mutex g_default_mu;
static Tuning g_default_tuning;
static const void* g_default_router = nullptr;
const void* default_router() {
  std::lock_guard<std::mutex> lk(g_default_mu);
  return g_default_router;
}
Tuning default_tuning() {
  std::lock_guard<std::mutex> lk(g_default_mu);
  return g_default_tuning;
}
static bool tuning_valid(const aot_tuning* t) {
  return !(t->warp_max_outdeg > 64 || t->cta_max_outdeg > 8192 ||
           t->cta_max_outdeg < t->warp_max_outdeg || t->cta_threads < 32 || t->cta_threads > 1024 ||
           (t->cta_threads & 31) || t->hub_bitmaps < 1 || t->hub_bitmaps > Tuning().hub_bitmaps ||
           t->hub_mode < 0 || t->hub_mode > 1 || t->seg_bits < 1024 || t->seg_bits > 1536u * 1024u ||
           (t->seg_bits & 31) || t->seg_long > (1u << 30) || t->seg_wide > (1u << 30) ||
           (t->tile_bits != 0 && (t->tile_bits < 16 || t->tile_bits > 31)) || t->seg_tail > (1u << 30) ||
           t->seg_threads < 256 || t->seg_threads > 1024 || (t->seg_threads & 31) ||
           t->seg_hash > (1u << 30));
}
}  // namespace aot

extern "C" aot_status aot_set_default_tuning(const aot_tuning* t) {
  if (!t || !tuning_valid(t)) return AOT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_default_mu);
  g_default_tuning.warp_max_outdeg = t->warp_max_outdeg;
  g_default_tuning.cta_max_outdeg = t->cta_max_outdeg;
  g_default_tuning.cta_threads = t->cta_threads;
  g_default_tuning.hub_bitmaps = t->hub_bitmaps;
  g_default_tuning.hub_mode = t->hub_mode;
  g_default_tuning.seg_bits = t->seg_bits;
  g_default_tuning.seg_long = t->seg_long;
  g_default_tuning.seg_wide = t->seg_wide;
  g_default_tuning.tile_bits = t->tile_bits;
  g_default_tuning.seg_tail = t->seg_tail;
  g_default_tuning.seg_threads = t->seg_threads;
  g_default_tuning.seg_hash = t->seg_hash;
  return AOT_OK;
}

extern "C" aot_status aot_set_default_router(const void* d_model) {
  if (d_model && (reinterpret_cast<uintptr_t>(d_model) & 15)) return AOT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_default_mu);
  g_default_router = d_model;
  return AOT_OK;
}

extern "C" aot_status aot_get_default_tuning(aot_tuning* t) {
  if (!t) return AOT_ERR_INVALID_ARG;
  Tuning d = default_tuning();
  t->warp_max_outdeg = d.warp_max_outdeg;
  t->cta_max_outdeg = d.cta_max_outdeg;
  t->cta_threads = d.cta_threads;
  t->hub_bitmaps = d.hub_bitmaps;
  t->hub_mode = d.hub_mode;
  t->seg_bits = d.seg_bits;
  t->seg_long = d.seg_long;
  t->seg_wide = d.seg_wide;
  t->tile_bits = d.tile_bits;
  t->seg_tail = d.seg_tail;
  t->seg_threads = d.seg_threads;
  t->seg_hash = d.seg_hash;
  return AOT_OK;
}

extern "C" const char* aot_status_string(aot_status st) {
  switch (st) {
    case AOT_OK: return "ok";
    case AOT_ERR_INVALID_ARG: return "invalid argument";
    case AOT_ERR_VERTEX_RANGE: return "vertex id outside [0, n)";
    case AOT_ERR_OVERFLOW: return "size exceeds the supported index range";
    case AOT_ERR_WORKSPACE: return "workspace too small or misaligned";
    case AOT_ERR_CUDA: return "CUDA runtime error";
    case AOT_ERR_TIMEOUT: return "bounded device wait timed out";
    case AOT_ERR_DEVICE_CHECK: return "device consistency check failed";
    case AOT_ERR_NOT_READY: return "not ready (missing router weights or unsupported route)";
  }
  return "unknown status";
}

extern "C" int aot_version(void) { return 100; }

extern "C" aot_status aot_graph_info(const aot_graph* g, int32_t* n, int64_t* m, uint64_t* work_w,
                                     uint64_t* staged_s, int32_t* max_outdeg) {
  if (!g) return AOT_ERR_INVALID_ARG;
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (work_w) *work_w = g->W;
  if (staged_s) *staged_s = g->S;
  if (max_outdeg) *max_outdeg = g->max_outdeg;
  return AOT_OK;
}

extern "C" aot_status aot_graph_costs(const aot_graph* g, aot_costs* out) {
  if (!g || !out) return AOT_ERR_INVALID_ARG;
  out->walk = g->W;
  out->merge = g->merge_work;
  out->staged = g->S;
  out->positive = g->positive;
  out->items = (uint64_t)g->m;
  return AOT_OK;
}

extern "C" aot_status aot_graph_export(const aot_graph* g, int32_t* d_perm, int32_t* d_rank,
                                       uint32_t* d_out_off, uint32_t* d_out_adj, uint32_t* d_items,
                                       uint64_t* d_walk, aot_stream_t stream) {
  if (!g) return AOT_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t n = (size_t)g->n, m = (size_t)g->m;
  auto cp = [&](void* dst, const void* src, size_t bytes) -> aot_status {
    if (dst && bytes) AOT_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
    return AOT_OK;
  };
  AOT_TRY(cp(d_perm, g->perm, n * sizeof(int32_t)));
  AOT_TRY(cp(d_rank, g->rank, n * sizeof(int32_t)));
  AOT_TRY(cp(d_out_off, g->off, (n + 1) * sizeof(uint32_t)));
  AOT_TRY(cp(d_out_adj, g->adj, m * sizeof(uint32_t)));
  AOT_TRY(cp(d_items, g->items, n * sizeof(uint32_t)));
  AOT_TRY(cp(d_walk, g->walk, n * sizeof(uint64_t)));
  return AOT_OK;
}

extern "C" aot_status aot_graph_bins(const aot_graph* g, aot_bin_stats out[3]) {
  if (!g || !out) return AOT_ERR_INVALID_ARG;
  for (int b = 0; b < NUM_BINS; ++b) {
    out[b].pivots = g->bin_stats[b][0];
    out[b].items = g->bin_stats[b][1];
    out[b].walk = g->bin_stats[b][2];
    out[b].staged = g->bin_stats[b][3];
  }
  return AOT_OK;
}

extern "C" aot_status aot_graph_get_tuning(const aot_graph* g, aot_tuning* t) {
  if (!g || !t) return AOT_ERR_INVALID_ARG;
  t->warp_max_outdeg = g->tune.warp_max_outdeg;
  t->cta_max_outdeg = g->tune.cta_max_outdeg;
  t->cta_threads = g->tune.cta_threads;
  t->hub_bitmaps = g->tune.hub_bitmaps;
  t->hub_mode = g->tune.hub_mode;
  t->seg_bits = g->tune.seg_bits;
  t->seg_long = g->tune.seg_long;
  t->seg_wide = g->tune.seg_wide;
  t->tile_bits = g->tune.tile_bits;
  t->seg_tail = g->tune.seg_tail;
  t->seg_threads = g->tune.seg_threads;
  t->seg_hash = g->tune.seg_hash;
  return AOT_OK;
}

extern "C" aot_status aot_graph_set_tuning(aot_graph* g, const aot_tuning* t, aot_stream_t stream) {
  if (!g || !t || !tuning_valid(t)) return AOT_ERR_INVALID_ARG;
  Tuning old = g->tune;
  g->tune.warp_max_outdeg = t->warp_max_outdeg;
  g->tune.cta_max_outdeg = t->cta_max_outdeg;
  g->tune.cta_threads = t->cta_threads;
  g->tune.hub_bitmaps = t->hub_bitmaps;
  g->tune.hub_mode = t->hub_mode;
  g->tune.seg_bits = t->seg_bits;
  g->tune.seg_long = t->seg_long;
  g->tune.seg_wide = t->seg_wide;
  g->tune.tile_bits = t->tile_bits;
  g->tune.seg_tail = t->seg_tail;
  g->tune.seg_threads = t->seg_threads;
  g->tune.seg_hash = t->seg_hash;
  aot_status st = bin_pivots(g, reinterpret_cast<cudaStream_t>(stream));
  if (st != AOT_OK) g->tune = old;
  return st;
}

extern "C" aot_status aot_graph_destroy(aot_graph* g) {
  delete g;
  return AOT_OK;
}
