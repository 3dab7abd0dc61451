// aot_batch.cu - thousands of small graphs in one pass.
//
// The batch is processed as the disjoint union of its graphs: vertex v of
// graph g becomes voff[g] + v, where voff is the exclusive prefix of the
// vertex counts.  No edge joins two graphs, so every triangle of the union
// lies in one graph, the union's per-vertex counts are the graphs' per-vertex
// counts laid end to end, and T_g = (sum of t(v) over graph g) / 3.  One
// orientation covers the whole batch (its radix sorts see all graphs at
// once), and the counting phase -- the persistent bin kernels with their
// atomic work queues and the per-graph totals -- is captured into a CUDA
// graph and launched once.  Each host thread keeps its last instantiated
// graph per device and updates it in place (cudaGraphExecUpdate) when the
// next batch captures the same sequence of kernels, so repeated calls of one
// shape pay no instantiation.
#include <map>

#include "aot_internal.cuh"

namespace aot {

__global__ void k_batch_ids(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            int64_t E, const int64_t* __restrict__ edge_ofs, int32_t G,
                            const int32_t* __restrict__ nv, const uint32_t* __restrict__ voff,
                            int32_t* __restrict__ gsrc, int32_t* __restrict__ gdst,
                            uint32_t* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  int32_t lo = 0, hi = G;  // graph g with edge_ofs[g] <= i < edge_ofs[g + 1]
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (edge_ofs[mid] <= i) lo = mid;
    else hi = mid;
  }
  const int32_t a = src[i], b = dst[i], n = nv[lo];
  if (a < 0 || a >= n || b < 0 || b >= n) {  // an id outside its own graph
    gsrc[i] = -1;
    gdst[i] = -1;
    atomicOr(err, DEVERR_RANGE);
    return;
  }
  gsrc[i] = (int32_t)(voff[lo] + (uint32_t)a);
  gdst[i] = (int32_t)(voff[lo] + (uint32_t)b);
}

__global__ void k_batch_check(const int64_t* __restrict__ edge_ofs, int32_t G, int64_t E,
                              const int32_t* __restrict__ nv, const uint32_t* __restrict__ voff,
                              int64_t N, uint32_t* __restrict__ err) {
  const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g > G) return;
  if (g == 0 && (edge_ofs[0] != 0 || edge_ofs[G] != E || (int64_t)voff[G] != N)) atomicOr(err, DEVERR_CHECK);
  if (g < G && (edge_ofs[g + 1] < edge_ofs[g] || nv[g] < 0)) atomicOr(err, DEVERR_CHECK);
}

// warp per graph: T_g = sum of its per-vertex counts / 3
__global__ void k_batch_totals(const uint64_t* __restrict__ vcount, const uint32_t* __restrict__ voff,
                               int32_t G, uint64_t* __restrict__ tri) {
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (g >= G) return;
  uint64_t s = 0;
  for (uint32_t v = voff[g] + lane_id(); v < voff[g + 1]; v += 32) s += vcount[v];
  s = warp_sum(s);
  if (lane_id() == 0) tri[g] = s / 3;
}

struct BatchLayout {
  uint32_t* voff;
  uint32_t* err;
  void* scan_tmp;
  int32_t* gsrc;
  int32_t* gdst;
  void* orient_ws;
  size_t orient_bytes;
  size_t bytes;
};

static aot_status carve_batch(void* base, int64_t E, int32_t G, int64_t N, BatchLayout* L) {
  Carve c(base);
  L->voff = c.take<uint32_t>((size_t)G + 1);
  L->err = c.take<uint32_t>(1);
  L->scan_tmp = c.take<char>(scan_tmp_bytes((int64_t)G + 1));
  L->gsrc = c.take<int32_t>(E > 0 ? E : 1);
  L->gdst = c.take<int32_t>(E > 0 ? E : 1);
  size_t ob = 0;
  AOT_TRY(aot_orient_workspace_size(E, (int32_t)N, AOT_FLAG_NO_LIST, &ob));
  L->orient_bytes = ob;
  L->orient_ws = c.take<char>(ob);
  L->bytes = c.used();
  return AOT_OK;
}

// The calling thread's instantiated counting graph on each device.
struct ExecCache {
  std::map<int, cudaGraphExec_t> exec;
  ~ExecCache() {
    for (auto& kv : exec) cudaGraphExecDestroy(kv.second);
  }
};
static thread_local ExecCache t_exec;

// Launch a captured graph through the thread's cached executable (updated in
// place when the kernels match, else re-instantiated).
static aot_status launch_captured(cudaGraph_t graph, cudaStream_t s) {
  int dev = 0;
  AOT_CUDA(cudaGetDevice(&dev));
  cudaGraphExec_t& ex = t_exec.exec[dev];
  if (ex) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(ex, graph, &info) != cudaSuccess) {
      cudaGetLastError();  // an update that does not fit is not an error: re-instantiate
      cudaGraphExecDestroy(ex);
      ex = nullptr;
    }
  }
  if (!ex && cudaGraphInstantiate(&ex, graph, 0) != cudaSuccess) {
    ex = nullptr;
    return AOT_ERR_CUDA;
  }
  AOT_CUDA(cudaGraphLaunch(ex, s));
  return AOT_OK;
}

// Union graph of a batch, oriented (shared by aot_batch and aot_batch_tune).
static aot_status batch_union(const int32_t* d_src, const int32_t* d_dst, const int64_t* d_edge_ofs,
                              const int32_t* d_nv, int32_t G, int64_t E, int64_t N, const BatchLayout& L,
                              cudaStream_t s, aot_graph** out) {
  const int T = 256;
  AOT_CUDA(cudaMemsetAsync(L.err, 0, sizeof(uint32_t), s));
  AOT_TRY(scan_u32_u32(reinterpret_cast<const uint32_t*>(d_nv), L.voff, G, L.scan_tmp, s));
  AOT_KERNEL("k_batch_check", s)
    k_batch_check<<<(unsigned)((G + 1 + T - 1) / T), T, 0, s>>>(d_edge_ofs, G, E, d_nv, L.voff, N, L.err);
  AOT_TRY(last_launch());
  uint32_t herr = 0;
  AOT_CUDA(cudaMemcpyAsync(&herr, L.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  AOT_CUDA(cudaStreamSynchronize(s));
  if (herr) return AOT_ERR_INVALID_ARG;
  if (E > 0) {
    AOT_KERNEL("k_batch_ids", s)
      k_batch_ids<<<(unsigned)((E + T - 1) / T), T, 0, s>>>(d_src, d_dst, E, d_edge_ofs, G, d_nv,
                                                           L.voff, L.gsrc, L.gdst, L.err);
    AOT_TRY(last_launch());
  }
  // one orientation of the union graph (synchronises s)
  aot_graph* g = nullptr;
  AOT_TRY(aot_orient(L.gsrc, L.gdst, E, (int32_t)N, AOT_FLAG_NO_LIST, L.orient_ws, L.orient_bytes,
                     reinterpret_cast<aot_stream_t>(s), &g));
  if (g->tune.hub_mode != 0) {  // the global-bitmap hub path reads hub descriptors on the host
    aot_tuning t;
    aot_graph_get_tuning(g, &t);
    t.hub_mode = 0;
    aot_status st = aot_graph_set_tuning(g, &t, reinterpret_cast<aot_stream_t>(s));
    if (st != AOT_OK) {
      aot_graph_destroy(g);
      return st;
    }
  }
  *out = g;
  return AOT_OK;
}

static aot_status batch_args(const int32_t* d_src, const int32_t* d_dst, const int64_t* d_edge_ofs,
                             const int32_t* d_nv, int32_t G, int64_t E, int64_t N, void* d_ws,
                             size_t ws_bytes, BatchLayout* L) {
  if (G < 0 || E < 0 || N < 0) return AOT_ERR_INVALID_ARG;
  if (!d_edge_ofs || !d_nv || (E > 0 && (!d_src || !d_dst))) return AOT_ERR_INVALID_ARG;
  if (N >= (int64_t(1) << 31)) return AOT_ERR_OVERFLOW;
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255)) return AOT_ERR_WORKSPACE;
  AOT_TRY(carve_batch(d_ws, E, G, N, L));
  if (ws_bytes < L->bytes) return AOT_ERR_WORKSPACE;
  return AOT_OK;
}

}  // namespace aot

using namespace aot;

extern "C" aot_status aot_batch_workspace_size(int64_t total_edges, int32_t num_graphs,
                                               int64_t total_vertices, size_t* bytes) {
  if (!bytes || total_edges < 0 || num_graphs < 0 || total_vertices < 0) return AOT_ERR_INVALID_ARG;
  if (total_vertices >= (int64_t(1) << 31)) return AOT_ERR_OVERFLOW;
  BatchLayout L;
  AOT_TRY(carve_batch(nullptr, total_edges, num_graphs, total_vertices, &L));
  *bytes = L.bytes;
  return AOT_OK;
}

extern "C" aot_status aot_batch(const int32_t* d_src, const int32_t* d_dst, const int64_t* d_edge_ofs,
                                const int32_t* d_nv, int32_t num_graphs, int64_t total_edges,
                                int64_t total_vertices, aot_route route, uint64_t* d_tri,
                                uint64_t* d_vcount, void* d_ws, size_t ws_bytes, aot_stream_t stream) {
  if (num_graphs < 0 || total_edges < 0 || total_vertices < 0) return AOT_ERR_INVALID_ARG;
  if (num_graphs == 0) return AOT_OK;
  if (!d_tri || (total_vertices > 0 && !d_vcount)) return AOT_ERR_INVALID_ARG;
  BatchLayout L;
  AOT_TRY(batch_args(d_src, d_dst, d_edge_ofs, d_nv, num_graphs, total_edges, total_vertices, d_ws,
                     ws_bytes, &L));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int T = 256;
  const int32_t G = num_graphs;
  const int64_t N = total_vertices;
  aot_graph* g = nullptr;
  AOT_TRY(batch_union(d_src, d_dst, d_edge_ofs, d_nv, G, total_edges, N, L, s, &g));
  // counting phase, captured into a CUDA graph when the stream allows it
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capture = s != nullptr && cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
                       cs == cudaStreamCaptureStatusNone;
  aot_status st = AOT_OK;
  cudaGraph_t graph = nullptr;
  if (capture && cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = AOT_ERR_CUDA;
  if (st == AOT_OK && N > 0) st = aot_count_per_vertex(g, route, d_vcount, nullptr, stream);
  if (st == AOT_OK) {
    AOT_KERNEL("k_batch_totals", s)
      k_batch_totals<<<(unsigned)(((int64_t)G * 32 + T - 1) / T), T, 0, s>>>(d_vcount, L.voff, G, d_tri);
    st = last_launch();
  }
  if (capture) {
    const cudaError_t ec = cudaStreamEndCapture(s, &graph);
    if (st == AOT_OK && ec != cudaSuccess) st = AOT_ERR_CUDA;
    if (st == AOT_OK) st = launch_captured(graph, s);
    if (graph) cudaGraphDestroy(graph);
  }
  if (st == AOT_OK && cudaStreamSynchronize(s) != cudaSuccess) st = AOT_ERR_CUDA;
  if (st == AOT_OK) st = read_device_error(g, s);
  aot_graph_destroy(g);
  return st;
}

extern "C" aot_status aot_batch_tune(const int32_t* d_src, const int32_t* d_dst, const int64_t* d_edge_ofs,
                                     const int32_t* d_nv, int32_t num_graphs, int64_t total_edges,
                                     int64_t total_vertices, int32_t reps, aot_tuning* best_out,
                                     float* h_best_ms, void* d_ws, size_t ws_bytes, aot_stream_t stream) {
  if (num_graphs <= 0 || !best_out) return AOT_ERR_INVALID_ARG;
  BatchLayout L;
  AOT_TRY(batch_args(d_src, d_dst, d_edge_ofs, d_nv, num_graphs, total_edges, total_vertices, d_ws,
                     ws_bytes, &L));
  aot_graph* g = nullptr;
  AOT_TRY(batch_union(d_src, d_dst, d_edge_ofs, d_nv, num_graphs, total_edges, total_vertices, L,
                      reinterpret_cast<cudaStream_t>(stream), &g));
  aot_status st = aot_tune(g, 1, reps, best_out, h_best_ms, stream);
  if (st == AOT_OK) best_out->hub_mode = 0;  // batches keep the hubs on the segmented bitmap
  aot_graph_destroy(g);
  return st;
}
