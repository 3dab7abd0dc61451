// aot_static.cu - per-vertex triangle counting for callers that cannot
// allocate device memory.
//
// The regular entry points take a caller-owned device workspace.  Some callers
// cannot provide one: code that runs where cudaMalloc is not allowed (inside
// an allocator hook, under a strict memory budget owned by someone else, or in
// a host framework that hands out only its own input and output buffers).
// aot_count_per_vertex_static serves them: its scratch memory is one
// file-scope __device__ array of AOT_STATIC_SCRATCH_BYTES, compiled into this
// library, so the call itself allocates no device memory.
//
//  - Every GPU that loads libaot.so holds this array until the process exits.
//  - Host code may not use the array's symbol as a device address.  The first
//    call on each device (with that device current) asks the runtime for the
//    array's device address with cudaGetSymbolAddress and caches it; make that
//    first call outside any stream capture.
//  - The cached address belongs to the device's current context: after
//    cudaDeviceReset it is stale, so a process that resets a device must not
//    call this entry point on that device again.
//  - All calls share the one array and it keeps the previous call's contents;
//    the orientation clears every part that must start at zero.  Two calls
//    whose work overlaps on the GPU (different streams or host threads) race
//    on the array: serialise them.  A call that fails after it has queued
//    kernels waits for them before it returns, so a retry on another stream
//    never overlaps them.
#include <mutex>

#include "aot_internal.cuh"

static __device__ __align__(256) unsigned char g_aot_static_scratch[AOT_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};
}  // namespace

extern "C" aot_status aot_count_per_vertex_static(const int32_t* d_src, const int32_t* d_dst,
                                                  int64_t num_edges, int32_t num_vertices,
                                                  uint64_t* d_counts, uint64_t* h_total,
                                                  aot_stream_t stream) {
  if (num_edges < 0 || num_vertices < 0 || !h_total) return AOT_ERR_INVALID_ARG;
  size_t need = 0;
  aot_status st = aot_orient_workspace_size(num_edges, num_vertices, AOT_FLAG_NO_LIST, &need);
  if (st != AOT_OK) return st;
  if (need > (size_t)AOT_STATIC_SCRATCH_BYTES) return AOT_ERR_OVERFLOW;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AOT_ERR_CUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_aot_static_scratch) != cudaSuccess || !p) return AOT_ERR_CUDA;
      g_static_ptr[dev] = p;
    }
    scratch = g_static_ptr[dev];
  }
  aot_graph* g = nullptr;
  st = aot_orient(d_src, d_dst, num_edges, num_vertices, AOT_FLAG_NO_LIST, scratch,
                  (size_t)AOT_STATIC_SCRATCH_BYTES, stream, &g);
  if (st == AOT_OK) {
    if (d_counts) {
      st = aot_count_per_vertex(g, AOT_ROUTE_PLAIN, d_counts, h_total, stream);
    } else {
      st = aot_count(g, AOT_ROUTE_PLAIN, h_total, stream);
    }
    aot_graph_destroy(g);
  }
  // kernels queued before a failure still use the shared array: let them finish
  if (st != AOT_OK) cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  return st;
}
