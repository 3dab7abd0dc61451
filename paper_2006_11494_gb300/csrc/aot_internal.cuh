// aot_internal.cuh - internal declarations shared by the libaot translation
// units: status plumbing, workspace carving, warp helpers, the graph handle.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <stdint.h>
#include <stddef.h>

#include "../../include/aot.h"

namespace aot {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t EMPTY = 0xffffffffu;  // empty hash slot (no vertex has this rank)

// Device error word bits (or-ed by kernels, read back by the API).
constexpr uint32_t DEVERR_RANGE = 1u;    // input id outside [0, n)
constexpr uint32_t DEVERR_CHECK = 2u;    // internal consistency check failed
constexpr uint32_t DEVERR_TIMEOUT = 4u;  // a bounded wait ran out

#define AOT_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return AOT_ERR_CUDA;         \
  } while (0)
#define AOT_TRY(call)                                   \
  do {                                                  \
    aot_status s_ = (call);                             \
    if (s_ != AOT_OK) return s_;                        \
  } while (0)

inline aot_status last_launch() {
  return cudaGetLastError() == cudaSuccess ? AOT_OK : AOT_ERR_CUDA;
}

// Raise the dynamic shared-memory limit of kernel `func` on the CURRENT device
// to at least `bytes`.  cudaFuncSetAttribute acts on one device only, so the
// largest value set so far is remembered per (device, kernel), under a mutex
// (calls may come from several host threads and devices).
aot_status ensure_dyn_smem(const void* func, size_t bytes);
// Ask for the largest shared-memory carveout for kernel `func` on the current
// device (once per device and kernel), so that several of its blocks fit.
aot_status prefer_max_smem(const void* func);
// Streaming multiprocessors of the current device (cached per device).
int sm_count();

// Launch accounting: AOT_KERNEL(name, stream) <launch statement>;
// counts the launch and, while profiling is on, brackets it with events.
struct ProfScope {
  bool once = true;
  int slot = -1;
  cudaStream_t s;
  ProfScope(const char* name, cudaStream_t st);
  ~ProfScope();
};
#define AOT_KERNEL(name, stream) for (aot::ProfScope ps_(name, stream); ps_.once; ps_.once = false)

// Bump allocator over a caller-owned device workspace.  With base == nullptr
// it only measures (used by the *_workspace_size queries).
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t used() const { return (off + 255) & ~size_t(255); }
};

inline int ceil_log2(uint64_t x) {  // smallest b with 2^b >= x (x >= 1)
  int b = 0;
  while ((uint64_t(1) << b) < x) ++b;
  return b;
}

// ------------------------------------------------------------ device helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
template <class T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T o = __shfl_up_sync(FULL, v, d);
    if ((int)lane_id() >= d) v += o;
  }
  return v;
}
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
  return v;
}
__device__ __forceinline__ uint32_t hash_slot(uint32_t w, uint32_t mask) {
  return (w * 2654435761u) & mask;  // Fibonacci-style multiplicative hash
}

// ------------------------------------------------------------ scan / sort
// Exclusive prefix sum: out[i] = sum in[0..i), out[N] = total.
size_t scan_tmp_bytes(int64_t N);
aot_status scan_u32_u32(const uint32_t* in, uint32_t* out, int64_t N, void* tmp, cudaStream_t s);
aot_status scan_u32_u64(const uint32_t* in, uint64_t* out, int64_t N, void* tmp, cudaStream_t s);
aot_status scan_u64_u64(const uint64_t* in, uint64_t* out, int64_t N, void* tmp, cudaStream_t s);

// LSD radix sort on bits [0, bits) of the keys; stable.  Returns (via *out)
// whichever of the two key buffers holds the result (and the values with it).
// A bounded wait that runs out sets DEVERR_TIMEOUT in *err (a device word).
size_t radix_tmp_bytes(int64_t N);
aot_status radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, int64_t N, int bits, void* tmp,
                          uint32_t* err, cudaStream_t s, uint64_t** out);
aot_status radix_sort_u32_pairs(uint32_t* keys, uint32_t* keys_alt, uint32_t* vals,
                                uint32_t* vals_alt, int64_t N, int bits, void* tmp, uint32_t* err,
                                cudaStream_t s, uint32_t** keys_out, uint32_t** vals_out);

// ------------------------------------------------------------ graph handle
// Pivot bins of the intersection kernels (by deg+ of the pivot).
enum Bin { BIN_WARP = 0, BIN_CTA = 1, BIN_HUB = 2, NUM_BINS = 3 };

struct Tuning {
  uint32_t warp_max_outdeg = 64;    // BIN_WARP: 1..warp_max (table 2*pow2 slots)
  uint32_t cta_max_outdeg = 512;    // BIN_CTA: ..cta_max (smem hash)
  int cta_threads = 32;              // 32: the CTA bin a warp per pivot
  int warp_cta_threads = 256;
  int hub_bitmaps = 32;             // concurrent hub bitmaps (n bits each)
  int hub_mode = 0;                 // 0: segmented shared-memory bitmap, 1: global bitmaps
  uint32_t seg_bits = 1280u * 1024u;  // ranks per shared-memory bitmap segment (hub_mode 0)
  uint32_t seg_wide = 512;            // hub_mode 0: warp walks take rounds of 256 while this many entries remain
  uint32_t seg_long = 128;            // hub_mode 0: items this long walked warp-wide, shorter ones per thread
  uint32_t tile_bits = 0;             // hub_mode 0: tasks tile by tile of 2^tile_bits list entries (0: off)
  uint32_t seg_tail = 128;            // hub_mode 0: after the first segment, items with fewer entries left walk per thread
  int seg_threads = 1024;             // hub_mode 0: threads per CTA of the segmented bitmap kernel
  uint32_t seg_hash = 12288;          // hub_mode 0: pivot tails up to this many entries take one hashed pass
};

struct DevScalars {  // small device-resident scalars
  unsigned long long total;      // triangle total
  unsigned long long aux[7];
  unsigned int err;              // error word
  unsigned int counters[15];     // work-queue cursors
  unsigned long long bins[4 * 3];  // per bin: pivots, items, walk, staged deg+
};

}  // namespace aot

struct aot_graph {
  int32_t n = 0;
  int64_t m = 0;
  int64_t num_edges = 0;
  uint32_t flags = 0;
  int bits = 1;          // ceil(log2(n)), >= 1
  uint64_t W = 0, S = 0;
  uint64_t merge_work = 0;  // W + sum over pivots of items x deg+ (merge route)
  uint64_t positive = 0;    // items whose pivot is the tail of their edge
  int32_t max_outdeg = 0;
  // rank-space arrays in the workspace
  int32_t* perm = nullptr;   // n : eta position -> original id
  int32_t* rank = nullptr;   // n : original id -> eta position
  uint32_t* degr = nullptr;  // n : undirected degree per eta position
  uint32_t* off = nullptr;   // n+1
  uint32_t* adj = nullptr;   // m
  uint32_t* outdeg = nullptr;  // n
  uint32_t* wofs = nullptr;  // n+1 work-CSR offsets per pivot
  uint2* witem = nullptr;    // m : walk range [x, y) in adj
  uint32_t* wvert = nullptr; // m : the walked vertex (v or x)
  uint32_t* wedge = nullptr; // m : oriented edge id of the item
  uint32_t* items = nullptr; // n : items per pivot
  uint64_t* walk = nullptr;  // n : walk length per pivot
  uint32_t* bin_pivots = nullptr;  // n : pivots grouped by bin
  uint32_t* bin_flag = nullptr;    // n : scratch for binning
  uint32_t* bin_pos = nullptr;     // n+1
  uint32_t* hub_bitmap = nullptr;  // hub_bitmaps * ceil(n/32)
  uint32_t* hubinfo = nullptr;     // 4 * n : hub descriptors
  uint64_t* tv = nullptr;          // n : per-vertex counts (rank space)
  uint32_t* tcnt = nullptr;        // m : triangles per oriented edge (list)
  uint64_t* toff = nullptr;        // m+1
  uint8_t* route = nullptr;        // m : variant per item (routed runs)
  uint32_t* rprobe = nullptr;      // n : probe items per pivot (routed runs)
  uint2* eplist = nullptr;         // m : (item, pivot) of staging-free items
  bool routed = false;             // route/rprobe/eplist valid for the current run
  const void* model = nullptr;     // learned router parameters (device)
  void* scan_tmp = nullptr;
  aot::DevScalars* dev = nullptr;
  bool has_list = false;
  bool list_ready = false;
  uint64_t* lblk = nullptr;       // listing block ranges (in tcnt's words once the offsets are scanned)
  uint64_t list_total = 0;
  // bins (host copy of counts), valid for the thresholds in `binned_for`
  uint32_t bin_count[aot::NUM_BINS] = {0, 0, 0};
  uint64_t bin_stats[aot::NUM_BINS][4] = {};  // pivots, items, walk, staged
  uint32_t binned_warp_max = 0, binned_cta_max = 0;
  aot::Tuning tune;
};

namespace aot {
enum Variant { V_PROBE = 0, V_MERGE = 1, V_BSEARCH = 2, V_SKIP = 3 };
aot_status learned_routes(aot_graph* g, cudaStream_t s);
aot_status bin_pivots(aot_graph* g, cudaStream_t s);
Tuning default_tuning();
const void* default_router();
aot_status read_device_error(aot_graph* g, cudaStream_t s);
}  // namespace aot
