// aot_sort.cu - device-wide exclusive scan and LSD radix sort.
//
// Scan: three phases per level (tile reduce, recursive scan of the tile sums,
// tile scan with offsets); tile = 256 threads x 8 items.
// Radix sort: 8-bit digits, per pass (1) per-tile digit histograms, (2) an
// exclusive scan of the digit-major histogram table, (3) a stable scatter
// that ranks keys inside each warp with __match_any_sync, stages the tile in
// shared memory in digit order and writes each digit run contiguously.
#include "aot_internal.cuh"

namespace aot {

// ---------------------------------------------------------------------- scan
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class Tin, class Tout>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_reduce(const Tin* __restrict__ in, int64_t N,
                                                              Tout* __restrict__ sums) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  Tout acc = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t k = base + i * SCAN_THREADS + threadIdx.x;
    if (k < N) acc += (Tout)in[k];
  }
  acc = warp_sum(acc);
  __shared__ Tout ws[SCAN_THREADS / 32];
  if (lane_id() == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    Tout v = threadIdx.x < SCAN_THREADS / 32 ? ws[threadIdx.x] : Tout(0);
    v = warp_sum(v);
    if (threadIdx.x == 0) sums[blockIdx.x] = v;
  }
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const Tin* in, int64_t N,
                                                            const Tout* __restrict__ offsets,
                                                            Tout* out) {
  __shared__ Tout sh[SCAN_TILE];
  __shared__ Tout wsum[SCAN_THREADS / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  const int t = threadIdx.x;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t k = base + i * SCAN_THREADS + t;
    sh[i * SCAN_THREADS + t] = k < N ? (Tout)in[k] : Tout(0);
  }
  __syncthreads();
  Tout loc[SCAN_ITEMS];
  Tout s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    loc[k] = sh[t * SCAN_ITEMS + k];
    s += loc[k];
  }
  Tout incl = warp_inclusive_scan(s);
  if (lane_id() == 31) wsum[t >> 5] = incl;
  __syncthreads();
  Tout wpre = 0, tile_total = 0;
#pragma unroll
  for (int w = 0; w < SCAN_THREADS / 32; ++w) {
    Tout x = wsum[w];
    if (w < (t >> 5)) wpre += x;
    tile_total += x;
  }
  Tout off0 = offsets ? offsets[blockIdx.x] : Tout(0);
  Tout run = off0 + wpre + incl - s;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    sh[t * SCAN_ITEMS + k] = run;
    run += loc[k];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int64_t k = base + i * SCAN_THREADS + t;
    if (k < N) out[k] = sh[i * SCAN_THREADS + t];
  }
  if (blockIdx.x == gridDim.x - 1 && t == 0) out[N] = off0 + tile_total;
}

size_t scan_tmp_bytes(int64_t N) {
  size_t bytes = 0;
  int64_t n = N;
  while (n > SCAN_TILE) {
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    bytes += ((size_t)(tiles + 1) * 8 + 255) & ~size_t(255);
    n = tiles;
  }
  return bytes + 256;
}

template <class Tin, class Tout>
static aot_status scan_impl(const Tin* in, Tout* out, int64_t N, char* tmp, cudaStream_t s) {
  if (N <= 0) {
    AOT_CUDA(cudaMemsetAsync(out, 0, sizeof(Tout), s));
    return AOT_OK;
  }
  int64_t tiles = (N + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles == 1) {
    AOT_KERNEL("k_tile_scan", s)
      k_tile_scan<Tin, Tout><<<1, SCAN_THREADS, 0, s>>>(in, N, nullptr, out);
    return last_launch();
  }
  Tout* sums = reinterpret_cast<Tout*>(tmp);
  char* next = tmp + (((size_t)(tiles + 1) * 8 + 255) & ~size_t(255));
  AOT_KERNEL("k_tile_reduce", s)
    k_tile_reduce<Tin, Tout><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, N, sums);
  AOT_TRY(last_launch());
  AOT_TRY((scan_impl<Tout, Tout>(sums, sums, tiles, next, s)));
  AOT_KERNEL("k_tile_scan", s)
    k_tile_scan<Tin, Tout><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, N, sums, out);
  return last_launch();
}

aot_status scan_u32_u32(const uint32_t* in, uint32_t* out, int64_t N, void* tmp, cudaStream_t s) {
  return scan_impl<uint32_t, uint32_t>(in, out, N, static_cast<char*>(tmp), s);
}
aot_status scan_u32_u64(const uint32_t* in, uint64_t* out, int64_t N, void* tmp, cudaStream_t s) {
  return scan_impl<uint32_t, uint64_t>(in, out, N, static_cast<char*>(tmp), s);
}
aot_status scan_u64_u64(const uint64_t* in, uint64_t* out, int64_t N, void* tmp, cudaStream_t s) {
  return scan_impl<uint64_t, uint64_t>(in, out, N, static_cast<char*>(tmp), s);
}

// ---------------------------------------------------------------- radix sort
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;                       // keys per lane
constexpr int RS_WARP_KEYS = 32 * RS_ROUNDS;        // 512
constexpr int RS_TILE = RS_WARPS * RS_WARP_KEYS;    // 4096
constexpr int RS_BUCKETS = 256;

template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const K* __restrict__ keys, int64_t N,
                                                           int shift, uint32_t* __restrict__ hist,
                                                           int64_t tiles) {
  __shared__ uint32_t h[RS_BUCKETS];
  h[threadIdx.x] = 0;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  int64_t base = (int64_t)blockIdx.x * RS_TILE + warp * RS_WARP_KEYS;
  unsigned dig[RS_ROUNDS];  // every load of the lane in flight before the first ranking
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int64_t idx = base + r * 32 + lane;
    dig[r] = idx < N ? (unsigned)((__ldcs(keys + idx) >> shift) & 0xFF) : 0x100u;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const unsigned d = dig[r];
    unsigned peers = __match_any_sync(FULL, d);
    if (d < 0x100u && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

template <class K, bool VALS>
__global__ void __launch_bounds__(RS_THREADS, 3) k_radix_scatter(const K* __restrict__ kin,
                                                              const uint32_t* __restrict__ vin,
                                                              int64_t N, int shift,
                                                              const uint32_t* __restrict__ offs,
                                                              int64_t tiles, K* __restrict__ kout,
                                                              uint32_t* __restrict__ vout) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  K* sk = reinterpret_cast<K*>(rs_smem);
  uint32_t* sv = reinterpret_cast<uint32_t*>(rs_smem + sizeof(K) * RS_TILE);
  __shared__ uint32_t wh[RS_WARPS][RS_BUCKETS];
  __shared__ uint32_t dstart[RS_BUCKETS];
  __shared__ uint32_t gofs[RS_BUCKETS];
  __shared__ uint32_t wtot[RS_WARPS];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, t = threadIdx.x;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) wh[w][t] = 0;
  gofs[t] = offs[(int64_t)t * tiles + blockIdx.x];
  __syncthreads();

  const int64_t tile_base = (int64_t)blockIdx.x * RS_TILE;
  const int64_t base = tile_base + warp * RS_WARP_KEYS;
  K key[RS_ROUNDS];
  uint32_t val[RS_ROUNDS];
  uint32_t lrk[RS_ROUNDS / 2];  // local ranks (< 512), two 16-bit halves per word
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {  // every load of the lane in flight first
    int64_t idx = base + r * 32 + lane;
    bool valid = idx < N;
    key[r] = valid ? __ldcs(kin + idx) : K(0);
    if (VALS) val[r] = valid ? __ldcs(vin + idx) : 0u;
  }
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int64_t idx = base + r * 32 + lane;
    bool valid = idx < N;
    unsigned d = valid ? (unsigned)((key[r] >> shift) & 0xFF) : 0x100u;
    unsigned peers = __match_any_sync(FULL, d);
    unsigned leader = (unsigned)(__ffs(peers) - 1);
    uint32_t before = 0;
    if (valid && lane == leader) {
      before = wh[warp][d];
      wh[warp][d] = before + (uint32_t)__popc(peers);
    }
    before = __shfl_sync(FULL, before, leader);
    const uint32_t lr = before + (uint32_t)__popc(peers & lanemask_lt());
    if (r & 1) lrk[r >> 1] |= lr << 16;
    else lrk[r >> 1] = lr;
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, digit totals
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) {
    uint32_t c = wh[w][t];
    wh[w][t] = tot;
    tot += c;
  }
  // block exclusive scan of the 256 digit totals
  uint32_t incl = warp_inclusive_scan(tot);
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  uint32_t wp = 0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w)
    if (w < (int)warp) wp += wtot[w];
  dstart[t] = wp + incl - tot;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    int64_t idx = base + r * 32 + lane;
    if (idx < N) {
      unsigned d = (unsigned)((key[r] >> shift) & 0xFF);
      const uint32_t lr = (r & 1) ? (lrk[r >> 1] >> 16) : (lrk[r >> 1] & 0xffffu);
      uint32_t pos = dstart[d] + wh[warp][d] + lr;
      sk[pos] = key[r];
      if (VALS) sv[pos] = val[r];
    }
  }
  __syncthreads();
  int64_t rem = N - tile_base;
  int tile_n = rem < RS_TILE ? (int)rem : RS_TILE;
  for (int j = t; j < tile_n; j += RS_THREADS) {
    K k = sk[j];
    unsigned d = (unsigned)((k >> shift) & 0xFF);
    uint32_t o = gofs[d] + (uint32_t)(j - (int)dstart[d]);
    kout[o] = k;
    if (VALS) vout[o] = sv[j];
  }
}

size_t radix_tmp_bytes(int64_t N) {
  int64_t tiles = (N + RS_TILE - 1) / RS_TILE;
  if (tiles < 1) tiles = 1;
  size_t hist = ((size_t)RS_BUCKETS * tiles + 1) * sizeof(uint32_t);
  hist = (hist + 255) & ~size_t(255);
  return 2 * hist + scan_tmp_bytes((int64_t)RS_BUCKETS * tiles) + 256;
}

template <class K, bool VALS>
static aot_status radix_impl(K* keys, K* keys_alt, uint32_t* vals, uint32_t* vals_alt, int64_t N,
                             int bits, void* tmp, cudaStream_t s, K** kout, uint32_t** vout) {
  *kout = keys;
  if (vout) *vout = vals;
  if (N <= 1 || bits <= 0) return AOT_OK;
  // the combined table index (digit * tiles + tile) must fit uint32
  if ((uint64_t)N + RS_TILE > 0xF0000000ull) return AOT_ERR_OVERFLOW;
  int64_t tiles = (N + RS_TILE - 1) / RS_TILE;
  size_t hist_bytes = (((size_t)RS_BUCKETS * tiles + 1) * sizeof(uint32_t) + 255) & ~size_t(255);
  uint32_t* hist = static_cast<uint32_t*>(tmp);
  uint32_t* offs = reinterpret_cast<uint32_t*>(static_cast<char*>(tmp) + hist_bytes);
  void* stmp = static_cast<char*>(tmp) + 2 * hist_bytes;
  size_t smem = sizeof(K) * RS_TILE + (VALS ? sizeof(uint32_t) * RS_TILE : 0);
  AOT_TRY(ensure_dyn_smem((const void*)k_radix_scatter<K, VALS>, smem));
  AOT_TRY(prefer_max_smem((const void*)k_radix_scatter<K, VALS>));
  K* a = keys;
  K* b = keys_alt;
  uint32_t* va = vals;
  uint32_t* vb = vals_alt;
  for (int shift = 0; shift < bits; shift += 8) {
    AOT_KERNEL("k_radix_hist", s)
      k_radix_hist<K><<<(unsigned)tiles, RS_THREADS, 0, s>>>(a, N, shift, hist, tiles);
    AOT_TRY(last_launch());
    AOT_TRY(scan_u32_u32(hist, offs, (int64_t)RS_BUCKETS * tiles, stmp, s));
    AOT_KERNEL("k_radix_scatter", s)
      k_radix_scatter<K, VALS><<<(unsigned)tiles, RS_THREADS, smem, s>>>(a, va, N, shift, offs,
                                                                         tiles, b, vb);
    AOT_TRY(last_launch());
    K* t = a; a = b; b = t;
    uint32_t* tv = va; va = vb; vb = tv;
  }
  *kout = a;
  if (vout) *vout = va;
  return AOT_OK;
}

aot_status radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, int64_t N, int bits, void* tmp,
                          cudaStream_t s, uint64_t** out) {
  return radix_impl<uint64_t, false>(keys, keys_alt, nullptr, nullptr, N, bits, tmp, s, out,
                                     nullptr);
}

aot_status radix_sort_u32_pairs(uint32_t* keys, uint32_t* keys_alt, uint32_t* vals,
                                uint32_t* vals_alt, int64_t N, int bits, void* tmp,
                                cudaStream_t s, uint32_t** keys_out, uint32_t** vals_out) {
  return radix_impl<uint32_t, true>(keys, keys_alt, vals, vals_alt, N, bits, tmp, s, keys_out,
                                    vals_out);
}

}  // namespace aot
