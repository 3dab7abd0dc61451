// aot_sort.cu - device-wide exclusive scan and LSD radix sort.
//
// Scan: three phases per level (tile reduce, recursive scan of the tile sums,
// tile scan with offsets); tile = 256 threads x 8 items.
// Radix sort: 8-bit digits; one histogram pass over all digits, then one
// sweep per digit with decoupled look-back for the tiles' output offsets
// (each wait bounded), ranking keys inside each warp with __match_any_sync
// and writing each digit run of a tile contiguously.
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
// LSD radix sort with 8-bit digits, one sweep per digit.  A first kernel
// counts every digit of every key (all passes at once) into global
// histograms, whose exclusive scans give each digit's first output position.
// Per pass, a CTA takes the next tile of 4096 keys from a counter (so every
// earlier tile is already held by a running or finished CTA), ranks its keys
// inside each warp with __match_any_sync, publishes its per-digit counts, and
// adds up the counts of the earlier tiles by looking back over what they
// published (decoupled look-back: a tile that has finished its look-back
// publishes its inclusive prefix, which ends the look-back of later tiles).
// Every wait on an unpublished predecessor is bounded: when it runs out the
// kernel sets the timeout bit of the error word and goes on.  The tile is
// staged in shared memory in digit order and written in contiguous runs.
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;                       // keys per lane
constexpr int RS_WARP_KEYS = 32 * RS_ROUNDS;        // 512
constexpr int RS_TILE = RS_WARPS * RS_WARP_KEYS;    // 4096
constexpr int RS_BUCKETS = 256;
constexpr int RS_MAX_PASSES = 8;                    // 64-bit keys

// look-back status words: flag in the top two bits, count below
constexpr uint64_t LB_AGG = 1ull << 62;             // the tile's own counts
constexpr uint64_t LB_PREFIX = 2ull << 62;          // the tile's and every earlier tile's
constexpr uint64_t LB_VALUE = (1ull << 62) - 1;
constexpr uint32_t LB_SPIN_LIMIT = 1u << 22;        // polls of one predecessor (~seconds)
constexpr int LB_BATCH = 4;                         // status words read per look-back step

// Global histograms of every digit (passes x 256), per-warp copies in shared
// memory (no lane serialisation across warps), grid-stride over the keys.
template <class K>
__global__ void __launch_bounds__(RS_THREADS) k_digit_hist(const K* __restrict__ keys, int64_t N,
                                                           int passes, uint32_t* __restrict__ hist) {
  extern __shared__ uint32_t dh[];  // [RS_WARPS][passes][256]
  const unsigned warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * passes * RS_BUCKETS; i += RS_THREADS) dh[i] = 0;
  __syncthreads();
  uint32_t* mine = dh + (size_t)warp * passes * RS_BUCKETS;
  const int64_t stride = (int64_t)gridDim.x * RS_THREADS;
  for (int64_t i = (int64_t)blockIdx.x * RS_THREADS + threadIdx.x; i < N; i += stride) {
    const K k = __ldcs(keys + i);
    for (int p = 0; p < passes; ++p) atomicAdd(&mine[p * RS_BUCKETS + (unsigned)((k >> (8 * p)) & 0xFF)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * RS_BUCKETS; i += RS_THREADS) {
    uint32_t c = 0;
    for (int w = 0; w < RS_WARPS; ++w) c += dh[w * passes * RS_BUCKETS + i];
    if (c) atomicAdd(&hist[i], c);
  }
}

// exclusive scan of each pass's 256 digit counts: the digit's first position
__global__ void __launch_bounds__(RS_THREADS) k_digit_base(const uint32_t* __restrict__ hist,
                                                           uint32_t* __restrict__ base) {
  __shared__ uint32_t wtot[RS_WARPS];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, t = threadIdx.x;
  const uint32_t c = hist[blockIdx.x * RS_BUCKETS + t];
  const uint32_t incl = warp_inclusive_scan(c);
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  uint32_t wp = 0;
  for (int w = 0; w < (int)warp; ++w) wp += wtot[w];
  base[blockIdx.x * RS_BUCKETS + t] = wp + incl - c;
}

__device__ __forceinline__ uint64_t lb_load(const uint64_t* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void lb_store(uint64_t* p, uint64_t v) {
  atomicExch(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}
__device__ __forceinline__ uint32_t lb_load(const uint32_t* p) { return *reinterpret_cast<const volatile uint32_t*>(p); }
__device__ __forceinline__ void lb_store(uint32_t* p, uint32_t v) { atomicExch(reinterpret_cast<unsigned int*>(p), v); }

// Look-back status words of the persistent kernel: 64-bit (counts up to
// 2^62, four words per look-back step) or, for fewer than 2^30 keys, 32-bit
// (flag in the top two bits, count below; eight words per step, the same
// bytes as four 64-bit ones).
template <class SW>
struct LbWord;
template <>
struct LbWord<uint64_t> {
  static constexpr uint64_t AGG = LB_AGG, PREFIX = LB_PREFIX, VALUE = LB_VALUE;
  static constexpr int BATCH = 4;
};
template <>
struct LbWord<uint32_t> {
  static constexpr uint32_t AGG = 1u << 30, PREFIX = 2u << 30, VALUE = (1u << 30) - 1;
  static constexpr int BATCH = 8;
};

template <class K, bool VALS>
__global__ void __launch_bounds__(RS_THREADS, 3) k_onesweep(const K* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin, int64_t N,
                                                         int shift, const uint32_t* __restrict__ dbase,
                                                         uint64_t* __restrict__ status,
                                                         unsigned int* __restrict__ tile_ctr,
                                                         K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                         uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  K* sk = reinterpret_cast<K*>(rs_smem);
  uint32_t* sv = reinterpret_cast<uint32_t*>(rs_smem + sizeof(K) * RS_TILE);
  __shared__ uint32_t wh[RS_WARPS][RS_BUCKETS];
  __shared__ uint32_t dstart[RS_BUCKETS];
  __shared__ uint32_t gofs[RS_BUCKETS];
  __shared__ uint32_t wtot[RS_WARPS];
  __shared__ uint32_t s_tile;
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, t = threadIdx.x;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) wh[w][t] = 0;
  if (t == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const int64_t tile_base = (int64_t)tile * RS_TILE;
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
  // per digit t: exclusive prefix over warps and the tile's count
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) {
    uint32_t c = wh[w][t];
    wh[w][t] = tot;
    tot += c;
  }
  // publish this tile's count of digit t at once (later tiles wait on it)
  uint64_t* st = status + (size_t)tile * RS_BUCKETS + t;
  lb_store(st, (tile == 0 ? LB_PREFIX : LB_AGG) | tot);
  // block exclusive scan of the 256 digit totals: digit runs inside the tile
  uint32_t incl = warp_inclusive_scan(tot);
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  uint32_t wp = 0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w)
    if (w < (int)warp) wp += wtot[w];
  dstart[t] = wp + incl - tot;
  __syncthreads();
  // the tile in digit order in shared memory (while earlier tiles publish)
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
  // add up the earlier tiles' counts of digit t, LB_BATCH status words per
  // step, back to the first inclusive prefix (tile 0 always has one)
  uint64_t excl = 0;
  if (tile > 0) {
    int64_t pt = (int64_t)tile - 1;
    uint32_t spins = 0;
    while (true) {
      uint64_t v[LB_BATCH];
#pragma unroll
      for (int q = 0; q < LB_BATCH; ++q)
        v[q] = pt - q >= 0 ? lb_load(status + (size_t)(pt - q) * RS_BUCKETS + t) : LB_PREFIX;
      int used = 0;
      bool done = false;
#pragma unroll
      for (int q = 0; q < LB_BATCH; ++q) {
        if (done || used < q) continue;  // stopped at an earlier word
        const uint64_t f = v[q] & ~LB_VALUE;
        if (!f) continue;  // not published yet: poll again from here
        excl += v[q] & LB_VALUE;
        used = q + 1;
        done = f == LB_PREFIX;
      }
      if (done) break;
      pt -= used;
      if (used < LB_BATCH) {  // waiting on tile pt
        if (++spins >= LB_SPIN_LIMIT) {
          atomicOr(err, DEVERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    lb_store(st, LB_PREFIX | (excl + tot));
  }
  gofs[t] = dbase[t] + (uint32_t)excl;
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

// ---- TMA bulk copies into shared memory, completed on an mbarrier (PTX)
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bytes: a multiple of 16; both addresses 16-byte aligned
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

constexpr uint32_t MB_SPIN_LIMIT = 1u << 24;  // try_wait polls of one copy

// Persistent form of k_onesweep for 8-byte keys (no values): each CTA takes
// tiles from the counter one ahead, so that the next tile's keys stream into
// shared memory (one TMA bulk copy, two buffers) while it ranks, publishes,
// looks back and writes the current one.  The tile is staged in digit order
// in its own input buffer (the keys are in registers by then).  Tiles are
// taken in increasing order and the tile held ahead is always later than the
// one in hand, so the earliest unfinished tile is always some CTA's current
// tile and every look-back ends.  A copy that does not complete within the
// poll limit sets the timeout bit; the CTA then stops taking tiles.
template <class SW>
__global__ void __launch_bounds__(RS_THREADS, 3) k_onesweep_tma(const uint64_t* __restrict__ kin, int64_t N,
                                                             int64_t tiles, int shift,
                                                             const uint32_t* __restrict__ dbase,
                                                             SW* __restrict__ status,
                                                             unsigned int* __restrict__ tile_ctr,
                                                             uint64_t* __restrict__ kout,
                                                             uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  uint64_t* buf = reinterpret_cast<uint64_t*>(rs_smem);  // [2][RS_TILE]
  __shared__ uint32_t wh[RS_WARPS][RS_BUCKETS];
  __shared__ uint32_t dstart[RS_BUCKETS];
  __shared__ uint32_t gofs[RS_BUCKETS];
  __shared__ uint32_t wtot[RS_WARPS];
  __shared__ uint32_t s_tile[2];
  __shared__ __align__(8) uint64_t s_bar[2];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, t = threadIdx.x;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) wh[w][t] = 0;
  // issue the copy of tile `tl` into buffer b (a plain arrive when there is
  // nothing to copy, so that the buffer's phase still completes)
  auto fetch = [&](uint32_t tl, int b) {
    const int64_t tb = (int64_t)tl * RS_TILE;
    const int64_t rem = N - tb;
    const uint32_t cnt = rem < RS_TILE ? (uint32_t)rem : (uint32_t)RS_TILE;
    const uint32_t bytes = (cnt & ~1u) * (uint32_t)sizeof(uint64_t);  // 16-byte multiple
    if (bytes) {
      mbar_expect_tx(&s_bar[b], bytes);
      bulk_load(buf + (size_t)b * RS_TILE, kin + tb, bytes, &s_bar[b]);
    } else {
      mbar_arrive(&s_bar[b]);
    }
  };
  if (t == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_mbar_init();
    const uint32_t t0 = atomicAdd(tile_ctr, 1u);
    s_tile[0] = t0;
    if ((int64_t)t0 < tiles) fetch(t0, 0);
  }
  __syncthreads();
  for (uint32_t it = 0;; ++it) {
    const int cb = (int)(it & 1u);
    const uint32_t tile = s_tile[cb];
    if ((int64_t)tile >= tiles) break;
    if (t == 0) {  // the next tile, one ahead
      fence_proxy_async();  // earlier generic accesses of that buffer before the copy
      const uint32_t nx = atomicAdd(tile_ctr, 1u);
      s_tile[cb ^ 1] = nx;
      if ((int64_t)nx < tiles) fetch(nx, cb ^ 1);
    }
    bool ok = false;
    for (uint32_t sp = 0; sp < MB_SPIN_LIMIT && !ok; ++sp) ok = mbar_try_wait(&s_bar[cb], (it >> 1) & 1u);
    if (__syncthreads_or(!ok)) {
      if (t == 0) atomicOr(err, DEVERR_TIMEOUT);
      // let this CTA's copies in flight land before it exits (bounded again)
      for (uint32_t sp = 0; sp < MB_SPIN_LIMIT && !mbar_try_wait(&s_bar[cb], (it >> 1) & 1u); ++sp) {
      }
      if ((int64_t)s_tile[cb ^ 1] < tiles)
        for (uint32_t sp = 0; sp < MB_SPIN_LIMIT && !mbar_try_wait(&s_bar[cb ^ 1], ((it + 1) >> 1) & 1u); ++sp) {
        }
      break;
    }
    const uint64_t* sk = buf + (size_t)cb * RS_TILE;
    uint64_t* so = buf + (size_t)cb * RS_TILE;
    const int64_t tile_base = (int64_t)tile * RS_TILE;
    const int64_t rem = N - tile_base;
    const int tile_n = rem < RS_TILE ? (int)rem : RS_TILE;
    const int copied = tile_n & ~1;
    const int wbase = (int)warp * RS_WARP_KEYS;
    uint64_t key[RS_ROUNDS];
    uint32_t lrk[RS_ROUNDS / 2];
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
      const int j = wbase + r * 32 + (int)lane;
      key[r] = j < copied ? sk[j] : (j < tile_n ? kin[tile_base + j] : 0ull);
    }
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
      const int j = wbase + r * 32 + (int)lane;
      const bool valid = j < tile_n;
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
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      uint32_t c = wh[w][t];
      wh[w][t] = tot;
      tot += c;
    }
    using W = LbWord<SW>;
    SW* st = status + (size_t)tile * RS_BUCKETS + t;
    lb_store(st, (SW)((tile == 0 ? W::PREFIX : W::AGG) | tot));
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
      const int j = wbase + r * 32 + (int)lane;
      if (j < tile_n) {
        unsigned d = (unsigned)((key[r] >> shift) & 0xFF);
        const uint32_t lr = (r & 1) ? (lrk[r >> 1] >> 16) : (lrk[r >> 1] & 0xffffu);
        so[dstart[d] + wh[warp][d] + lr] = key[r];
      }
    }
    uint64_t excl = 0;
    if (tile > 0) {
      int64_t pt = (int64_t)tile - 1;
      uint32_t spins = 0;
      while (true) {
        SW v[W::BATCH];
#pragma unroll
        for (int q = 0; q < W::BATCH; ++q)
          v[q] = pt - q >= 0 ? lb_load(status + (size_t)(pt - q) * RS_BUCKETS + t) : W::PREFIX;
        int used = 0;
        bool done = false;
#pragma unroll
        for (int q = 0; q < W::BATCH; ++q) {
          if (done || used < q) continue;  // stopped at an earlier word
          const SW f = v[q] & ~W::VALUE;
          if (!f) continue;  // not published yet: poll again from here
          excl += v[q] & W::VALUE;
          used = q + 1;
          done = f == W::PREFIX;
        }
        if (done) break;
        pt -= used;
        if (used < W::BATCH) {  // waiting on tile pt
          if (++spins >= LB_SPIN_LIMIT) {
            atomicOr(err, DEVERR_TIMEOUT);
            break;
          }
          __nanosleep(64);
        }
      }
      lb_store(st, (SW)(W::PREFIX | (excl + tot)));
    }
    gofs[t] = dbase[t] + (uint32_t)excl;
    __syncthreads();
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) wh[w][t] = 0;  // for the next tile's ranking
    for (int j = t; j < tile_n; j += RS_THREADS) {
      const uint64_t k = so[j];
      const unsigned d = (unsigned)((k >> shift) & 0xFF);
      kout[gofs[d] + (uint32_t)(j - (int)dstart[d])] = k;
    }
    __syncthreads();
  }
}

// tmp: histograms and digit bases (passes x 256 each), tile counters, and the
// look-back status words (tiles x 256)
size_t radix_tmp_bytes(int64_t N) {
  int64_t tiles = (N + RS_TILE - 1) / RS_TILE;
  if (tiles < 1) tiles = 1;
  return 2 * (size_t)RS_MAX_PASSES * RS_BUCKETS * sizeof(uint32_t) + 256 +
         (size_t)tiles * RS_BUCKETS * sizeof(uint64_t) + 256;
}

template <class K, bool VALS>
static aot_status radix_impl(K* keys, K* keys_alt, uint32_t* vals, uint32_t* vals_alt, int64_t N,
                             int bits, void* tmp, uint32_t* err, cudaStream_t s, K** kout,
                             uint32_t** vout) {
  *kout = keys;
  if (vout) *vout = vals;
  if (N <= 1 || bits <= 0) return AOT_OK;
  // output positions are 32-bit
  if ((uint64_t)N + RS_TILE > 0xF0000000ull) return AOT_ERR_OVERFLOW;
  const int passes = (bits + 7) / 8;
  if (passes > (int)sizeof(K)) return AOT_ERR_INVALID_ARG;
  const int64_t tiles = (N + RS_TILE - 1) / RS_TILE;
  char* c = static_cast<char*>(tmp);
  uint32_t* hist = reinterpret_cast<uint32_t*>(c);
  uint32_t* dbase = hist + RS_MAX_PASSES * RS_BUCKETS;
  unsigned int* ctr = reinterpret_cast<unsigned int*>(dbase + RS_MAX_PASSES * RS_BUCKETS);
  uint64_t* status = reinterpret_cast<uint64_t*>(c + 2 * (size_t)RS_MAX_PASSES * RS_BUCKETS * sizeof(uint32_t) + 256);
  const size_t status_bytes = (size_t)tiles * RS_BUCKETS * sizeof(uint64_t);
  AOT_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * RS_MAX_PASSES * RS_BUCKETS, s));
  AOT_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned int) * RS_MAX_PASSES, s));
  const size_t hsmem = (size_t)RS_WARPS * passes * RS_BUCKETS * sizeof(uint32_t);
  AOT_TRY(ensure_dyn_smem((const void*)k_digit_hist<K>, hsmem));
  int64_t hgrid = (int64_t)sm_count() * 8;
  if (hgrid > tiles) hgrid = tiles;
  AOT_KERNEL("k_digit_hist", s)
    k_digit_hist<K><<<(unsigned)hgrid, RS_THREADS, hsmem, s>>>(keys, N, passes, hist);
  AOT_TRY(last_launch());
  AOT_KERNEL("k_digit_base", s)
    k_digit_base<<<(unsigned)passes, RS_THREADS, 0, s>>>(hist, dbase);
  AOT_TRY(last_launch());
  const size_t smem = sizeof(K) * RS_TILE + (VALS ? sizeof(uint32_t) * RS_TILE : 0);
  AOT_TRY(ensure_dyn_smem((const void*)k_onesweep<K, VALS>, smem));
  AOT_TRY(prefer_max_smem((const void*)k_onesweep<K, VALS>));
  // 8-byte keys from 16-byte aligned buffers: the persistent kernel that
  // prefetches each CTA's next tile with a TMA bulk copy
  constexpr bool kTmaKeys = sizeof(K) == 8 && !VALS;
  const bool tma = kTmaKeys && ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(keys_alt)) & 15) == 0;
  const size_t tsmem = 2 * sizeof(uint64_t) * RS_TILE;
  int tgrid = 0;
  if (tma) {
    for (const void* f : {(const void*)k_onesweep_tma<uint32_t>, (const void*)k_onesweep_tma<uint64_t>}) {
      AOT_TRY(ensure_dyn_smem(f, tsmem));
      AOT_TRY(prefer_max_smem(f));
    }
    int per_sm = 0;
    AOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep_tma<uint64_t>, RS_THREADS, tsmem));
    int64_t g = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);
    tgrid = (int)(g < tiles ? g : tiles);
  }
  K* a = keys;
  K* b = keys_alt;
  uint32_t* va = vals;
  uint32_t* vb = vals_alt;
  for (int p = 0; p < passes; ++p) {
    AOT_CUDA(cudaMemsetAsync(status, 0, status_bytes, s));
    if constexpr (kTmaKeys) {
      if (tma) {
        AOT_KERNEL("k_onesweep", s) {
          const uint64_t* ka = reinterpret_cast<const uint64_t*>(a);
          uint64_t* kb = reinterpret_cast<uint64_t*>(b);
          if (N < (int64_t)LbWord<uint32_t>::VALUE)  // every count fits 30 bits
            k_onesweep_tma<uint32_t><<<(unsigned)tgrid, RS_THREADS, tsmem, s>>>(
                ka, N, tiles, 8 * p, dbase + p * RS_BUCKETS, reinterpret_cast<uint32_t*>(status), ctr + p, kb, err);
          else
            k_onesweep_tma<uint64_t><<<(unsigned)tgrid, RS_THREADS, tsmem, s>>>(
                ka, N, tiles, 8 * p, dbase + p * RS_BUCKETS, status, ctr + p, kb, err);
        }
        AOT_TRY(last_launch());
        K* t = a; a = b; b = t;
        continue;
      }
    }
    AOT_KERNEL("k_onesweep", s)
      k_onesweep<K, VALS><<<(unsigned)tiles, RS_THREADS, smem, s>>>(a, va, N, 8 * p, dbase + p * RS_BUCKETS,
                                                                    status, ctr + p, b, vb, err);
    AOT_TRY(last_launch());
    K* t = a; a = b; b = t;
    uint32_t* tv = va; va = vb; vb = tv;
  }
  *kout = a;
  if (vout) *vout = va;
  return AOT_OK;
}

aot_status radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, int64_t N, int bits, void* tmp,
                          uint32_t* err, cudaStream_t s, uint64_t** out) {
  return radix_impl<uint64_t, false>(keys, keys_alt, nullptr, nullptr, N, bits, tmp, err, s, out,
                                     nullptr);
}

aot_status radix_sort_u32_pairs(uint32_t* keys, uint32_t* keys_alt, uint32_t* vals,
                                uint32_t* vals_alt, int64_t N, int bits, void* tmp, uint32_t* err,
                                cudaStream_t s, uint32_t** keys_out, uint32_t** vals_out) {
  return radix_impl<uint32_t, true>(keys, keys_alt, vals, vals_alt, N, bits, tmp, err, s, keys_out,
                                    vals_out);
}

}  // namespace aot
