// aot_mlp.cu - the learned router: per-edge features, tensor-core inference,
// and the training kernels of its 8 -> 64 -> 64 -> 3 perceptron.
//
// The network predicts, for one work item, the standardised log cost of its
// three intersection variants (probe, merge, binary search); the router takes
// the cheapest, keeping the probe of Algorithm 3 unless another variant is
// predicted cheaper by more than a margin.  Routing never changes the output.
//
// Numerics (the same in inference and training): inputs, parameters and
// hidden activations are bfloat16 (round to nearest even); every dot product
// and bias add accumulates in fp32; the output stays fp32.
//   inference: one warp per 16 items, mma.sync m16n8k16 (bf16 in, fp32
//              accumulate); a layer's fp32 accumulator fragments are exactly
//              the next layer's A fragments, so activations stay in registers
//   training:  SIMT kernels (fp32 accumulate over bf16 values), loss
//              sum (y - t)^2 / B, Adam on an fp32 master copy that is rounded
//              back to bf16 after each step.
#include <cuda_bf16.h>

#include "aot_internal.cuh"
#include "aot_kparams.cuh"

namespace aot {

constexpr int MLP_IN = 8, MLP_H = 64, MLP_OUT = 3;
constexpr int P_W1 = 0, P_B1 = 512, P_W2 = 576, P_B2 = 4672, P_W3 = 4736, P_B3 = 4928;
constexpr int P_TOTAL = 4931;
static_assert(P_B1 == P_W1 + MLP_H * MLP_IN && P_W2 == P_B1 + MLP_H && P_B2 == P_W2 + MLP_H * MLP_H &&
                  P_W3 == P_B2 + MLP_H && P_B3 == P_W3 + MLP_OUT * MLP_H && P_TOTAL == P_B3 + MLP_OUT &&
                  P_TOTAL == AOT_MLP_PARAMS,
              "parameter layout W1[64][8], b1[64], W2[64][64], b2[64], W3[3][64], b3[3]");
constexpr size_t MO_PARAMS = 128;  // byte offset of the bf16 parameters in a model

struct ModelView {
  const float* in_mean;
  const float* in_std;
  const float* out_mean;
  const float* out_std;
  const float* margin;
  const __nv_bfloat16* prm;
};
__host__ __device__ inline ModelView model_view(const void* m) {
  const char* b = static_cast<const char*>(m);
  ModelView v;
  v.in_mean = reinterpret_cast<const float*>(b + 0);
  v.in_std = reinterpret_cast<const float*>(b + 32);
  v.out_mean = reinterpret_cast<const float*>(b + 64);
  v.out_std = reinterpret_cast<const float*>(b + 80);
  v.margin = reinterpret_cast<const float*>(b + 96);
  v.prm = reinterpret_cast<const __nv_bfloat16*>(b + MO_PARAMS);
  return v;
}

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

// d = a(16x16 bf16, row) * b(16x8 bf16, col) + c, fp32 accumulate
__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1,
                                         const float c[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%10,%11,%12,%13};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]),
        "f"(c[2]), "f"(c[3]));
}

// the eight features of oriented edge e = <u, v> (u < v in rank space)
__device__ __forceinline__ void edge_features(uint32_t u, uint32_t v, uint32_t e,
                                              const uint32_t* __restrict__ off,
                                              const uint32_t* __restrict__ outdeg,
                                              const uint32_t* __restrict__ degr, int32_t n,
                                              float f[8]) {
  const uint32_t du = outdeg[u], dv = outdeg[v], gu = degr[u], gv = degr[v];
  const uint32_t suffix = off[u] + du - e - 1;
  f[0] = log1pf((float)du);
  f[1] = log1pf((float)dv);
  f[2] = log1pf((float)suffix);
  f[3] = log1pf((float)(gu - du));
  f[4] = log1pf((float)(gv - dv));
  f[5] = log1pf((float)gu);
  f[6] = log1pf((float)gv);
  f[7] = (float)(v - u) / (float)(n > 0 ? n : 1);
}

// warp per pivot: pivot of every item (into a scratch array)
__global__ void k_item_pivot(const uint32_t* __restrict__ wofs, int32_t n, uint32_t* __restrict__ ip) {
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (p >= n) return;
  for (uint32_t i = wofs[p] + lane_id(); i < wofs[p + 1]; i += 32) ip[i] = (uint32_t)p;
}

// features per oriented edge, written in CSR edge order
__global__ void k_features(const uint32_t* __restrict__ ip, const uint32_t* __restrict__ wvert,
                           const uint32_t* __restrict__ wedge, int64_t m,
                           const uint32_t* __restrict__ off, const uint32_t* __restrict__ outdeg,
                           const uint32_t* __restrict__ degr, int32_t n, float* __restrict__ feat) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint32_t p = ip[i], x = wvert[i], e = wedge[i];
  float f[8];
  edge_features(min(p, x), max(p, x), e, off, outdeg, degr, n, f);
#pragma unroll
  for (int k = 0; k < 8; ++k) feat[(size_t)e * 8 + k] = f[k];
}

// ------------------------------------------------------------ inference
struct InferGraph {  // item source when routing a graph
  const uint32_t* ip;
  const uint32_t* wvert;
  const uint32_t* wedge;
  const uint32_t* off;
  const uint32_t* outdeg;
  const uint32_t* degr;
  int32_t n;
  uint8_t* route;
};

template <bool FROM_GRAPH>
__global__ void __launch_bounds__(256) k_mlp_infer(const void* __restrict__ model, int64_t count,
                                                  InferGraph G, const float* __restrict__ x,
                                                  float* __restrict__ y) {
  __shared__ __align__(16) __nv_bfloat16 sW1[64 * 8], sB1[64], sW2[64 * 64], sB2[64], sW3[8 * 64], sB3[8];
  __shared__ float sNorm[24];
  __shared__ float sFeat[8][16][8];
  const ModelView M = model_view(model);
  for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) sW2[i] = M.prm[P_W2 + i];
  for (int i = threadIdx.x; i < 64 * 8; i += blockDim.x) {
    sW1[i] = M.prm[P_W1 + i];
    sW3[i] = i < 3 * 64 ? M.prm[P_W3 + i] : __float2bfloat16_rn(0.f);
  }
  if (threadIdx.x < 64) {
    sB1[threadIdx.x] = M.prm[P_B1 + threadIdx.x];
    sB2[threadIdx.x] = M.prm[P_B2 + threadIdx.x];
  }
  if (threadIdx.x < 8) sB3[threadIdx.x] = threadIdx.x < 3 ? M.prm[P_B3 + threadIdx.x] : __float2bfloat16_rn(0.f);
  if (threadIdx.x < 8) {
    sNorm[threadIdx.x] = M.in_mean[threadIdx.x];
    sNorm[8 + threadIdx.x] = M.in_std[threadIdx.x];
  }
  if (threadIdx.x < 3) {
    sNorm[16 + threadIdx.x] = M.out_mean[threadIdx.x];
    sNorm[20 + threadIdx.x] = M.out_std[threadIdx.x];
  }
  __syncthreads();
  const float margin = *M.margin;
  const unsigned lane = lane_id(), wid = threadIdx.x >> 5;
  const unsigned g = lane >> 2, t = lane & 3;
  const int64_t tiles = (count + 15) / 16;
  for (int64_t tile = (int64_t)blockIdx.x * 8 + wid; tile < tiles; tile += (int64_t)gridDim.x * 8) {
    const int64_t base = tile * 16;
    if (lane < 16) {
      const int64_t i = base + lane;
      float f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (i < count) {
        if (FROM_GRAPH) {
          const uint32_t p = G.ip[i], xv = G.wvert[i], e = G.wedge[i];
          edge_features(min(p, xv), max(p, xv), e, G.off, G.outdeg, G.degr, G.n, f);
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) f[k] = x[i * 8 + k];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) f[k] = (f[k] - sNorm[k]) / sNorm[8 + k];
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) sFeat[wid][lane][k] = f[k];
    }
    __syncwarp();
    // layer 1: K = 16 (features 8..15 are zero padding)
    uint32_t A[4];
    A[0] = pack_bf16(sFeat[wid][g][2 * t], sFeat[wid][g][2 * t + 1]);
    A[1] = pack_bf16(sFeat[wid][g + 8][2 * t], sFeat[wid][g + 8][2 * t + 1]);
    A[2] = 0u;
    A[3] = 0u;
    __syncwarp();
    float h[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float b0 = __bfloat162float(sB1[j * 8 + 2 * t]), b1 = __bfloat162float(sB1[j * 8 + 2 * t + 1]);
      const float c[4] = {b0, b1, b0, b1};
      const uint32_t w0 = *reinterpret_cast<const uint32_t*>(&sW1[(j * 8 + g) * 8 + 2 * t]);
      mma_bf16(h[j], A, w0, 0u, c);
#pragma unroll
      for (int q = 0; q < 4; ++q) h[j][q] = fmaxf(h[j][q], 0.f);
    }
    // layer 2
    uint32_t A2[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      A2[kk][0] = pack_bf16(h[2 * kk][0], h[2 * kk][1]);
      A2[kk][1] = pack_bf16(h[2 * kk][2], h[2 * kk][3]);
      A2[kk][2] = pack_bf16(h[2 * kk + 1][0], h[2 * kk + 1][1]);
      A2[kk][3] = pack_bf16(h[2 * kk + 1][2], h[2 * kk + 1][3]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float b0 = __bfloat162float(sB2[j * 8 + 2 * t]), b1 = __bfloat162float(sB2[j * 8 + 2 * t + 1]);
      float c[4] = {b0, b1, b0, b1};
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const __nv_bfloat16* row = &sW2[(j * 8 + g) * 64 + kk * 16 + 2 * t];
        mma_bf16(c, A2[kk], *reinterpret_cast<const uint32_t*>(row),
                 *reinterpret_cast<const uint32_t*>(row + 8), c);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) h[j][q] = fmaxf(c[q], 0.f);
    }
    // layer 3 (3 outputs in an 8-wide tile)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      A2[kk][0] = pack_bf16(h[2 * kk][0], h[2 * kk][1]);
      A2[kk][1] = pack_bf16(h[2 * kk][2], h[2 * kk][3]);
      A2[kk][2] = pack_bf16(h[2 * kk + 1][0], h[2 * kk + 1][1]);
      A2[kk][3] = pack_bf16(h[2 * kk + 1][2], h[2 * kk + 1][3]);
    }
    const float o0 = __bfloat162float(sB3[2 * t]), o1 = __bfloat162float(sB3[2 * t + 1]);
    float o[4] = {o0, o1, o0, o1};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const __nv_bfloat16* row = &sW3[g * 64 + kk * 16 + 2 * t];
      mma_bf16(o, A2[kk], *reinterpret_cast<const uint32_t*>(row),
               *reinterpret_cast<const uint32_t*>(row + 8), o);
    }
    // row g: cols 2t, 2t+1 in o[0], o[1]; row g + 8 in o[2], o[3]
    const float r0c2 = __shfl_down_sync(FULL, o[0], 1);
    const float r8c2 = __shfl_down_sync(FULL, o[2], 1);
    if (FROM_GRAPH) {
      if (t == 0) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int64_t i = base + g + 8 * half;
          if (i >= count) continue;
          const float yv[3] = {half ? o[2] : o[0], half ? o[3] : o[1], half ? r8c2 : r0c2};
          float cost[3];
#pragma unroll
          for (int v = 0; v < 3; ++v) cost[v] = sNorm[16 + v] + sNorm[20 + v] * yv[v];
          uint8_t r = V_PROBE;
          const float other = fminf(cost[1], cost[2]);
          if (other + margin < cost[0]) r = cost[1] <= cost[2] ? V_MERGE : V_BSEARCH;
          G.route[i] = r;
        }
      }
    } else {
      const int64_t r0 = base + g, r8 = base + g + 8;
      if (t == 0) {
        if (r0 < count) { y[r0 * 3 + 0] = o[0]; y[r0 * 3 + 1] = o[1]; y[r0 * 3 + 2] = r0c2; }
        if (r8 < count) { y[r8 * 3 + 0] = o[2]; y[r8 * 3 + 1] = o[3]; y[r8 * 3 + 2] = r8c2; }
      }
    }
  }
}

static int infer_grid() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 4;
}

aot_status learned_routes(aot_graph* g, cudaStream_t s) {
  if (!g->model) return AOT_ERR_NOT_READY;
  const int T = 256;
  uint32_t* ip = reinterpret_cast<uint32_t*>(g->eplist);  // scratch until the lists are built
  AOT_KERNEL("k_item_pivot", s)
    k_item_pivot<<<(unsigned)(((int64_t)g->n * 32 + T - 1) / T), T, 0, s>>>(g->wofs, g->n, ip);
  AOT_TRY(last_launch());
  InferGraph G{ip, g->wvert, g->wedge, g->off, g->outdeg, g->degr, g->n, g->route};
  AOT_KERNEL("k_mlp_infer/route", s)
    k_mlp_infer<true><<<infer_grid(), 256, 0, s>>>(g->model, g->m, G, nullptr, nullptr);
  return last_launch();
}

// ------------------------------------------------------------- training
__global__ void k_train_in(const void* __restrict__ model, const float* __restrict__ x, int B,
                           float* __restrict__ xin) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * 8) return;
  const ModelView M = model_view(model);
  const int k = i & 7;
  xin[i] = bfr((x[i] - M.in_mean[k]) / M.in_std[k]);
}

// out[b][j] = act(bias[j] + sum_k in[b][k] * W[j][k]); thread per (b, j)
__global__ void k_dense_fwd(const void* __restrict__ model, int wofs, int bofs,
                            const float* __restrict__ in, int K, int N, int B,
                            float* __restrict__ z, float* __restrict__ h, bool relu) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * N) return;
  const int b = i / N, j = i % N;
  const ModelView M = model_view(model);
  float acc = __bfloat162float(M.prm[bofs + j]);
  for (int k = 0; k < K; ++k) acc = fmaf(in[b * K + k], __bfloat162float(M.prm[wofs + j * K + k]), acc);
  z[i] = acc;
  if (h) h[i] = relu ? bfr(fmaxf(acc, 0.f)) : acc;
}

__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ tgt, int B,
                       float* __restrict__ dy, float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < B * 3) {
    const float d = y[i] - tgt[i];
    dy[i] = 2.f * d / (float)B;
    l = d * d / (float)B;
  }
  l = warp_sum(l);
  if (lane_id() == 0 && l != 0.f) atomicAdd(loss, l);
}

// dW[j][k] = sum_b d[b][j] in[b][k]; k == K gives db[j]; thread per (j, k)
__global__ void k_dense_bwd_w(const float* __restrict__ d, const float* __restrict__ in, int K,
                              int N, int B, float* __restrict__ grad, int wofs, int bofs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * (K + 1)) return;
  const int j = i / (K + 1), k = i % (K + 1);
  float acc = 0.f;
  if (k < K)
    for (int b = 0; b < B; ++b) acc = fmaf(d[b * N + j], in[b * K + k], acc);
  else
    for (int b = 0; b < B; ++b) acc += d[b * N + j];
  if (k < K) grad[wofs + j * K + k] = acc;
  else grad[bofs + j] = acc;
}

// din[b][k] = [z[b][k] > 0] * sum_j d[b][j] W[j][k]; thread per (b, k)
__global__ void k_dense_bwd_in(const void* __restrict__ model, int wofs, const float* __restrict__ d,
                               int N, int K, int B, const float* __restrict__ z,
                               float* __restrict__ din) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * K) return;
  const int b = i / K, k = i % K;
  const ModelView M = model_view(model);
  float acc = 0.f;
  for (int j = 0; j < N; ++j) acc = fmaf(d[b * N + j], __bfloat162float(M.prm[wofs + j * K + k]), acc);
  din[i] = z[i] > 0.f ? acc : 0.f;
}

__global__ void k_adam(void* __restrict__ model, float* __restrict__ master, float* __restrict__ m1,
                       float* __restrict__ m2, const float* __restrict__ grad, int step, float lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P_TOTAL) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float gr = grad[i];
  const float a = b1 * m1[i] + (1.f - b1) * gr;
  const float v = b2 * m2[i] + (1.f - b2) * gr * gr;
  m1[i] = a;
  m2[i] = v;
  const float mh = a / (1.f - powf(b1, (float)step));
  const float vh = v / (1.f - powf(b2, (float)step));
  const float w = master[i] - lr * mh / (sqrtf(vh) + eps);
  master[i] = w;
  reinterpret_cast<__nv_bfloat16*>(static_cast<char*>(model) + MO_PARAMS)[i] = __float2bfloat16_rn(w);
}

struct TrainWs {
  float *xin, *z1, *h1, *z2, *h2, *y, *dy, *dh2, *dh1, *grad, *loss;
  size_t bytes;
};
static TrainWs carve_train(void* base, int B) {
  Carve c(base);
  TrainWs w;
  w.xin = c.take<float>((size_t)B * 8);
  w.z1 = c.take<float>((size_t)B * 64);
  w.h1 = c.take<float>((size_t)B * 64);
  w.z2 = c.take<float>((size_t)B * 64);
  w.h2 = c.take<float>((size_t)B * 64);
  w.y = c.take<float>((size_t)B * 3);
  w.dy = c.take<float>((size_t)B * 3);
  w.dh2 = c.take<float>((size_t)B * 64);
  w.dh1 = c.take<float>((size_t)B * 64);
  w.grad = c.take<float>(P_TOTAL);
  w.loss = c.take<float>(1);
  w.bytes = c.used();
  return w;
}

static inline unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace aot

using namespace aot;

extern "C" aot_status aot_mlp_train_workspace_size(int32_t batch, size_t* bytes) {
  if (!bytes || batch < 1 || batch > (1 << 20)) return AOT_ERR_INVALID_ARG;
  *bytes = carve_train(nullptr, batch).bytes;
  return AOT_OK;
}

extern "C" aot_status aot_mlp_forward(const void* d_model, const float* d_x, int64_t n, float* d_y,
                                      aot_stream_t stream) {
  if (!d_model || (n > 0 && (!d_x || !d_y)) || n < 0) return AOT_ERR_INVALID_ARG;
  if (n == 0) return AOT_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  InferGraph G{};
  AOT_KERNEL("k_mlp_infer/forward", s)
    k_mlp_infer<false><<<infer_grid(), 256, 0, s>>>(d_model, n, G, d_x, d_y);
  return last_launch();
}

extern "C" aot_status aot_mlp_train_step(void* d_model, float* d_master, float* d_m1, float* d_m2,
                                         int32_t step, float lr, const float* d_x, const float* d_t,
                                         int32_t batch, void* d_ws, size_t ws_bytes,
                                         float* d_grad_out, float* h_loss, aot_stream_t stream) {
  if (!d_model || !d_x || !d_t || batch < 1 || batch > (1 << 20)) return AOT_ERR_INVALID_ARG;
  if (lr > 0.f && (!d_master || !d_m1 || !d_m2 || step < 1)) return AOT_ERR_INVALID_ARG;
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255)) return AOT_ERR_WORKSPACE;
  TrainWs w = carve_train(d_ws, batch);
  if (ws_bytes < w.bytes) return AOT_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int B = batch;
  AOT_CUDA(cudaMemsetAsync(w.loss, 0, sizeof(float), s));
  AOT_KERNEL("k_train_in", s) k_train_in<<<blocks((int64_t)B * 8), 256, 0, s>>>(d_model, d_x, B, w.xin);
  AOT_TRY(last_launch());
  AOT_KERNEL("k_dense_fwd", s)
    k_dense_fwd<<<blocks((int64_t)B * 64), 256, 0, s>>>(d_model, P_W1, P_B1, w.xin, 8, 64, B, w.z1, w.h1, true);
  AOT_TRY(last_launch());
  AOT_KERNEL("k_dense_fwd", s)
    k_dense_fwd<<<blocks((int64_t)B * 64), 256, 0, s>>>(d_model, P_W2, P_B2, w.h1, 64, 64, B, w.z2, w.h2, true);
  AOT_TRY(last_launch());
  AOT_KERNEL("k_dense_fwd", s)
    k_dense_fwd<<<blocks((int64_t)B * 3), 256, 0, s>>>(d_model, P_W3, P_B3, w.h2, 64, 3, B, w.y, nullptr, false);
  AOT_TRY(last_launch());
  AOT_KERNEL("k_loss", s) k_loss<<<blocks((int64_t)B * 3), 256, 0, s>>>(w.y, d_t, B, w.dy, w.loss);
  AOT_TRY(last_launch());
  AOT_KERNEL("k_dense_bwd_w", s)
    k_dense_bwd_w<<<blocks(3 * 65), 256, 0, s>>>(w.dy, w.h2, 64, 3, B, w.grad, P_W3, P_B3);
  AOT_TRY(last_launch());
  AOT_KERNEL("k_dense_bwd_in", s)
    k_dense_bwd_in<<<blocks((int64_t)B * 64), 256, 0, s>>>(d_model, P_W3, w.dy, 3, 64, B, w.z2, w.dh2);
  AOT_TRY(last_launch());
  AOT_KERNEL("k_dense_bwd_w", s)
    k_dense_bwd_w<<<blocks(64 * 65), 256, 0, s>>>(w.dh2, w.h1, 64, 64, B, w.grad, P_W2, P_B2);
  AOT_TRY(last_launch());
  AOT_KERNEL("k_dense_bwd_in", s)
    k_dense_bwd_in<<<blocks((int64_t)B * 64), 256, 0, s>>>(d_model, P_W2, w.dh2, 64, 64, B, w.z1, w.dh1);
  AOT_TRY(last_launch());
  AOT_KERNEL("k_dense_bwd_w", s)
    k_dense_bwd_w<<<blocks(64 * 9), 256, 0, s>>>(w.dh1, w.xin, 8, 64, B, w.grad, P_W1, P_B1);
  AOT_TRY(last_launch());
  if (d_grad_out)
    AOT_CUDA(cudaMemcpyAsync(d_grad_out, w.grad, sizeof(float) * P_TOTAL, cudaMemcpyDeviceToDevice, s));
  if (lr > 0.f) {
    AOT_KERNEL("k_adam", s)
      k_adam<<<blocks(P_TOTAL), 256, 0, s>>>(d_model, d_master, d_m1, d_m2, w.grad, step, lr);
    AOT_TRY(last_launch());
  }
  if (h_loss) {
    AOT_CUDA(cudaMemcpyAsync(h_loss, w.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    AOT_CUDA(cudaStreamSynchronize(s));
  }
  return AOT_OK;
}

extern "C" aot_status aot_graph_features(aot_graph* g, float* d_feat, aot_stream_t stream) {
  if (!g || (g->m > 0 && !d_feat)) return AOT_ERR_INVALID_ARG;
  if (g->flags & AOT_FLAG_LOCAL_RANDOM) return AOT_ERR_INVALID_ARG;  // suffix lengths need sorted lists
  if (g->m == 0) return AOT_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int T = 256;
  uint32_t* ip = reinterpret_cast<uint32_t*>(g->eplist);
  AOT_KERNEL("k_item_pivot", s)
    k_item_pivot<<<(unsigned)(((int64_t)g->n * 32 + T - 1) / T), T, 0, s>>>(g->wofs, g->n, ip);
  AOT_TRY(last_launch());
  AOT_KERNEL("k_features", s)
    k_features<<<blocks(g->m), T, 0, s>>>(ip, g->wvert, g->wedge, g->m, g->off, g->outdeg, g->degr,
                                          g->n, d_feat);
  return last_launch();
}

extern "C" aot_status aot_graph_set_router(aot_graph* g, const void* d_model) {
  if (!g) return AOT_ERR_INVALID_ARG;
  if (d_model && (reinterpret_cast<uintptr_t>(d_model) & 15)) return AOT_ERR_INVALID_ARG;
  g->model = d_model;
  return AOT_OK;
}
