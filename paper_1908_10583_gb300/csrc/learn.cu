// Learned r_max: per-source features and a 16-64-64-1 MLP with BF16 weights and
// activations and FP32 accumulation, with hand-written forward, backward and Adam
// kernels.  The network predicts log2(r_max / r_rule) for a source; the query then uses
// r_max = r_rule * 2^prediction.  Any r_max keeps the accuracy guarantee of Lemma
// (layerppr-conc) (omega scales with r_sum), so the network only trades push work
// against walk work, as the balancing of Section 4.2 does with timing.
//
// Parameter vector (FP32 masters, kNumParams floats):
//   W1 [64][16] | b1 [64] | W2 [64][64] | b2 [64] | W3 [64] | b3
// Forward for one sample (every product accumulated in FP32):
//   x  = bf16((f - mu) / sigma)
//   z1 = bf16(W1) x + bf16(b1),  h1 = bf16(relu(z1))
//   z2 = bf16(W2) h1 + bf16(b2), h2 = bf16(relu(z2))
//   y  = bf16(W3) . h2 + bf16(b3)
// Loss 0.5 * mean (y - t)^2; gradients w.r.t. the BF16 weights are applied to the
// FP32 masters (Adam).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "fora.h"
#include "fora_engine.cuh"

namespace fora {

namespace {

constexpr int kIn = FORA_NUM_FEATURES;
constexpr int kHid = 64;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid;
constexpr int kNumParams = kOffB3 + 1;
static_assert(kNumParams == FORA_MODEL_PARAMS, "parameter count");
constexpr int kTile = 64;  // samples per block in the backward kernel

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---------------------------------------------------------------- features

// Warp per source.  Sums of integer degrees are exact in FP64.
__global__ void k_features(GraphDev g, const uint32_t* __restrict__ indeg,
                           const int32_t* __restrict__ sources, int nsrc, double alpha,
                           double rmax_rule, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= nsrc) return;
  const uint32_t s = (uint32_t)sources[w];
  const uint32_t rb = g.row[s], d = g.row[s + 1] - rb;
  const double inc = (1.0 - alpha) / (double)d;  // residue one edge carries in round 1
  double sum_out = 0.0, sum_in = 0.0, f1 = 0.0, f1_edges = 0.0;
  for (uint32_t e = lane; e < d; e += 32) {
    const uint32_t u = (uint32_t)g.col[rb + e];
    const uint32_t du = g.row[u + 1] - g.row[u];
    sum_out += (double)du;
    sum_in += (double)indeg[u];
    if (inc > rmax_rule * (double)du) {
      f1 += 1.0;
      f1_edges += (double)du;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum_out += __shfl_down_sync(0xFFFFFFFFu, sum_out, o);
    sum_in += __shfl_down_sync(0xFFFFFFFFu, sum_in, o);
    f1 += __shfl_down_sync(0xFFFFFFFFu, f1, o);
    f1_edges += __shfl_down_sync(0xFFFFFFFFu, f1_edges, o);
  }
  if (lane == 0) {
    float* f = out + (size_t)w * kIn;
    f[0] = (float)log1p((double)d);
    f[1] = (float)log1p((double)indeg[s]);
    f[2] = (float)log1p(sum_out);
    f[3] = (float)log1p(sum_in);
    f[4] = (float)log1p(f1);
    f[5] = (float)log1p(f1_edges);
    f[6] = (float)log(rmax_rule * (double)g.m);
    f[7] = (float)log((double)g.m / (double)g.n);
    for (int i = 8; i < kIn; ++i) f[i] = 0.0f;
  }
}

__global__ void k_indegree(GraphDev g, uint32_t* indeg) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       e < (unsigned long long)g.m; e += stride)
    atomicAdd(&indeg[g.col[e]], 1u);
}

// ---------------------------------------------------------------- network

// Loads the BF16-rounded parameters into shared memory as floats.
__device__ __forceinline__ void load_params(const float* __restrict__ master, float* sp) {
  for (int i = threadIdx.x; i < kNumParams; i += blockDim.x) sp[i] = bf(master[i]);
}

struct Act {  // one sample's activations (BF16-rounded values held as floats)
  float x[kIn];
  float h1[kHid];
  float h2[kHid];
};

__device__ __forceinline__ float forward_one(const float* sp, const float* __restrict__ f,
                                             const float* __restrict__ norm, float* x, float* z1,
                                             float* h1, float* z2, float* h2) {
#pragma unroll
  for (int i = 0; i < kIn; ++i) x[i] = bf(__fdiv_rn(__fsub_rn(f[i], norm[i]), norm[kIn + i]));
  for (int j = 0; j < kHid; ++j) {
    float a = sp[kOffB1 + j];
#pragma unroll
    for (int i = 0; i < kIn; ++i) a = __fmaf_rn(sp[kOffW1 + j * kIn + i], x[i], a);
    z1[j] = a;
    h1[j] = bf(fmaxf(a, 0.0f));
  }
  for (int j = 0; j < kHid; ++j) {
    float a = sp[kOffB2 + j];
    for (int i = 0; i < kHid; ++i) a = __fmaf_rn(sp[kOffW2 + j * kHid + i], h1[i], a);
    z2[j] = a;
    h2[j] = bf(fmaxf(a, 0.0f));
  }
  float y = sp[kOffB3];
  for (int i = 0; i < kHid; ++i) y = __fmaf_rn(sp[kOffW3 + i], h2[i], y);
  return y;
}

__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ master,
                                                     const float* __restrict__ norm,
                                                     const float* __restrict__ X, int n,
                                                     float* __restrict__ Y) {
  extern __shared__ float sp[];
  load_params(master, sp);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x[kIn], z1[kHid], h1[kHid], z2[kHid], h2[kHid];
  Y[i] = forward_one(sp, X + (size_t)i * kIn, norm, x, z1, h1, z2, h2);
}

// Forward and backward of one tile of kTile samples (rows idx[tile*kTile ...] of X, T).
// Per-sample backward in threads 0..kTile-1, then every thread reduces the weight
// gradients over the tile in a fixed order; the tile's gradient goes to partial[tile].
__global__ void __launch_bounds__(256) k_mlp_backward(const float* __restrict__ master,
                                                      const float* __restrict__ norm,
                                                      const float* __restrict__ X,
                                                      const float* __restrict__ T,
                                                      const int32_t* __restrict__ idx, int n,
                                                      float inv_batch, float* __restrict__ partial,
                                                      float* __restrict__ loss_partial) {
  extern __shared__ float smem[];
  float* sp = smem;                          // kNumParams
  float* sx = sp + kNumParams;               // [kTile][kIn]
  float* sh1 = sx + kTile * kIn;             // [kTile][kHid]
  float* sh2 = sh1 + kTile * kHid;           // [kTile][kHid]
  float* sd1 = sh2 + kTile * kHid;           // dz1 [kTile][kHid]
  float* sd2 = sd1 + kTile * kHid;           // dz2 [kTile][kHid]
  float* sdy = sd2 + kTile * kHid;           // dy [kTile]
  load_params(master, sp);
  __syncthreads();
  const int t = threadIdx.x;
  const int first = blockIdx.x * kTile;
  const int cnt = min(kTile, n - first);
  if (t < kTile) {
    float x[kIn], z1[kHid], h1[kHid], z2[kHid], h2[kHid];
    float dy = 0.0f;
    if (t < cnt) {
      const int row = idx ? idx[first + t] : first + t;
      const float y = forward_one(sp, X + (size_t)row * kIn, norm, x, z1, h1, z2, h2);
      const float err = __fsub_rn(y, T[row]);
      dy = __fmul_rn(err, inv_batch);
      sdy[t] = dy;
      loss_partial[first + t] = __fmul_rn(0.5f, __fmul_rn(err, err));
    } else {
      for (int i = 0; i < kIn; ++i) x[i] = 0.0f;
      for (int j = 0; j < kHid; ++j) { z1[j] = 0.0f; h1[j] = 0.0f; z2[j] = 0.0f; h2[j] = 0.0f; }
      sdy[t] = 0.0f;
    }
    for (int i = 0; i < kIn; ++i) sx[t * kIn + i] = x[i];
    for (int j = 0; j < kHid; ++j) {
      sh1[t * kHid + j] = h1[j];
      sh2[t * kHid + j] = h2[j];
    }
    // dz2 = dy * W3 * [z2 > 0]; dz1 = (W2^T dz2) * [z1 > 0]
    float dz2[kHid];
    for (int j = 0; j < kHid; ++j) {
      dz2[j] = z2[j] > 0.0f ? __fmul_rn(dy, sp[kOffW3 + j]) : 0.0f;
      sd2[t * kHid + j] = dz2[j];
    }
    for (int i = 0; i < kHid; ++i) {
      float a = 0.0f;
      for (int j = 0; j < kHid; ++j) a = __fmaf_rn(sp[kOffW2 + j * kHid + i], dz2[j], a);
      sd1[t * kHid + i] = z1[i] > 0.0f ? a : 0.0f;
    }
  }
  __syncthreads();
  // weight gradients summed over the tile, samples in order
  float* out = partial + (size_t)blockIdx.x * kNumParams;
  for (int p = t; p < kNumParams; p += blockDim.x) {
    float a = 0.0f;
    if (p < kOffB1) {  // W1[j][i] += dz1[j] x[i]
      const int j = (p - kOffW1) / kIn, i = (p - kOffW1) % kIn;
      for (int b = 0; b < kTile; ++b) a = __fmaf_rn(sd1[b * kHid + j], sx[b * kIn + i], a);
    } else if (p < kOffW2) {  // b1
      const int j = p - kOffB1;
      for (int b = 0; b < kTile; ++b) a = __fadd_rn(a, sd1[b * kHid + j]);
    } else if (p < kOffB2) {  // W2[j][i] += dz2[j] h1[i]
      const int j = (p - kOffW2) / kHid, i = (p - kOffW2) % kHid;
      for (int b = 0; b < kTile; ++b) a = __fmaf_rn(sd2[b * kHid + j], sh1[b * kHid + i], a);
    } else if (p < kOffW3) {  // b2
      const int j = p - kOffB2;
      for (int b = 0; b < kTile; ++b) a = __fadd_rn(a, sd2[b * kHid + j]);
    } else if (p < kOffB3) {  // W3[i] += dy h2[i]
      const int i = p - kOffW3;
      for (int b = 0; b < kTile; ++b) a = __fmaf_rn(sdy[b], sh2[b * kHid + i], a);
    } else {  // b3
      for (int b = 0; b < kTile; ++b) a = __fadd_rn(a, sdy[b]);
    }
    out[p] = a;
  }
}

// grad[p] = sum over tiles (in tile order) of partial[tile][p]
__global__ void k_mlp_reduce(const float* __restrict__ partial, int tiles, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNumParams) return;
  float a = 0.0f;
  for (int t = 0; t < tiles; ++t) a = __fadd_rn(a, partial[(size_t)t * kNumParams + p]);
  grad[p] = a;
}

__global__ void k_adam(float* __restrict__ master, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ grad, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNumParams) return;
  const float gr = grad[p];
  const float mp = b1 * m[p] + (1.0f - b1) * gr;
  const float vp = b2 * v[p] + (1.0f - b2) * gr * gr;
  m[p] = mp;
  v[p] = vp;
  master[p] -= lr * (mp / c1) / (sqrtf(vp / c2) + eps);
}

__global__ void k_pred_to_rmax(const float* __restrict__ pred, int n, double rmax_rule, float lo,
                               float hi, double* __restrict__ rmax) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float p = fminf(fmaxf(pred[i], lo), hi);
  rmax[i] = rmax_rule * exp2((double)p);
}

size_t backward_smem_bytes() {
  return sizeof(float) * (kNumParams + kTile * kIn + 4 * kTile * kHid + kTile);
}

}  // namespace

cudaError_t launch_indegree(const GraphDev& g, uint32_t* indeg, int num_sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(indeg, 0, (size_t)g.n * sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  k_indegree<<<num_sms * 8, 256, 0, st>>>(g, indeg);
  return cudaGetLastError();
}

cudaError_t launch_features(const GraphDev& g, const uint32_t* indeg, const int32_t* sources,
                            int nsrc, double alpha, double rmax_rule, float* out, cudaStream_t st) {
  if (nsrc <= 0) return cudaSuccess;
  const int warps_per_block = 8;
  k_features<<<(nsrc + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
      g, indeg, sources, nsrc, alpha, rmax_rule, out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float* master, const float* norm, const float* X, int n,
                               float* Y, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const size_t smem = sizeof(float) * kNumParams;
  k_mlp_forward<<<(n + 127) / 128, 128, smem, st>>>(master, norm, X, n, Y);
  return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const float* master, const float* norm, const float* X,
                            const float* T, const int32_t* idx, int n, float* partial,
                            float* loss_partial, float* grad, cudaStream_t st) {
  const size_t smem = backward_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles = (n + kTile - 1) / kTile;
  k_mlp_backward<<<tiles, 256, smem, st>>>(master, norm, X, T, idx, n, 1.0f / (float)n, partial,
                                           loss_partial);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mlp_reduce<<<(kNumParams + 255) / 256, 256, 0, st>>>(partial, tiles, grad);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* master, float* m, float* v, const float* grad, int step, float lr,
                        cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adam<<<(kNumParams + 255) / 256, 256, 0, st>>>(master, m, v, grad, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_pred_to_rmax(const float* pred, int n, double rmax_rule, float lo, float hi,
                                double* rmax, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_pred_to_rmax<<<(n + 255) / 256, 256, 0, st>>>(pred, n, rmax_rule, lo, hi, rmax);
  return cudaGetLastError();
}

int mlp_tile() { return kTile; }

}  // namespace fora
