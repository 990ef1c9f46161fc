// cnn.cu -- the learned proposal's 3-layer CNN (not in the paper):
// conv3x3(1->16)-ReLU-conv3x3(16->16)-ReLU-conv3x3(16->1), zero padding,
// activations [B][C][H][W] FP32.  Weights are an FP32 master vector; with
// bf16 = 1 every kernel rounds them to BF16 as it stages them (the inference
// weights), accumulating in FP32.  Forward, backward (data and weight
// gradients), BCE-with-logits and Adam are hand-written kernels.
#include <cuda_bf16.h>

#include "internal.h"

namespace ofdm {
namespace {

constexpr int kTile = 16;                   // 16 x 16 output pixels per CTA
constexpr int kHalo = kTile + 2;
constexpr int kMaxC = 16;

// Offsets of the parameter blocks in the flat vector.
constexpr int kW1 = 0, kB1 = kW1 + 16 * 1 * 9, kW2 = kB1 + 16, kB2 = kW2 + 16 * 16 * 9, kW3 = kB2 + 16,
              kB3 = kW3 + 1 * 16 * 9, kNParams = kB3 + 1;

__device__ __forceinline__ float wval(const float* w, int i, int bf16) {
  const float v = w[i];
  return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}

// y[b][o] = conv(x[b], w) + bias, optionally ReLU (Ci, Co <= 16), used by
// inference and training: 16 x 16 output pixels per CTA, 64 threads of 1 x 4
// pixels each, so every weight read from shared memory serves four
// multiply-adds (the 16 -> 16 layer reads 2304 weights per pixel).  Each
// output sums over (c, dy, dx) in that order.
constexpr int kPx = 4;                       // pixels per thread (along x)
template <int CI, int CO>
__global__ void __launch_bounds__(kTile * kTile / kPx)
conv3x3_fwd_x4(const float* __restrict__ x, const float* __restrict__ w, const float* __restrict__ bias,
               float* __restrict__ y, int H, int W, int relu, int bf16) {
  __shared__ float sx[CI][kHalo][kHalo];
  __shared__ float sw[CO * CI * 9];
  const int b = blockIdx.z;
  const int ty = threadIdx.x / (kTile / kPx), tx0 = (threadIdx.x % (kTile / kPx)) * kPx;
  const int y0 = blockIdx.y * kTile, x0 = blockIdx.x * kTile;
  for (int i = threadIdx.x; i < CO * CI * 9; i += blockDim.x) sw[i] = wval(w, i, bf16);
  for (int i = threadIdx.x; i < CI * kHalo * kHalo; i += blockDim.x) {
    const int c = i / (kHalo * kHalo), r = (i / kHalo) % kHalo, q = i % kHalo;
    const int gy = y0 + r - 1, gx = x0 + q - 1;
    sx[c][r][q] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? x[(((long)b * CI + c) * H + gy) * W + gx] : 0.f;
  }
  __syncthreads();
  const int gy = y0 + ty;
  if (gy >= H) return;
  float acc[kPx][CO];
#pragma unroll
  for (int p = 0; p < kPx; ++p)
#pragma unroll
    for (int o = 0; o < CO; ++o) acc[p][o] = 0.f;
#pragma unroll 2
  for (int c = 0; c < CI; ++c)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
      float v[kPx + 2];
#pragma unroll
      for (int q = 0; q < kPx + 2; ++q) v[q] = sx[c][ty + dy][tx0 + q];
#pragma unroll
      for (int dx = 0; dx < 3; ++dx)
#pragma unroll
        for (int o = 0; o < CO; ++o) {
          const float wt = sw[(o * CI + c) * 9 + dy * 3 + dx];
#pragma unroll
          for (int p = 0; p < kPx; ++p) acc[p][o] = fmaf(wt, v[p + dx], acc[p][o]);
        }
    }
#pragma unroll
  for (int p = 0; p < kPx; ++p) {
    const int gx = x0 + tx0 + p;
    if (gx >= W) continue;
#pragma unroll
    for (int o = 0; o < CO; ++o) {
      float val = acc[p][o] + bias[o];
      if (relu) val = fmaxf(val, 0.f);
      y[(((long)b * CO + o) * H + gy) * W + gx] = val;
    }
  }
}

// gx[b][c] = sum_o sum_k w[o][c][k] * gy[b][o](shifted), times (act > 0) if act != null.
__global__ void __launch_bounds__(kTile * kTile)
conv3x3_bwd_data(const float* __restrict__ gy, const float* __restrict__ w, const float* __restrict__ act,
                 float* __restrict__ gx, int Ci, int Co, int H, int W, int bf16) {
  __shared__ float sg[kMaxC][kHalo][kHalo];
  __shared__ float sw[kMaxC * kMaxC * 9];
  const int b = blockIdx.z;
  const int ty = threadIdx.x / kTile, tx = threadIdx.x % kTile;
  const int y0 = blockIdx.y * kTile, x0 = blockIdx.x * kTile;
  for (int i = threadIdx.x; i < Co * Ci * 9; i += blockDim.x) sw[i] = wval(w, i, bf16);
  for (int i = threadIdx.x; i < Co * kHalo * kHalo; i += blockDim.x) {
    const int o = i / (kHalo * kHalo), r = (i / kHalo) % kHalo, q = i % kHalo;
    const int yy = y0 + r - 1, xx = x0 + q - 1;
    sg[o][r][q] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? gy[(((long)b * Co + o) * H + yy) * W + xx] : 0.f;
  }
  __syncthreads();
  const int py = y0 + ty, px = x0 + tx;
  if (py >= H || px >= W) return;
  // input pixel (py, px) feeds output (py - dy + 1, px - dx + 1) through tap (dy, dx)
  for (int c = 0; c < Ci; ++c) {
    float acc = 0.f;
    for (int o = 0; o < Co; ++o)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
          acc = fmaf(sw[(o * Ci + c) * 9 + dy * 3 + dx], sg[o][ty + 2 - dy][tx + 2 - dx], acc);
    const long idx = (((long)b * Ci + c) * H + py) * W + px;
    if (act) acc = act[idx] > 0.f ? acc : 0.f;
    gx[idx] = acc;
  }
}

// gw[o][c][k] += sum over the tile of gy[b][o] * x[b][c](shifted); gb[o] += sum gy[b][o].
__global__ void __launch_bounds__(kTile * kTile)
conv3x3_bwd_weight(const float* __restrict__ x, const float* __restrict__ gy, float* __restrict__ gw,
                   float* __restrict__ gb, int Ci, int Co, int H, int W) {
  __shared__ float sx[kMaxC][kHalo][kHalo];
  __shared__ float sg[kMaxC][kTile][kTile];
  const int b = blockIdx.z;
  const int y0 = blockIdx.y * kTile, x0 = blockIdx.x * kTile;
  for (int i = threadIdx.x; i < Ci * kHalo * kHalo; i += blockDim.x) {
    const int c = i / (kHalo * kHalo), r = (i / kHalo) % kHalo, q = i % kHalo;
    const int yy = y0 + r - 1, xx = x0 + q - 1;
    sx[c][r][q] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? x[(((long)b * Ci + c) * H + yy) * W + xx] : 0.f;
  }
  for (int i = threadIdx.x; i < Co * kTile * kTile; i += blockDim.x) {
    const int o = i / (kTile * kTile), r = (i / kTile) % kTile, q = i % kTile;
    const int yy = y0 + r, xx = x0 + q;
    sg[o][r][q] = (yy < H && xx < W) ? gy[(((long)b * Co + o) * H + yy) * W + xx] : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < Co * Ci * 9 + Co; k += blockDim.x) {
    float acc = 0.f;
    if (k < Co * Ci * 9) {
      const int o = k / (Ci * 9), c = (k / 9) % Ci, t = k % 9, dy = t / 3, dx = t % 3;
      for (int r = 0; r < kTile; ++r)
        for (int q = 0; q < kTile; ++q) acc = fmaf(sg[o][r][q], sx[c][r + dy][q + dx], acc);
      atomicAdd(gw + k, acc);
    } else {
      const int o = k - Co * Ci * 9;
      for (int r = 0; r < kTile; ++r)
        for (int q = 0; q < kTile; ++q) acc += sg[o][r][q];
      atomicAdd(gb + o, acc);
    }
  }
}

// Mean BCE with logits; loss accumulated into *loss, gradient written.
__global__ void bce_kernel(const float* __restrict__ z, const float* __restrict__ lab, int n, float pw,
                           float* __restrict__ loss, float* __restrict__ g) {
  float part = 0.f;
  const float inv = 1.f / (float)n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float zi = z[i], yi = lab[i];
    // log sigmoid(z) = -softplus(-z), log(1 - sigmoid(z)) = -softplus(z)
    const float sp_neg = fmaxf(-zi, 0.f) + log1pf(expf(-fabsf(zi)));
    const float sp_pos = fmaxf(zi, 0.f) + log1pf(expf(-fabsf(zi)));
    part += pw * yi * sp_neg + (1.f - yi) * sp_pos;
    const float s = 1.f / (1.f + expf(-zi));
    g[i] = (pw * yi * (s - 1.f) + (1.f - yi) * s) * inv;
  }
  for (int off = 16; off; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, part * inv);
}

__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

dim3 conv_grid(int B, int H, int W) { return dim3((W + kTile - 1) / kTile, (H + kTile - 1) / kTile, B); }

}  // namespace

cudaError_t cnn_forward(const float* th, int bf16, const float* x, int B, int H, int W, float* a1, float* a2,
                        float* z, cudaStream_t s) {
  const dim3 g = conv_grid(B, H, W);
  constexpr int T = kTile * kTile / kPx;
  conv3x3_fwd_x4<1, 16><<<g, T, 0, s>>>(x, th + kW1, th + kB1, a1, H, W, 1, bf16);
  conv3x3_fwd_x4<16, 16><<<g, T, 0, s>>>(a1, th + kW2, th + kB2, a2, H, W, 1, bf16);
  conv3x3_fwd_x4<16, 1><<<g, T, 0, s>>>(a2, th + kW3, th + kB3, z, H, W, 0, bf16);
  return cudaGetLastError();
}

}  // namespace ofdm

extern "C" {

int ofdm_cnn_param_count(void) { return ofdm::kNParams; }

int ofdm_cnn_forward(const float* theta, int32_t bf16, const float* x, int32_t B, int32_t H, int32_t W, float* a1,
                     float* a2, float* logits, void* stream) {
  if (!theta || !x || !a1 || !a2 || !logits || B < 1 || H < 1 || W < 1) return OFDM_ERR_INVALID_ARG;
  return ofdm::cnn_forward(theta, bf16, x, B, H, W, a1, a2, logits, (cudaStream_t)stream) == cudaSuccess
             ? OFDM_OK : OFDM_ERR_CUDA;
}

int ofdm_cnn_backward(const float* theta, int32_t bf16, const float* x, const float* a1, const float* a2,
                      const float* glogits, int32_t B, int32_t H, int32_t W, float* ga1, float* ga2,
                      float* gtheta, void* stream) {
  using namespace ofdm;
  if (!theta || !x || !a1 || !a2 || !glogits || !ga1 || !ga2 || !gtheta || B < 1 || H < 1 || W < 1)
    return OFDM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const dim3 g = conv_grid(B, H, W);
  cudaError_t e = cudaMemsetAsync(gtheta, 0, kNParams * sizeof(float), s);
  if (e != cudaSuccess) return OFDM_ERR_CUDA;
  // layer 3: z = conv(a2, w3)
  conv3x3_bwd_weight<<<g, kTile * kTile, 0, s>>>(a2, glogits, gtheta + kW3, gtheta + kB3, 16, 1, H, W);
  conv3x3_bwd_data<<<g, kTile * kTile, 0, s>>>(glogits, theta + kW3, a2, ga2, 16, 1, H, W, bf16);
  // layer 2: a2 = relu(conv(a1, w2)); ga2 already masked by (a2 > 0)
  conv3x3_bwd_weight<<<g, kTile * kTile, 0, s>>>(a1, ga2, gtheta + kW2, gtheta + kB2, 16, 16, H, W);
  conv3x3_bwd_data<<<g, kTile * kTile, 0, s>>>(ga2, theta + kW2, a1, ga1, 16, 16, H, W, bf16);
  // layer 1: a1 = relu(conv(x, w1))
  conv3x3_bwd_weight<<<g, kTile * kTile, 0, s>>>(x, ga1, gtheta + kW1, gtheta + kB1, 1, 16, H, W);
  return cudaGetLastError() == cudaSuccess ? OFDM_OK : OFDM_ERR_CUDA;
}

int ofdm_cnn_bce(const float* logits, const float* labels, int32_t n, float pos_weight, float* loss,
                 float* glogits, void* stream) {
  if (!logits || !labels || !loss || !glogits || n < 1) return OFDM_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return OFDM_ERR_CUDA;
  ofdm::bce_kernel<<<256, 256, 0, s>>>(logits, labels, n, pos_weight, loss, glogits);
  return cudaGetLastError() == cudaSuccess ? OFDM_OK : OFDM_ERR_CUDA;
}

int ofdm_cnn_adam(float* theta, const float* g, float* m, float* v, int32_t n, int32_t step, float lr, float b1,
                  float b2, float eps, void* stream) {
  if (!theta || !g || !m || !v || n < 1 || step < 1) return OFDM_ERR_INVALID_ARG;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  ofdm::adam_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(theta, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? OFDM_OK : OFDM_ERR_CUDA;
}

}  // extern "C"
