// The learned cost model of the tuner: a 4 -> 64 -> 64 -> 1 perceptron
// (ReLU hidden layers) mapping standardized (log m, log n, NB/512, IB/256)
// to log(seconds), trained with mean squared error and Adam, in FP32.
//
// The paper tunes purely empirically and argues that models of multicore
// performance are unreliable (Secs. 1 and 2.3); here the model only ranks
// candidates, and the measured time keeps the final say.
//
// Parameters live in one flat FP32 array: W1 (64 x 4, row-major [out][in]),
// b1 (64), W2 (64 x 64), b2 (64), W3 (1 x 64), b3 (1).
#include <cuda_runtime.h>

#include <cstdint>

#include "tileqr_internal.h"

namespace {

constexpr int H = 64;
constexpr int OFF_W1 = 0, OFF_B1 = 256, OFF_W2 = 320, OFF_B2 = 4416, OFF_W3 = 4480, OFF_B3 = 4544;
constexpr int NP = 4545;
constexpr int SAMPLES_PER_CTA = 32;

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 64 threads; thread j owns hidden unit j of both layers.
// mode 0: forward only (out[s] = prediction). mode 1: forward + backward,
// per-CTA partial gradients of mean((yhat - y)^2) into part[blockIdx.x][NP]
// and the partial loss into part[blockIdx.x][NP].
__global__ void __launch_bounds__(H) mlp_kernel(int nsamp, const float* __restrict__ X, const float* __restrict__ y,
                                                const float* __restrict__ P, float* out, float* part, int mode) {
  __shared__ float W2s[H * H];
  __shared__ float h1s[H], dz2s[H], red[2];
  const int j = threadIdx.x;
  for (int e = j; e < H * H; e += H) W2s[e] = P[OFF_W2 + e];
  float w1[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) w1[i] = P[OFF_W1 + j * 4 + i];
  const float b1 = P[OFF_B1 + j], b2 = P[OFF_B2 + j], w3 = P[OFF_W3 + j], b3 = P[OFF_B3];
  float gW2[H];
#pragma unroll
  for (int i = 0; i < H; ++i) gW2[i] = 0.f;
  float gW1[4] = {0.f, 0.f, 0.f, 0.f};
  float gb1 = 0.f, gb2 = 0.f, gW3 = 0.f, gb3 = 0.f, loss = 0.f;
  __syncthreads();
  const int s0 = blockIdx.x * SAMPLES_PER_CTA;
  const int s1 = min(nsamp, s0 + SAMPLES_PER_CTA);
  const float inv = 2.f / (float)nsamp;
  for (int s = s0; s < s1; ++s) {
    float x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = X[s * 4 + i];
    float z1 = b1;
#pragma unroll
    for (int i = 0; i < 4; ++i) z1 = fmaf(w1[i], x[i], z1);
    const float h1 = fmaxf(z1, 0.f);
    h1s[j] = h1;
    __syncthreads();
    float z2 = b2;
#pragma unroll 8
    for (int i = 0; i < H; ++i) z2 = fmaf(W2s[j * H + i], h1s[i], z2);
    const float h2 = fmaxf(z2, 0.f);
    float yh = wsum(w3 * h2);
    if ((j & 31) == 0) red[j >> 5] = yh;
    __syncthreads();
    yh = red[0] + red[1] + b3;
    if (mode == 0) {
      if (j == 0) out[s] = yh;
      __syncthreads();
      continue;
    }
    const float r = yh - y[s];
    loss += r * r;
    const float dy = inv * r;
    gW3 = fmaf(dy, h2, gW3);
    gb3 += dy;
    const float dz2 = (z2 > 0.f) ? dy * w3 : 0.f;
    gb2 += dz2;
#pragma unroll
    for (int i = 0; i < H; ++i) gW2[i] = fmaf(dz2, h1s[i], gW2[i]);
    dz2s[j] = dz2;
    __syncthreads();
    float dh1 = 0.f;
#pragma unroll 8
    for (int q = 0; q < H; ++q) dh1 = fmaf(W2s[q * H + j], dz2s[q], dh1);
    const float dz1 = (z1 > 0.f) ? dh1 : 0.f;
    gb1 += dz1;
#pragma unroll
    for (int i = 0; i < 4; ++i) gW1[i] = fmaf(dz1, x[i], gW1[i]);
    __syncthreads();
  }
  if (mode == 0) return;
  float* g = part + (size_t)blockIdx.x * (NP + 1);
#pragma unroll
  for (int i = 0; i < 4; ++i) g[OFF_W1 + j * 4 + i] = gW1[i];
  g[OFF_B1 + j] = gb1;
#pragma unroll
  for (int i = 0; i < H; ++i) g[OFF_W2 + j * H + i] = gW2[i];
  g[OFF_B2 + j] = gb2;
  g[OFF_W3 + j] = gW3;
  if (j == 0) {
    g[OFF_B3] = gb3;
    g[NP] = loss / (float)nsamp;
  }
}

// grads[e] = sum over CTAs of part[cta][e] (e < NP + 1: last = loss)
__global__ void mlp_reduce(int nblk, const float* part, float* grads) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > NP) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * (NP + 1) + e];
  grads[e] = s;
}

// Adam (Kingma & Ba 2015) with bias correction; step t counts from 1.
__global__ void mlp_adam(const float* g, float* p, float* m, float* v, int t, float lr, float b1, float b2, float eps) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NP) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.f - b1) * gi;
  const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  const float mh = mi / (1.f - powf(b1, (float)t));
  const float vh = vi / (1.f - powf(b2, (float)t));
  p[e] -= lr * mh / (sqrtf(vh) + eps);
}

int nblocks(int nsamp) { return (nsamp + SAMPLES_PER_CTA - 1) / SAMPLES_PER_CTA; }

}  // namespace

extern "C" {

int qr_mlp_workspace(int nsamp, int64_t* floats) {
  if (nsamp < 1) return -1;
  if (!floats) return -2;
  *floats = (int64_t)nblocks(nsamp) * (NP + 1) + (NP + 1);
  return 0;
}

int qr_mlp_forward(int nsamp, const float* X, const float* params, float* out, void* stream) {
  if (nsamp < 0) return -1;
  if (nsamp == 0) return 0;
  if (!X) return -2;
  if (!params) return -3;
  if (!out) return -4;
  mlp_kernel<<<nblocks(nsamp), H, 0, (cudaStream_t)stream>>>(nsamp, X, nullptr, params, out, nullptr, 0);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

int qr_mlp_grad(int nsamp, const float* X, const float* y, const float* params, float* grads, float* work,
                void* stream) {
  if (nsamp < 1) return -1;
  if (!X) return -2;
  if (!y) return -3;
  if (!params) return -4;
  if (!grads) return -5;
  if (!work) return -6;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = nblocks(nsamp);
  mlp_kernel<<<nb, H, 0, st>>>(nsamp, X, y, params, nullptr, work, 1);
  mlp_reduce<<<(NP + 1 + 255) / 256, 256, 0, st>>>(nb, work, grads);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

int qr_mlp_adam_step(const float* grads, float* params, float* m, float* v, int t, float lr, void* stream) {
  if (!grads) return -1;
  if (!params) return -2;
  if (!m) return -3;
  if (!v) return -4;
  if (t < 1) return -5;
  mlp_adam<<<(NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(grads, params, m, v, t, lr, 0.9f, 0.999f, 1e-8f);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

int qr_mlp_train(int nsamp, const float* X, const float* y, float* params, float* m, float* v, int steps, float lr,
                 float* grads, float* work, void* stream) {
  if (nsamp < 1) return -1;
  if (steps < 0) return -7;
  for (int t = 1; t <= steps; ++t) {
    int rc = qr_mlp_grad(nsamp, X, y, params, grads, work, stream);
    if (rc) return rc;
    rc = qr_mlp_adam_step(grads, params, m, v, t, lr, stream);
    if (rc) return rc;
  }
  return 0;
}

}  // extern "C"
