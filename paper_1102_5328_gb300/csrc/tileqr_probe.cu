// Live FP64 throughput probe (qr_peak_fp64): the roofline reference for the
// factorization kernels, measured at the clocks the benchmark runs at.
#include <cuda_runtime.h>

#include <cstdint>

#include "tileqr_internal.h"

namespace {

__global__ void dfma_probe(double* sink, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
         x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  const double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == 1234.5) sink[blockIdx.x] = s;  // keeps the chains live; never true
}

}  // namespace

extern "C" int qr_peak_fp64(double* gflops, void* stream) {
  if (!gflops) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int blocks = sms * 4, threads = 256, iters = 1000;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  dfma_probe<<<blocks, threads, 0, st>>>(nullptr, 10, 0.999, 1e-3);  // warm-up
  cudaEventRecord(e0, st);
  dfma_probe<<<blocks, threads, 0, st>>>(nullptr, iters, 0.999, 1e-3);
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return (int)e;
  const double flops = 2.0 * 64.0 * iters * (double)blocks * threads;
  *gflops = flops / (ms * 1e-3) / 1e9;
  return 0;
}
