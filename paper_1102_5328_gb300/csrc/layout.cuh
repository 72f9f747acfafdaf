// Column-major <-> tile-layout conversion (Sec. 2.1: tiles of order NB,
// stored contiguously; ragged edges zero-padded) and status reset, shared
// by the factorization entry points.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tqr {

template <typename S>
__global__ void cm_to_tiles(const S* __restrict__ A, int64_t lda, int64_t m, int64_t n, S* __restrict__ W,
                            int NB, int MT, int NT, unsigned* zero_words, int64_t nzero) {
  const int64_t tile_elems = (int64_t)NB * NB;
  const int64_t total = tile_elems * MT * NT;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t t = e / tile_elems;
    const int64_t w = e - t * tile_elems;
    const int c = (int)(w / NB), r = (int)(w - (int64_t)c * NB);
    const int j = (int)(t / MT), i = (int)(t - (int64_t)j * MT);
    const int64_t row = (int64_t)i * NB + r, col = (int64_t)j * NB + c;
    W[e] = (row < m && col < n) ? A[row + col * lda] : S(0);
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nzero; e += stride) zero_words[e] = 0u;
}

template <typename S>
__global__ void tiles_to_cm(const S* __restrict__ W, S* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                            int NB, int MT) {
  const int64_t total = m * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t col = e / m, row = e - col * m;
    const int i = (int)(row / NB), j = (int)(col / NB);
    const int r = (int)(row - (int64_t)i * NB), c = (int)(col - (int64_t)j * NB);
    A[row + col * lda] = W[((int64_t)j * MT + i) * NB * NB + r + (int64_t)c * NB];
  }
}

}  // namespace tqr
