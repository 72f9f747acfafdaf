// Application of the tile-QR orthogonal factor: qr_apply_qt_{d,s}
// (C <- Q^T C or C <- Q C) from the column-major output of qr_factor.
//
// Q = prod_k [Q_kk prod_{i>k} Q_ik] in the flat-tree order of Sec. 2.1 (the
// GEQRT factor of tile (k,k), then each TSQRT factor of tile (i,k)). Columns
// of C are independent under Q, so each CTA owns a chunk of C's columns and
// walks the whole task sequence for it; there are no inter-CTA dependencies.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "tile_kernels.cuh"
#include "tileqr_internal.h"

using namespace tqr;

namespace {

template <typename S, bool TR>
__global__ void __launch_bounds__(NTHREADS, 2)
    apply_q_kernel(const S* A, int64_t lda, const S* T, int64_t m, int64_t n, int NB, int IB, int MT, int NT,
                   S* C, int64_t ldc, int64_t nrhs, int cols_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem<S> sm = carve<S>(reinterpret_cast<S*>(smem_raw));
  const int c0 = blockIdx.x * cols_per_cta;
  const int c1 = (int)min((int64_t)c0 + cols_per_cta, nrhs);
  if (c0 >= c1) return;
  const int K = min(MT, NT);
  auto tileA = [&](int i, int j) { return A + (size_t)i * NB + (size_t)j * NB * lda; };
  auto tfac = [&](int i, int k) { return T + ((size_t)k * MT + i) * (size_t)IB * NB; };
  auto rows_of = [&](int i) { return (int)min((int64_t)NB, m - (int64_t)i * NB); };
  auto cols_of = [&](int j) { return (int)min((int64_t)NB, n - (int64_t)j * NB); };
  for (int kk = 0; kk < K; ++kk) {
    const int k = TR ? kk : K - 1 - kk;
    const int ck = cols_of(k);
    S* Ck = C + (size_t)k * NB;
    if (TR) {
      apply_qt<S, false, true>(tileA(k, k), (int)lda, tfac(k, k), IB, false, 0, ck, IB, nullptr, 0, Ck, (int)ldc,
                               rows_of(k), c0, c1, sm);
      for (int i = k + 1; i < MT; ++i)
        apply_qt<S, true, true>(tileA(i, k), (int)lda, tfac(i, k), IB, false, 0, ck, IB, Ck, (int)ldc,
                                C + (size_t)i * NB, (int)ldc, rows_of(i), c0, c1, sm);
    } else {
      for (int i = MT - 1; i > k; --i)
        apply_qt<S, true, false>(tileA(i, k), (int)lda, tfac(i, k), IB, false, 0, ck, IB, Ck, (int)ldc,
                                 C + (size_t)i * NB, (int)ldc, rows_of(i), c0, c1, sm);
      apply_qt<S, false, false>(tileA(k, k), (int)lda, tfac(k, k), IB, false, 0, ck, IB, nullptr, 0, Ck,
                                (int)ldc, rows_of(k), c0, c1, sm);
    }
  }
}

template <typename S>
int apply_impl(int64_t m, int64_t n, int64_t nrhs, const S* A, int64_t lda, int nb, int ib, const S* T, S* C,
               int64_t ldc, int trans, void* stream) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (nrhs < 0) return -3;
  if (lda < std::max<int64_t>(m, 1)) return -5;
  if (nb == 0) {
    if (qr_table_lookup(m, n, (int)sizeof(S), &nb, &ib) != 0) return -6;
  }
  if (nb < 8 || nb > 512) return -6;
  if (ib < 1 || ib > nb || ib > 256) return -7;
  if (ldc < std::max<int64_t>(m, 1)) return -10;
  if (trans != 0 && trans != 1) return -11;
  if (m == 0 || n == 0 || nrhs == 0) return 0;
  if (!A) return -4;
  if (!T) return -8;
  if (!C) return -9;
  if (lda > INT32_MAX || ldc > INT32_MAX) return -5;
  const int MT = (int)((m + nb - 1) / nb), NT = (int)((n + nb - 1) / nb);
  const int per = 32;
  const int64_t grid = (nrhs + per - 1) / per;
  const size_t smem = smem_elems<S>() * sizeof(S);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (trans) {
    e = cudaFuncSetAttribute(apply_q_kernel<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    apply_q_kernel<S, true><<<(unsigned)grid, NTHREADS, smem, st>>>(A, lda, T, m, n, nb, ib, MT, NT, C, ldc, nrhs,
                                                                   per);
  } else {
    e = cudaFuncSetAttribute(apply_q_kernel<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    apply_q_kernel<S, false><<<(unsigned)grid, NTHREADS, smem, st>>>(A, lda, T, m, n, nb, ib, MT, NT, C, ldc,
                                                                    nrhs, per);
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace

extern "C" {

int qr_apply_qt_d(int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb, int ib,
                  const double* T, double* C, int64_t ldc, int trans, void* stream) {
  return apply_impl<double>(m, n, nrhs, A, lda, nb, ib, T, C, ldc, trans, stream);
}

int qr_apply_qt_s(int64_t m, int64_t n, int64_t nrhs, const float* A, int64_t lda, int nb, int ib,
                  const float* T, float* C, int64_t ldc, int trans, void* stream) {
  return apply_impl<float>(m, n, nrhs, A, lda, nb, ib, T, C, ldc, trans, stream);
}

}  // extern "C"
