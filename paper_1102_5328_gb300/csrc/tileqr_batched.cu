// Batched QR of many small matrices of uneven sizes in one persistent launch.
//
// Each CTA pulls the next matrix from a global counter (matrices ordered by
// decreasing flop count, so the largest start first: longest-processing-time
// list scheduling) and factors it alone with the same tile kernels as the
// single-matrix path, run in the flat-tree order of Sec. 2.1 on tiles of
// order NB (NB >= m means one GEQRT on the whole matrix). NB and IB come per
// size class (rows m) from a small table the batched tuner fills. Everything
// the launch needs lives in device arrays, so memset + kernel can be captured
// in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <numeric>
#include <vector>

#include "tile_kernels.cuh"
#include "tileqr_internal.h"

using namespace tqr;

namespace {

std::mutex g_bmu;
struct ClassEntry {
  int m_hi, nb, ib;
};
std::vector<ClassEntry> g_classes[2];  // per precision, sorted by m_hi

void class_pair(int prec, int m, int* nb, int* ib) {
  std::lock_guard<std::mutex> lock(g_bmu);
  for (const ClassEntry& c : g_classes[prec]) {
    if (m <= c.m_hi) {
      *nb = c.nb;
      *ib = c.ib;
      return;
    }
  }
  *nb = 512;  // default: one tile per matrix, IB 16
  *ib = 16;
}

template <typename S>
__global__ void __launch_bounds__(NTHREADS, 2)
    batched_qr(int count, const int* __restrict__ ms, const int* __restrict__ ns, S* const* __restrict__ As,
               const int* __restrict__ ldas, S* Tbase, const int64_t* __restrict__ toff, const int* __restrict__ nbs,
               const int* __restrict__ ibs, const int* __restrict__ order, unsigned* counter, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem<S> sm = carve<S>(reinterpret_cast<S*>(smem_raw));
  __shared__ int s_idx;
  for (;;) {
    if (threadIdx.x == 0) s_idx = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= count) break;
    const int b = order[idx];
    const int m = ms[b], n = ns[b], lda = ldas[b];
    const int NB = min(nbs[b], m), IB = ibs[b];
    S* A = As[b];
    S* T = Tbase + toff[b];
    const int MT = (m + NB - 1) / NB, NT = (n + NB - 1) / NB;
    auto tile = [&](int i, int j) { return A + (size_t)i * NB + (size_t)j * NB * lda; };
    auto tf = [&](int i, int k) { return T + ((size_t)k * MT + i) * (size_t)IB * NB; };
    auto rows = [&](int i) { return min(NB, m - i * NB); };
    auto cols = [&](int j) { return min(NB, n - j * NB); };
    for (int k = 0; k < min(MT, NT); ++k) {
      geqrt<S>(tile(k, k), lda, rows(k), cols(k), IB, tf(k, k), sm, status);
      __syncthreads();
      for (int j = k + 1; j < NT; ++j) {
        unmqr<S>(tile(k, k), lda, tf(k, k), IB, rows(k), cols(k), tile(k, j), lda, 0, cols(j), sm);
        __syncthreads();
      }
      for (int i = k + 1; i < MT; ++i) {
        tsqrt<S>(tile(k, k), lda, tile(i, k), lda, rows(i), cols(k), IB, tf(i, k), sm, status);
        __syncthreads();
        for (int j = k + 1; j < NT; ++j) {
          tsmqr<S>(tile(i, k), lda, tf(i, k), IB, rows(i), cols(k), tile(k, j), lda, tile(i, j), lda, 0, cols(j), sm);
          __syncthreads();
        }
      }
    }
  }
}

template <typename S>
int launch(int count, const int* ms, const int* ns, S* const* As, const int* ldas, S* T, const int64_t* toff,
           const int* nbs, const int* ibs, const int* order, void* scratch, void* stream) {
  if (count < 0) return -1;
  if (count == 0) return 0;
  if (!ms || !ns || !As || !ldas || !T || !toff || !nbs || !ibs || !order) return -2;
  if (!scratch) return -11;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* counter = (unsigned*)scratch;
  int* status = (int*)((char*)scratch + 64);
  cudaError_t e = cudaMemsetAsync(scratch, 0, 128, st);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = smem_elems<S>() * sizeof(S);
  e = cudaFuncSetAttribute(batched_qr<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_qr<S>, NTHREADS, smem);
  if (e != cudaSuccess) return (int)e;
  const int grid = std::max(1, std::min(count, sms * std::max(occ, 1)));
  batched_qr<S><<<grid, NTHREADS, smem, st>>>(count, ms, ns, As, ldas, T, toff, nbs, ibs, order, counter, status);
  e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

}  // namespace

extern "C" {

int qr_batched_set_class(int prec, int m_hi, int nb, int ib) {
  if (prec != QR_PREC_F64 && prec != QR_PREC_F32) return -1;
  if (m_hi < 1) return -2;
  if (nb < 8 || nb > 512) return -3;
  if (ib < 1 || ib > nb || ib > 256) return -4;
  std::lock_guard<std::mutex> lock(g_bmu);
  auto& v = g_classes[prec];
  for (auto& c : v)
    if (c.m_hi == m_hi) {
      c.nb = nb;
      c.ib = ib;
      return 0;
    }
  v.push_back({m_hi, nb, ib});
  std::sort(v.begin(), v.end(), [](const ClassEntry& a, const ClassEntry& b) { return a.m_hi < b.m_hi; });
  return 0;
}

int qr_batched_clear_classes(int prec) {
  if (prec != QR_PREC_F64 && prec != QR_PREC_F32) return -1;
  std::lock_guard<std::mutex> lock(g_bmu);
  g_classes[prec].clear();
  return 0;
}

int qr_batched_plan(int count, const int* m, const int* n, int prec, int force_nb, int force_ib, int* nb_out,
                    int* ib_out, int* order_out, int64_t* t_offset_out, int64_t* t_total) {
  if (count < 0) return -1;
  if (count > 0 && (!m || !n)) return -2;
  if (prec != QR_PREC_F64 && prec != QR_PREC_F32) return -4;
  if (!nb_out || !ib_out || !order_out || !t_offset_out || !t_total) return -7;
  std::vector<double> fl(count);
  int64_t off = 0;
  for (int b = 0; b < count; ++b) {
    if (m[b] < 1 || n[b] < 1 || n[b] > m[b] || m[b] > 65535) return -2;
    int nb, ib;
    if (force_nb > 0) {
      nb = force_nb;
      ib = force_ib;
    } else {
      class_pair(prec, m[b], &nb, &ib);
    }
    nb = std::min(nb, 512);
    ib = std::max(1, std::min(ib, std::min(nb, 256)));
    const int NBe = std::min(nb, m[b]);
    nb_out[b] = nb;
    ib_out[b] = ib;
    const int64_t MT = (m[b] + NBe - 1) / NBe, NT = (n[b] + NBe - 1) / NBe;
    t_offset_out[b] = off;
    off += MT * NT * (int64_t)ib * NBe;
    off = (off + 31) & ~(int64_t)31;
    fl[b] = 2.0 * m[b] * (double)n[b] * n[b] - 2.0 * (double)n[b] * n[b] * n[b] / 3.0;
  }
  std::vector<int> ord(count);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return fl[a] > fl[b]; });
  for (int b = 0; b < count; ++b) order_out[b] = ord[b];
  *t_total = std::max<int64_t>(off, 1);
  return 0;
}

int qr_factor_batched_d(int count, const int* d_m, const int* d_n, double* const* d_A, const int* d_lda, double* d_T,
                        const int64_t* d_t_offset, const int* d_nb, const int* d_ib, const int* d_order,
                        void* d_scratch, void* stream) {
  return launch<double>(count, d_m, d_n, d_A, d_lda, d_T, d_t_offset, d_nb, d_ib, d_order, d_scratch, stream);
}

int qr_factor_batched_s(int count, const int* d_m, const int* d_n, float* const* d_A, const int* d_lda, float* d_T,
                        const int64_t* d_t_offset, const int* d_nb, const int* d_ib, const int* d_order,
                        void* d_scratch, void* stream) {
  return launch<float>(count, d_m, d_n, d_A, d_lda, d_T, d_t_offset, d_nb, d_ib, d_order, d_scratch, stream);
}

int qr_batched_status(const void* d_scratch, int* status, void* stream) {
  if (!d_scratch) return -1;
  if (!status) return -2;
  cudaError_t e = cudaMemcpyAsync(status, (const char*)d_scratch + 64, sizeof(int), cudaMemcpyDeviceToHost,
                                  (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  return e == cudaSuccess ? 0 : (int)e;
}

}  // extern "C"
