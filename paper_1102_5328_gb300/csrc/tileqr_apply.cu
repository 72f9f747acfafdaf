// Application of the tile-QR orthogonal factor: qr_apply_qt_{d,s}
// (C <- Q^T C or C <- Q C) from the column-major output of qr_factor.
//
// Q = prod_k [Q_kk prod_{i>k} Q_ik] in the flat-tree order of Sec. 2.1 (the
// GEQRT factor of tile (k,k), then each TSQRT factor of tile (i,k)).
// Two schedules:
//  * qr_apply_qt_{d,s}: columns of C are independent under Q, so each CTA
//    owns a chunk of C's columns and walks the whole task sequence for it
//    (no scratch, no inter-CTA dependencies; parallel only across columns).
//  * qr_apply_qt_ws_{d,s}: the same tasks as the factorization's updates with
//    C in place of a trailing tile column (UNMQR on C's row block k, TSMQR on
//    row blocks k and i), run by a persistent kernel over a dependency-ordered
//    task list, so few right-hand sides still use many SMs: the row blocks
//    of consecutive elimination steps proceed as a wavefront.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "sched.cuh"
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

// ---------------------------------------------------------------------------
// Persistent, dependency-ordered application (qr_apply_qt_ws_*).
//
// Per (row block r of C, column chunk s) a counter of completed writes.
// Q^T (program order k ascending: GE(k); TS(i, k) for i ascending): the
// required counts are those of the factorization's trailing tiles:
//   GE(k): C_k >= k;  TS(i, k): top C_k >= i, bottom C_i >= k.
// Q (program order k descending: TS(i, k) for i descending; then GE(k)):
// C_r is first written at step r (its MT-1-r TS tasks as top, then GE(r)),
// then once per earlier step as bottom:
//   TS(i, k): top C_k >= MT-1-i, bottom C_i >= (i < K ? MT-i : 0) + min(i,K)-1-k;
//   GE(k): C_k >= MT-1-k.
std::mutex g_amu;
struct AKey {
  int MT, NT, S, tr;
  bool operator<(const AKey& o) const { return std::tie(MT, NT, S, tr) < std::tie(o.MT, o.NT, o.S, o.tr); }
};
std::map<AKey, std::vector<uint64_t>> g_asched;

const std::vector<uint64_t>& apply_schedule(int MT, int NT, int S, int tr) {
  AKey key{MT, NT, S, tr};
  auto it = g_asched.find(key);
  if (it != g_asched.end()) return it->second;
  const int K = std::min(MT, NT);
  std::vector<uint64_t> code;
  std::vector<double> est;
  std::vector<double> fin((size_t)MT * S, 0.0);
  auto F = [&](int r, int s) -> double& { return fin[(size_t)r * S + s]; };
  auto ge = [&](int k) {
    for (int s = 0; s < S; ++s) {
      const double st = F(k, s);
      F(k, s) = st + 1.0;
      code.push_back(encode_task(TASK_UNMQR, s, k, 0, k));
      est.push_back(st);
    }
  };
  auto ts = [&](int i, int k) {
    for (int s = 0; s < S; ++s) {
      const double st = std::max(F(k, s), F(i, s));
      F(k, s) = F(i, s) = st + 2.0;
      code.push_back(encode_task(TASK_TSMQR, s, i, 0, k));
      est.push_back(st);
    }
  };
  if (tr) {
    for (int k = 0; k < K; ++k) {
      ge(k);
      for (int i = k + 1; i < MT; ++i) ts(i, k);
    }
  } else {
    for (int k = K - 1; k >= 0; --k) {
      for (int i = MT - 1; i > k; --i) ts(i, k);
      ge(k);
    }
  }
  std::vector<int64_t> idx(code.size());
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return est[a] < est[b]; });
  std::vector<uint64_t> out(code.size());
  for (size_t t = 0; t < idx.size(); ++t) out[t] = code[idx[t]];
  return g_asched.emplace(key, std::move(out)).first->second;
}

int apply_split(int64_t nrhs) { return (int)std::max<int64_t>(1, (nrhs + 63) / 64); }

struct ALayout {
  int MT, NT, S;
  int64_t ntasks;
  size_t off_cnt, off_tasks, bytes;
};

ALayout apply_layout(int64_t m, int64_t n, int64_t nrhs, int nb) {
  ALayout L;
  L.MT = (int)((m + nb - 1) / nb);
  L.NT = (int)((n + nb - 1) / nb);
  L.S = apply_split(nrhs);
  const int K = std::min(L.MT, L.NT);
  int64_t c = 0;
  for (int k = 0; k < K; ++k) c += (int64_t)L.S * (1 + (L.MT - k - 1));
  L.ntasks = c;
  L.off_cnt = 256;
  L.off_tasks = (L.off_cnt + (size_t)L.MT * L.S * 4 + 255) & ~(size_t)255;
  L.bytes = (L.off_tasks + (size_t)L.ntasks * 8 + 255) & ~(size_t)255;
  return L;
}

template <typename S>
struct ApplyArgs {
  const S* A;
  int64_t lda;
  const S* T;
  int64_t m, n;
  int NB, IB, MT, NT, S_;
  S* C;
  int64_t ldc, nrhs;
  const uint64_t* tasks;
  int64_t ntasks;
  unsigned* cnt;
  DevCtl* ctl;
  uint64_t timeout_ns;
};

__global__ void zero_words(unsigned* p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0u;
}

template <typename S, bool TR>
__global__ void __launch_bounds__(NTHREADS, 2) persistent_apply(ApplyArgs<S> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem<S> sm = carve<S>(reinterpret_cast<S*>(smem_raw));
  __shared__ int64_t s_ticket;
  __shared__ int s_ok;
  const int NB = a.NB, MT = a.MT, Sp = a.S_;
  const int K = min(a.MT, a.NT);
  auto tileA = [&](int i, int j) { return a.A + (size_t)i * NB + (size_t)j * NB * a.lda; };
  auto tfac = [&](int i, int k) { return a.T + ((size_t)k * MT + i) * (size_t)a.IB * NB; };
  auto rows_of = [&](int i) { return (int)min((int64_t)NB, a.m - (int64_t)i * NB); };
  auto cols_of = [&](int j) { return (int)min((int64_t)NB, a.n - (int64_t)j * NB); };
  auto ctr = [&](int r, int s) { return a.cnt + (size_t)r * Sp + s; };
  for (;;) {
    if (threadIdx.x == 0) {
      int64_t t = -1;
      if (!((volatile int*)&a.ctl->abort)[0]) t = (int64_t)atomicAdd(&a.ctl->ticket, 1u);
      s_ticket = t;
    }
    __syncthreads();
    const int64_t t = s_ticket;
    if (t < 0 || t >= a.ntasks) break;
    int type, sch, i, j, k;
    decode_task(a.tasks[t], type, sch, i, j, k);
    const int c0 = (int)((int64_t)sch * a.nrhs / Sp), c1 = (int)((int64_t)(sch + 1) * a.nrhs / Sp);
    S* Ck = a.C + (size_t)k * NB;
    const int ck = cols_of(k);
    const int rw = type == TASK_UNMQR ? rows_of(k) : rows_of(i);
    // few right-hand sides: stage the whole task in shared memory once; the
    // reflectors and T are final (written by the factorization), so they are
    // staged before the wait for the task's rows of C
    const bool nar = narrow_fits(rw, ck, a.IB, c1 - c0);
    if (nar) {
      if (type == TASK_UNMQR)
        narrow_stage_vt<S, false>(tileA(k, k), (int)a.lda, tfac(k, k), a.IB, ck, a.IB, rw, sm);
      else
        narrow_stage_vt<S, true>(tileA(i, k), (int)a.lda, tfac(i, k), a.IB, ck, a.IB, rw, sm);
    }
    if (threadIdx.x == 0) {
      bool ok;
      const uint64_t to = a.timeout_ns;
      if (type == TASK_UNMQR) {
        ok = wait_ge(ctr(k, sch), 1, TR ? (unsigned)k : (unsigned)(MT - 1 - k), a.ctl, to);
      } else {
        const unsigned rt = TR ? (unsigned)i : (unsigned)(MT - 1 - i);
        const unsigned rb = TR ? (unsigned)k : (unsigned)((i < K ? MT - i : 0) + min(i, K) - 1 - k);
        ok = wait_ge(ctr(k, sch), 1, rt, a.ctl, to) && wait_ge(ctr(i, sch), 1, rb, a.ctl, to);
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    if (type == TASK_UNMQR) {
      if (nar)
        apply_narrow<S, false, TR>(tileA(k, k), (int)a.lda, tfac(k, k), a.IB, ck, a.IB, nullptr, 0, Ck, (int)a.ldc,
                                   rows_of(k), c0, c1, sm, false, true);
      else
        apply_qt<S, false, TR>(tileA(k, k), (int)a.lda, tfac(k, k), a.IB, false, 0, ck, a.IB, nullptr, 0, Ck,
                               (int)a.ldc, rows_of(k), c0, c1, sm);
    } else {
      if (nar)
        apply_narrow<S, true, TR>(tileA(i, k), (int)a.lda, tfac(i, k), a.IB, ck, a.IB, Ck, (int)a.ldc,
                                  a.C + (size_t)i * NB, (int)a.ldc, rows_of(i), c0, c1, sm, false, true);
      else
        apply_qt<S, true, TR>(tileA(i, k), (int)a.lda, tfac(i, k), a.IB, false, 0, ck, a.IB, Ck, (int)a.ldc,
                              a.C + (size_t)i * NB, (int)a.ldc, rows_of(i), c0, c1, sm);
    }
    // publish: the barrier orders every thread's C writes before thread
    // 0's fence and release (cumulative), one fence per task
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      red_release_add(ctr(k, sch), 1u);
      if (type == TASK_TSMQR) red_release_add(ctr(i, sch), 1u);
    }
  }
}

template <typename S, bool TR>
int launch_ws(const ApplyArgs<S>& aa, cudaStream_t st) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = smem_elems<S>() * sizeof(S);
  cudaError_t e = cudaFuncSetAttribute(persistent_apply<S, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_apply<S, TR>, NTHREADS, smem);
  if (e != cudaSuccess) return (int)e;
  if (occ < 1) return (int)cudaErrorInvalidConfiguration;
  const int64_t grid = std::min<int64_t>((int64_t)sms * occ, aa.ntasks);
  persistent_apply<S, TR><<<(unsigned)grid, NTHREADS, smem, st>>>(aa);
  e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

template <typename S>
int apply_ws_impl(int64_t m, int64_t n, int64_t nrhs, const S* A, int64_t lda, int nb, int ib, const S* T, S* C,
                  int64_t ldc, int trans, void* scratch, int64_t scratch_bytes, void* stream) {
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
  if (!scratch) return -12;
  if (lda > INT32_MAX || ldc > INT32_MAX) return -5;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_amu);
  const ALayout L = apply_layout(m, n, nrhs, nb);
  if (scratch_bytes < (int64_t)L.bytes) return -13;
  if (L.MT > 65535) return -1;
  const std::vector<uint64_t>& sc = apply_schedule(L.MT, L.NT, L.S, trans);
  char* base = (char*)scratch;
  cudaError_t e = cudaMemcpyAsync(base + L.off_tasks, sc.data(), sc.size() * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return (int)e;
  zero_words<<<64, 256, 0, st>>>((unsigned*)base, (int64_t)(L.off_tasks / 4));
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  ApplyArgs<S> aa;
  aa.A = A; aa.lda = lda; aa.T = T; aa.m = m; aa.n = n; aa.NB = nb; aa.IB = ib; aa.MT = L.MT; aa.NT = L.NT;
  aa.S_ = L.S; aa.C = C; aa.ldc = ldc; aa.nrhs = nrhs; aa.tasks = (const uint64_t*)(base + L.off_tasks);
  aa.ntasks = L.ntasks; aa.cnt = (unsigned*)(base + L.off_cnt); aa.ctl = (DevCtl*)base;
  aa.timeout_ns = (uint64_t)qr_get_option(QR_OPT_WAIT_TIMEOUT_US) * 1000ull;
  return trans ? launch_ws<S, true>(aa, st) : launch_ws<S, false>(aa, st);
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

int qr_apply_workspace(int64_t m, int64_t n, int64_t nrhs, int nb, int64_t* bytes) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (nrhs < 1) return -3;
  if (nb == 0) {
    int ib = 0;
    if (qr_table_lookup(m, n, 8, &nb, &ib) != 0) return -4;
  }
  if (nb < 8 || nb > 512) return -4;
  if (!bytes) return -5;
  *bytes = (int64_t)apply_layout(m, n, nrhs, nb).bytes;
  return 0;
}

int qr_apply_qt_ws_d(int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb, int ib,
                     const double* T, double* C, int64_t ldc, int trans, void* scratch, int64_t scratch_bytes,
                     void* stream) {
  return apply_ws_impl<double>(m, n, nrhs, A, lda, nb, ib, T, C, ldc, trans, scratch, scratch_bytes, stream);
}

int qr_apply_qt_ws_s(int64_t m, int64_t n, int64_t nrhs, const float* A, int64_t lda, int nb, int ib,
                     const float* T, float* C, int64_t ldc, int trans, void* scratch, int64_t scratch_bytes,
                     void* stream) {
  return apply_ws_impl<float>(m, n, nrhs, A, lda, nb, ib, T, C, ldc, trans, scratch, scratch_bytes, stream);
}

}  // extern "C"
