// Tile Cholesky factorization A = L L^T on the persistent DAG scheduler, and
// its empirical NB tuner: the sister factorization the paper names for the
// same tile framework and the same autotuning method (Secs. 1 and 7; the
// paper tunes QR only).
//
// Tasks over the lower triangle of NT x NT tiles of order NB:
//   POTRF(k)      L_kk = chol(A_kk)
//   TRSM(i, k)    L_ik = A_ik L_kk^-T                          (i > k)
//   SYRK(i, k)    A_ii -= L_ik L_ik^T                          (i > k)
//   GEMM(i, j, k) A_ij -= L_ik L_jk^T                          (i > j > k)
// A tile's counter counts the operations applied to it: its k updates in
// order, then its POTRF or TRSM; a task waits (bounded, acquire) until the
// counters of what it reads and writes reach their values and publishes
// with a release increment -- the scheme of the QR kernels. All arithmetic
// is FP64 on the CUDA cores (the FP64 pipe bounds every task); the in-tile
// POTRF and TRSM are blocked by 32 columns, and every product runs in one
// staged kernel of 64 x 64 output passes (16 outputs per thread).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "layout.cuh"
#include "listsched.h"
#include "sched.cuh"
#include "tileqr_internal.h"

using namespace tqr;

// nb for an order n from the Cholesky tuning table (closest tuned order, ties
// to the smaller); 128 when nothing is tuned (returns 1 then).
int chol_table_lookup(int64_t n, int* nb);

namespace {

constexpr int CT = 256;  // threads per CTA
constexpr int CB = 32;   // column block of the in-tile POTRF / TRSM
constexpr int KC = 32;   // k-slice of a staged product
constexpr int BLD = CB + 1;

enum { CH_POTRF = 0, CH_TRSM = 1, CH_SYRK = 2, CH_GEMM = 3 };

struct CSmem {
  double* a;     // [KC * 64] staged slice of the left operand
  double* b;     // [KC * 64] staged slice of the right operand
  double* blk;   // [CB * BLD] a diagonal block of L (column-major, ld BLD)
  double* rinv;  // [CB] reciprocals of its diagonal
};
constexpr size_t kCSmemDoubles = 2 * KC * 64 + CB * BLD + CB;

__device__ __forceinline__ CSmem ccarve(double* base) {
  CSmem s;
  s.a = base;
  s.b = s.a + KC * 64;
  s.blk = s.b + KC * 64;
  s.rinv = s.blk + CB * BLD;
  return s;
}

__device__ __forceinline__ double ldc_(const double* p) { return __ldcg(p); }
__device__ __forceinline__ void stc_(double* p, double v) { __stcg(p, v); }

// C(r, c) -= sum_{k < K} A(r, k) B(c, k) for r < M, c < N (column-major
// operands, leading dimensions lda, ldb, ldc; tiles written by other CTAs
// are read through L2). lower: only c <= r is needed (output passes wholly
// above the diagonal are skipped, the others write c <= r only). Passes of
// 64 x 64 outputs; thread (tx, ty) of 16 x 16 owns rows tx + 16 a and
// columns ty + 16 b, a, b < 4; KC-slices of both operands staged in shared
// memory.
__device__ void gemm_update(double* C, int ldc, const double* A, int lda, const double* B, int ldb, int M, int N,
                            int K, bool lower, const CSmem& sm) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int r0 = 0; r0 < M; r0 += 64)
    for (int c0 = 0; c0 < N; c0 += 64) {
      if (lower && c0 > r0 + 63) continue;  // uniform over the CTA
      double acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
      for (int k0 = 0; k0 < K; k0 += KC) {
        const int kc = min(KC, K - k0);
        __syncthreads();  // the previous slice's readers are done
#pragma unroll
        for (int u = 0; u < KC * 64 / CT; ++u) {
          const int idx = tid + u * CT;
          const int kk = idx >> 6, rr = idx & 63;
          sm.a[idx] = (kk < kc && r0 + rr < M) ? ldc_(A + (r0 + rr) + (size_t)(k0 + kk) * lda) : 0.0;
          sm.b[idx] = (kk < kc && c0 + rr < N) ? ldc_(B + (c0 + rr) + (size_t)(k0 + kk) * ldb) : 0.0;
        }
        __syncthreads();
        for (int kk = 0; kk < kc; ++kk) {
          double av[4], bv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = sm.a[kk * 64 + tx + 16 * a];
#pragma unroll
          for (int b = 0; b < 4; ++b) bv[b] = sm.b[kk * 64 + ty + 16 * b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int r = r0 + tx + 16 * a, c = c0 + ty + 16 * b;
          if (r < M && c < N && (!lower || c <= r)) {
            double* p = C + r + (size_t)c * ldc;
            stc_(p, ldc_(p) - acc[a][b]);
          }
        }
    }
  __syncthreads();
}

// X (rows x w, columns of a tile) <- X L_blk^-T with the w x w lower block of
// L in sm.blk and its reciprocal diagonal in sm.rinv: row r solves
// x L_blk^T = b, x_j = (b_j - sum_{l<j} L_jl x_l) / L_jj, one thread per
// row (rows <= CT), the row's w unknowns in registers.
__device__ void block_solve(double* X, int ldx, int rows, int w, const CSmem& sm) {
  const int r = threadIdx.x;
  if (r < rows) {
    double x[CB];
#pragma unroll
    for (int j = 0; j < CB; ++j) x[j] = j < w ? ldc_(X + r + (size_t)j * ldx) : 0.0;
#pragma unroll
    for (int j = 0; j < CB; ++j) {
      if (j < w) {
        double s = x[j];
#pragma unroll
        for (int l = 0; l < j; ++l) s = fma(-sm.blk[j + l * BLD], x[l], s);
        x[j] = s * sm.rinv[j];
      }
    }
#pragma unroll
    for (int j = 0; j < CB; ++j)
      if (j < w) stc_(X + r + (size_t)j * ldx, x[j]);
  }
  __syncthreads();
}

// The w x w lower block of L at L + jb (1 + ldl) into sm.blk (zero above the
// diagonal and outside) and the reciprocals of its diagonal into sm.rinv.
__device__ void stage_diag_block(const double* L, int ldl, int jb, int w, const CSmem& sm) {
  __syncthreads();
  for (int idx = threadIdx.x; idx < CB * CB; idx += CT) {
    const int i = idx % CB, j = idx / CB;
    sm.blk[i + j * BLD] = (i < w && j < w && i >= j) ? ldc_(L + (jb + i) + (size_t)(jb + j) * ldl) : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < w) sm.rinv[threadIdx.x] = 1.0 / sm.blk[threadIdx.x * (BLD + 1)];
  __syncthreads();
}

// POTRF of an n x n diagonal tile in place (lower triangle), blocked by CB
// columns: factor the diagonal block (one warp, column by column), solve the
// panel below it (block_solve), update the trailing lower triangle
// (gemm_update). A pivot that is not positive (or not finite) sets
// QR_DEV_NOT_SPD and records its global column (gcol0 + j) in *first_bad as
// INT_MAX - column under atomicMax, so the smallest failing column wins.
__device__ void potrf_tile(double* A, int lda, int n, int64_t gcol0, DevCtl* ctl, int* first_bad,
                           const CSmem& sm) {
  for (int jb = 0; jb < n; jb += CB) {
    const int w = min(CB, n - jb);
    __syncthreads();
    for (int idx = threadIdx.x; idx < CB * CB; idx += CT) {
      const int i = idx % CB, j = idx / CB;
      sm.blk[i + j * BLD] = (i < w && j < w && i >= j) ? ldc_(A + (jb + i) + (size_t)(jb + j) * lda) : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int j = 0; j < w; ++j) {
        if (lane == j) {
          double d = sm.blk[j * (BLD + 1)];
          for (int l = 0; l < j; ++l) d = fma(-sm.blk[j + l * BLD], sm.blk[j + l * BLD], d);
          if (!(d > 0.0) || !isfinite(d)) {
            atomicOr(&ctl->status, QR_DEV_NOT_SPD);
            const int64_t col = gcol0 + jb + j;
            atomicMax(first_bad, INT_MAX - (int)(col < INT_MAX - 1 ? col : INT_MAX - 1));
          }
          const double ljj = sqrt(d);
          sm.blk[j * (BLD + 1)] = ljj;
          sm.rinv[j] = 1.0 / ljj;
        }
        __syncwarp();
        if (lane > j && lane < w) {
          double s = sm.blk[lane + j * BLD];
          for (int l = 0; l < j; ++l) s = fma(-sm.blk[lane + l * BLD], sm.blk[j + l * BLD], s);
          sm.blk[lane + j * BLD] = s * sm.rinv[j];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < CB * CB; idx += CT) {
      const int i = idx % CB, j = idx / CB;
      if (i < w && j < w && i >= j) stc_(A + (jb + i) + (size_t)(jb + j) * lda, sm.blk[i + j * BLD]);
    }
    __syncthreads();
    const int rest = n - jb - w;
    if (rest > 0) {
      double* P = A + (jb + w) + (size_t)jb * lda;
      block_solve(P, lda, rest, w, sm);
      gemm_update(A + (jb + w) + (size_t)(jb + w) * lda, lda, P, lda, P, lda, rest, rest, w, true, sm);
    }
  }
  __syncthreads();
}

// TRSM of a rows x nk tile X against the nk x nk factor L (lower):
// X <- X L^-T, blocked by CB columns.
__device__ void trsm_tile(double* X, int ldx, int rows, const double* L, int ldl, int nk, const CSmem& sm) {
  for (int jb = 0; jb < nk; jb += CB) {
    const int w = min(CB, nk - jb);
    stage_diag_block(L, ldl, jb, w, sm);
    block_solve(X + (size_t)jb * ldx, ldx, rows, w, sm);
    const int rest = nk - jb - w;
    if (rest > 0)
      gemm_update(X + (size_t)(jb + w) * ldx, ldx, X + (size_t)jb * ldx, ldx, L + (jb + w) + (size_t)jb * ldl, ldl,
                  rows, rest, w, false, sm);
  }
}

// Lower triangle of the tile layout back to column-major (the strict upper
// triangle of the caller's A is left as it was, as LAPACK's dpotrf does).
__global__ void tiles_to_cm_lower(const double* __restrict__ W, double* __restrict__ A, int64_t lda, int64_t n, int NB,
                                  int NT) {
  const int64_t total = n * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t col = e / n, row = e - col * n;
    if (row < col) continue;
    const int i = (int)(row / NB), j = (int)(col / NB);
    const int r = (int)(row - (int64_t)i * NB), c = (int)(col - (int64_t)j * NB);
    A[row + col * lda] = W[((int64_t)j * NT + i) * NB * NB + r + (int64_t)c * NB];
  }
}

struct CholArgs {
  double* W;
  int64_t n;
  int NB, NT;
  const uint64_t* tasks;
  int64_t ntasks;
  unsigned* cnt;  // NT x NT, the lower triangle used
  DevCtl* ctl;
  int* first_bad;
  uint64_t timeout_ns;
  TraceRec* trace;
  int64_t trace_cap;
};

__global__ void __launch_bounds__(CT, 2) persistent_chol(CholArgs a) {
  extern __shared__ __align__(16) double csm_raw[];
  const CSmem sm = ccarve(csm_raw);
  __shared__ int64_t s_ticket;
  __shared__ int s_ok;
  const int NB = a.NB, NT = a.NT;
  const size_t te = (size_t)NB * NB;
  auto tile = [&](int i, int j) { return a.W + ((size_t)j * NT + i) * te; };
  auto ctr = [&](int i, int j) { return a.cnt + (size_t)j * NT + i; };
  auto dim_of = [&](int i) { return (int)min((int64_t)NB, a.n - (int64_t)i * NB); };
  for (;;) {
    if (threadIdx.x == 0) {
      int64_t t = -1;
      if (!((volatile int*)&a.ctl->abort)[0]) t = (int64_t)atomicAdd(&a.ctl->ticket, 1u);
      s_ticket = t;
    }
    __syncthreads();
    const int64_t t = s_ticket;
    if (t < 0 || t >= a.ntasks) break;
    int type, s_, i, j, k;
    decode_task(a.tasks[t], type, s_, i, j, k);
    uint64_t t_take = 0, t_ready = 0;
    if (threadIdx.x == 0) {
      if (a.trace) t_take = globaltimer();
      const uint64_t to = a.timeout_ns;
      bool ok = true;
      switch (type) {
        case CH_POTRF: ok = wait_ge(ctr(k, k), 1, (unsigned)k, a.ctl, to); break;
        case CH_TRSM:
          ok = wait_ge(ctr(k, k), 1, (unsigned)k + 1, a.ctl, to) && wait_ge(ctr(i, k), 1, (unsigned)k, a.ctl, to);
          break;
        case CH_SYRK:
          ok = wait_ge(ctr(i, k), 1, (unsigned)k + 1, a.ctl, to) && wait_ge(ctr(i, i), 1, (unsigned)k, a.ctl, to);
          break;
        default:
          ok = wait_ge(ctr(i, k), 1, (unsigned)k + 1, a.ctl, to) && wait_ge(ctr(j, k), 1, (unsigned)k + 1, a.ctl, to) &&
               wait_ge(ctr(i, j), 1, (unsigned)k, a.ctl, to);
          break;
      }
      s_ok = ok;
      if (a.trace) t_ready = globaltimer();
    }
    __syncthreads();
    if (!s_ok) break;
    const int nk = dim_of(k);
    switch (type) {
      case CH_POTRF: potrf_tile(tile(k, k), NB, nk, (int64_t)k * NB, a.ctl, a.first_bad, sm); break;
      case CH_TRSM: trsm_tile(tile(i, k), NB, dim_of(i), tile(k, k), NB, nk, sm); break;
      case CH_SYRK: gemm_update(tile(i, i), NB, tile(i, k), NB, tile(i, k), NB, dim_of(i), dim_of(i), nk, true, sm); break;
      default: gemm_update(tile(i, j), NB, tile(i, k), NB, tile(j, k), NB, dim_of(i), dim_of(j), nk, false, sm); break;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      switch (type) {
        case CH_POTRF: red_release_add(ctr(k, k), 1u); break;
        case CH_TRSM: red_release_add(ctr(i, k), 1u); break;
        case CH_SYRK: red_release_add(ctr(i, i), 1u); break;
        default: red_release_add(ctr(i, j), 1u); break;
      }
      trace_put(a.trace, a.trace_cap, t, type, t_take, t_ready);
    }
  }
}

// ---------------------------------------------------------------------------
// Host: layout, the task order, launch.
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct CLayout {
  int NT;
  int64_t ntasks;
  size_t off_cnt, off_tasks, off_tiles, bytes;
};

int64_t chol_task_count(int NT) {
  int64_t c = 0;
  for (int k = 0; k < NT; ++k) {
    const int64_t r = NT - k - 1;
    c += 1 + 2 * r + r * (r - 1) / 2;
  }
  return c;
}

CLayout chol_layout(int64_t n, int nb) {
  CLayout L;
  L.NT = (int)((n + nb - 1) / nb);
  L.ntasks = chol_task_count(L.NT);
  L.off_cnt = 256;  // DevCtl at 0, first_bad at 64
  L.off_tasks = al256(L.off_cnt + (size_t)L.NT * L.NT * 4);
  L.off_tiles = al256(L.off_tasks + (size_t)L.ntasks * 8);
  L.bytes = al256(L.off_tiles + (size_t)L.NT * L.NT * nb * nb * 8);
  return L;
}

std::mutex g_cmu;
std::map<std::pair<int, int>, std::vector<uint64_t>> g_corders;  // (NT, workers) -> ticket order (host copy)

// Program order (k-major, topological) with direct predecessors, then the
// list schedule for the kernel's workers. Costs: flops of each task (POTRF
// NB^3/3 weighted 2x for its serial column chain, TRSM NB^3, SYRK NB^3,
// GEMM 2 NB^3).
const std::vector<uint64_t>& chol_order(int NT, int workers) {
  auto key = std::make_pair(NT, workers);
  auto it = g_corders.find(key);
  if (it != g_corders.end()) return it->second;
  std::vector<uint64_t> code;
  std::vector<double> w;
  std::vector<int64_t> poff{0};
  std::vector<int32_t> pred;
  std::map<std::tuple<int, int, int>, int32_t> last;  // last task that wrote tile (i, j): its index
  auto writer = [&](int i, int j) {
    auto f = last.find(std::make_tuple(i, j, 0));
    return f == last.end() ? -1 : f->second;
  };
  auto add = [&](int type, int i, int j, int k, double cost, std::initializer_list<int32_t> deps) {
    for (int32_t d : deps)
      if (d >= 0) pred.push_back(d);
    code.push_back(encode_task(type, 0, i, j, k));
    w.push_back(cost);
    poff.push_back((int64_t)pred.size());
    return (int32_t)(code.size() - 1);
  };
  for (int k = 0; k < NT; ++k) {
    const int32_t p = add(CH_POTRF, k, k, k, 2.0 / 3.0, {writer(k, k)});
    last[std::make_tuple(k, k, 0)] = p;
    for (int i = k + 1; i < NT; ++i) last[std::make_tuple(i, k, 0)] = add(CH_TRSM, i, k, k, 1.0, {p, writer(i, k)});
    for (int i = k + 1; i < NT; ++i)
      last[std::make_tuple(i, i, 0)] = add(CH_SYRK, i, i, k, 1.0, {writer(i, k), writer(i, i)});
    for (int i = k + 1; i < NT; ++i)
      for (int j = k + 1; j < i; ++j)
        last[std::make_tuple(i, j, 0)] = add(CH_GEMM, i, j, k, 2.0, {writer(i, k), writer(j, k), writer(i, j)});
  }
  const std::vector<int64_t> idx = list_schedule(w, poff, pred, workers);
  std::vector<uint64_t> order(code.size());
  for (size_t t = 0; t < idx.size(); ++t) order[t] = code[idx[t]];
  return g_corders.emplace(key, std::move(order)).first->second;
}

int chol_grid(int* grid_out, int* workers) {
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
  const size_t smem = kCSmemDoubles * sizeof(double);
  if ((e = cudaFuncSetAttribute(persistent_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return (int)e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_chol, CT, smem)) != cudaSuccess) return (int)e;
  if (occ < 1) return (int)cudaErrorInvalidConfiguration;
  int per = occ;
  const int64_t cps = qr_get_option(QR_OPT_CTAS_PER_SM);
  if (cps > 0) per = std::min<int>(per, (int)cps);
  int use = sms;
  const int64_t budget = qr_get_option(QR_OPT_SM_BUDGET);
  if (budget > 0) use = (int)std::min<int64_t>(budget, sms);
  int grid = use * per;
  const int64_t gl = qr_get_option(QR_OPT_GRID_LIMIT);
  if (gl > 0) grid = std::min<int>(grid, (int)gl);
  *grid_out = grid;
  *workers = 2 * use;
  return 0;
}

int chol_impl(int64_t n, double* A, int64_t lda, int nb, void* scratch, int64_t scratch_bytes, void* stream) {
  if (n < 0) return -1;
  if (!A && n > 0) return -2;
  if (lda < std::max<int64_t>(n, 1)) return -3;
  if (nb == 0) chol_table_lookup(n, &nb);
  if (nb < 16 || nb > 256 || nb % 16) return -4;
  if (n == 0) return 0;
  if (!scratch) return -5;
  cudaStream_t st = (cudaStream_t)stream;
  const CLayout L = chol_layout(n, nb);
  if (scratch_bytes < (int64_t)L.bytes) return -6;
  if (L.NT > 65535) return -1;
  int grid = 0, workers = 0;
  int rc = chol_grid(&grid, &workers);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_cmu);
  const std::vector<uint64_t>& order = chol_order(L.NT, workers);
  char* base = (char*)scratch;
  cudaError_t e = cudaMemcpyAsync(base + L.off_tasks, order.data(), order.size() * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return (int)e;  // cached orders are never freed: the host copy outlives the copy
  double* W = (double*)(base + L.off_tiles);
  const int64_t nzero = (int64_t)(L.off_cnt / 4) + (int64_t)L.NT * L.NT;
  cm_to_tiles<double><<<1184, 256, 0, st>>>(A, lda, n, n, W, nb, L.NT, L.NT, (unsigned*)base, nzero);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  CholArgs ca;
  ca.W = W; ca.n = n; ca.NB = nb; ca.NT = L.NT;
  ca.tasks = (const uint64_t*)(base + L.off_tasks); ca.ntasks = (int64_t)order.size();
  ca.cnt = (unsigned*)(base + L.off_cnt); ca.ctl = (DevCtl*)base; ca.first_bad = (int*)(base + 64);
  ca.timeout_ns = (uint64_t)qr_get_option(QR_OPT_WAIT_TIMEOUT_US) * 1000ull;
  {
    void* tb = nullptr;
    int64_t tcap = 0;
    qr_trace_target(&tb, &tcap);
    ca.trace = (TraceRec*)tb;
    ca.trace_cap = tcap;
  }
  persistent_chol<<<grid, CT, kCSmemDoubles * sizeof(double), st>>>(ca);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  tiles_to_cm_lower<<<1184, 256, 0, st>>>(W, A, lda, n, nb, L.NT);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  return 0;
}

// ---------------------------------------------------------------------------
// The empirical NB tuner for the Cholesky factorization, Secs. 5–6 applied
// to its one tuning parameter: Step 1 times the dominant task (GEMM, about
// NT^3 / 6 of them) on a device-filling batch for every NB of the grid
// {32, 64, ..., 256}; the upper hull of (NB, GFLOP/s) and Heuristic 0/1/2
// (qr_tune_preselect) preselect; Step 2 times the factorization for the
// survivors at each order, ascending, and prunes with Property 6.1
// (qr_tune_payg). Untuned orders take the closest tuned one.
__global__ void __launch_bounds__(CT, 2) gemm_batch(const double* A, const double* B, double* C, int NB) {
  extern __shared__ __align__(16) double gsm_raw[];
  const CSmem sm = ccarve(gsm_raw);
  gemm_update(C + blockIdx.x * (size_t)NB * NB, NB, A, NB, B, NB, NB, NB, NB, false, sm);
}

__device__ __forceinline__ double hash_unit(uint64_t x) {
  // SplitMix64 finalizer (Steele, Lea, Flood 2014) -> uniform in [0, 1)
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

// Symmetric uniform[-0.5, 0.5) entries plus n on the diagonal: diagonally
// dominant, hence positive definite (the tuner's timing input).
__global__ void fill_spd(double* A, int64_t n, uint64_t seed) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / n, r = e - c * n;
    const int64_t lo = r < c ? r : c, hi = r < c ? c : r;
    A[e] = hash_unit(seed * 0x100000001B3ull + (uint64_t)(hi * n + lo)) - 0.5 + (r == c ? (double)n : 0.0);
  }
}

__global__ void fill_plain(double* p, int64_t cnt, uint64_t seed) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
    p[e] = hash_unit(seed * 0x100000001B3ull + (uint64_t)e) - 0.5;
}

int dev_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    sms = 152;
  }
  return sms;
}

int64_t step1_bytes_c(int nb) { return (int64_t)(2 + 2 * (int64_t)dev_sms()) * nb * nb * 8 + 256; }

int step1_time_c(int nb, int launches, double* sec, void* work, int64_t wbytes, cudaStream_t st) {
  const int nbatch = 2 * dev_sms();
  if (step1_bytes_c(nb) > wbytes) return -7;
  const size_t te = (size_t)nb * nb;
  double* A = (double*)work;
  double* B = A + te;
  double* C = B + te;
  fill_plain<<<1024, 256, 0, st>>>(A, (int64_t)(2 + nbatch) * te, 21);
  const size_t smem = kCSmemDoubles * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(gemm_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  gemm_batch<<<nbatch, CT, smem, st>>>(A, B, C, nb);  // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  if (launches <= 0) {  // as many launches as fill ~30 ms, 3 to the paper's 50
    cudaEventRecord(e0, st);
    gemm_batch<<<nbatch, CT, smem, st>>>(A, B, C, nb);
    cudaEventRecord(e1, st);
    float ms1 = 1.f;
    if ((e = cudaEventSynchronize(e1)) == cudaSuccess) e = cudaEventElapsedTime(&ms1, e0, e1);
    if (e != cudaSuccess) return (int)e;
    launches = std::max(3, std::min(50, (int)std::ceil(30.0 / std::max(ms1, 1e-3f))));
  }
  cudaEventRecord(e0, st);
  for (int l = 0; l < launches; ++l) gemm_batch<<<nbatch, CT, smem, st>>>(A, B, C, nb);
  cudaEventRecord(e1, st);
  float ms = 0.f;
  if ((e = cudaEventSynchronize(e1)) == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return (int)e;
  *sec = ms * 1e-3 / launches;
  return 0;
}

// reps timed factorizations of a fresh SPD matrix of order n (CUDA events
// around each call); median and minimum seconds. work holds A then scratch.
int time_chol(int64_t n, int nb, int reps, void* work, int64_t wbytes, cudaStream_t st, double* med, double* mn) {
  const size_t a_bytes = al256((size_t)n * n * 8);
  const CLayout L = chol_layout(n, nb);
  if ((int64_t)(a_bytes + L.bytes) > wbytes) return -7;
  double* A = (double*)work;
  void* scr = (char*)work + a_bytes;
  std::vector<double> ts;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int warm = n * n <= 4000000 ? 1 : 0;
  int rc = 0;
  for (int r = 1 - warm; r < reps + 1; ++r) {
    fill_spd<<<1184, 256, 0, st>>>(A, n, (uint64_t)n * 131 + 7);
    cudaEventRecord(e0, st);
    rc = chol_impl(n, A, n, nb, scr, (int64_t)L.bytes, st);
    cudaEventRecord(e1, st);
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      rc = (int)e;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    int st2[2] = {0, -1};
    const DevCtl* ctl = (const DevCtl*)scr;
    if ((e = cudaMemcpy(st2, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) {
      rc = (int)e;
      break;
    }
    if (st2[0]) {
      rc = 1000 + st2[0];
      break;
    }
    if (r > 0) ts.push_back(ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  std::sort(ts.begin(), ts.end());
  *med = ts.size() % 2 ? ts[ts.size() / 2] : 0.5 * (ts[ts.size() / 2 - 1] + ts[ts.size() / 2]);
  *mn = ts.front();
  return 0;
}

struct CEntry {
  int64_t n;
  int nb;
  double gflops;
};
std::mutex g_ctmu;
std::vector<CEntry> g_ctab;

}  // namespace

int chol_table_lookup(int64_t n, int* nb) {
  std::lock_guard<std::mutex> lock(g_ctmu);
  if (g_ctab.empty()) {
    *nb = 128;  // built-in default when nothing is tuned
    return 1;
  }
  const CEntry* best = &g_ctab[0];
  for (const CEntry& e : g_ctab) {
    const int64_t d = std::llabs(e.n - n), db = std::llabs(best->n - n);
    if (d < db || (d == db && e.n < best->n)) best = &e;
  }
  *nb = best->nb;
  return 0;
}

namespace {
void chol_append_log(const char* path, int kind, int64_t n, int nb, double sec, double smin, int reps) {
  if (!path || !path[0]) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"kind\": %d, \"n\": %lld, \"nb\": %d, \"seconds\": %.9g, \"min\": %.9g, \"reps\": %d}\n", kind,
          (long long)n, nb, sec, smin, reps);
  fclose(f);
}

void chol_read_log(const char* path, std::map<std::tuple<int, int64_t, int>, double>* seen) {
  if (!path || !path[0]) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof(line), f)) {
    int kind, nb;
    long long n;
    double sec;
    if (sscanf(line, "{\"kind\": %d, \"n\": %lld, \"nb\": %d, \"seconds\": %lf", &kind, &n, &nb, &sec) == 4)
      (*seen)[std::make_tuple(kind, (int64_t)n, nb)] = sec;
  }
  fclose(f);
}
}  // namespace

extern "C" {

int chol_workspace(int64_t n, int nb, int64_t* bytes) {
  if (n < 0) return -1;
  if (nb == 0) chol_table_lookup(n, &nb);
  if (nb < 16 || nb > 256 || nb % 16) return -2;
  if (!bytes) return -3;
  *bytes = n == 0 ? 256 : (int64_t)chol_layout(n, nb).bytes;
  return 0;
}

int chol_factor_d(int64_t n, double* A, int64_t lda, int nb, void* scratch, int64_t scratch_bytes, void* stream) {
  return chol_impl(n, A, lda, nb, scratch, scratch_bytes, stream);
}

int chol_status(const void* scratch, int* status, int64_t* first_bad_col, void* stream) {
  if (!scratch) return -1;
  if (!status) return -2;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return (int)e;
  int v[2] = {0, 0};
  if ((e = cudaMemcpy(&v[0], scratch, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpy(&v[1], (const char*)scratch + 64, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return (int)e;
  *status = v[0];
  if (first_bad_col) *first_bad_col = v[1] > 0 ? (int64_t)(INT_MAX - v[1]) : -1;
  return 0;
}

int64_t chol_task_count_n(int64_t n, int nb) {
  if (n < 1 || nb < 1) return 0;
  return chol_task_count((int)((n + nb - 1) / nb));
}

int chol_step1_workspace(int nb, int64_t* bytes) {
  if (nb < 16 || nb > 256 || nb % 16) return -1;
  if (!bytes) return -2;
  *bytes = step1_bytes_c(nb);
  return 0;
}

int chol_step1_time(int nb, int launches, double* seconds_per_launch, double* gflops, void* d_work, int64_t work_bytes,
                    void* stream) {
  if (nb < 16 || nb > 256 || nb % 16) return -1;
  if (!seconds_per_launch) return -3;
  if (!d_work) return -5;
  double s = 0;
  const int rc = step1_time_c(nb, launches, &s, d_work, work_bytes, (cudaStream_t)stream);
  if (rc) return rc;
  *seconds_per_launch = s;
  if (gflops) *gflops = 2.0 * dev_sms() * 2.0 * nb * (double)nb * nb / s / 1e9;
  return 0;
}

int chol_time_factor(int64_t n, int nb, int reps, double* median_s, double* min_s, void* d_work, int64_t work_bytes,
                     void* stream) {
  if (n < 1) return -1;
  if (nb < 16 || nb > 256 || nb % 16) return -2;
  if (reps < 1) return -3;
  if (!median_s || !min_s) return -4;
  if (!d_work) return -6;
  return time_chol(n, nb, reps, d_work, work_bytes, (cudaStream_t)stream, median_s, min_s);
}

int chol_tune_workspace(int64_t max_n, int64_t* bytes) {
  if (max_n < 1) return -1;
  if (!bytes) return -2;
  int64_t best = step1_bytes_c(256);
  for (int nb = 32; nb <= 256; nb += 32)
    best = std::max<int64_t>(best, (int64_t)(al256((size_t)max_n * max_n * 8) + chol_layout(max_n, nb).bytes));
  *bytes = best;
  return 0;
}

int chol_tune(const int64_t* ns, int nshapes, int heuristic, int reps, const char* table_path, const char* log_path,
              void* d_work, int64_t work_bytes, double* seconds_out, void* stream) {
  if (!ns || nshapes < 1) return -1;
  if (heuristic < 0 || heuristic > 2) return -3;
  if (reps < 1) return -4;
  if (!d_work) return -7;
  cudaStream_t st = (cudaStream_t)stream;
  const auto t_start = std::chrono::steady_clock::now();
  auto since = [](std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  };
  std::map<std::tuple<int, int64_t, int>, double> seen;
  chol_read_log(log_path, &seen);
  std::vector<int> grid;
  for (int nb = 32; nb <= 256; nb += 32) grid.push_back(nb);
  std::vector<int> ibs(grid.size(), 1);
  std::vector<double> perf(grid.size());
  double step1_s = 0, step2_s = 0;
  int measured = 0;
  for (size_t g = 0; g < grid.size(); ++g) {
    double s = 0, gf = 0;
    auto it = seen.find(std::make_tuple(11, (int64_t)0, grid[g]));
    if (it != seen.end()) {
      s = it->second;
    } else {
      const auto t0 = std::chrono::steady_clock::now();
      int rc = chol_step1_time(grid[g], 0, &s, &gf, d_work, work_bytes, stream);
      if (rc) return rc;
      step1_s += since(t0);
      chol_append_log(log_path, 11, 0, grid[g], s, s, 0);
    }
    perf[g] = 2.0 * dev_sms() * 2.0 * grid[g] * (double)grid[g] * grid[g] / s / 1e9;
  }
  std::vector<int> snb(grid.size()), sib(grid.size());
  const int k = qr_tune_preselect((int)grid.size(), grid.data(), ibs.data(), perf.data(), heuristic, 8, 8, snb.data(),
                                  sib.data());
  std::vector<int> surv(snb.begin(), snb.begin() + k);
  std::vector<int64_t> order(ns, ns + nshapes);
  std::sort(order.begin(), order.end());
  std::vector<CEntry> table;
  for (int64_t n : order) {
    std::vector<double> pf(surv.size());
    for (size_t c = 0; c < surv.size(); ++c) {
      double med = 0, mn = 0;
      auto it = seen.find(std::make_tuple(12, n, surv[c]));
      if (it != seen.end()) {
        med = it->second;
      } else {
        const auto t0 = std::chrono::steady_clock::now();
        int rc = time_chol(n, surv[c], reps, d_work, work_bytes, st, &med, &mn);
        if (rc) return rc;
        step2_s += since(t0);
        chol_append_log(log_path, 12, n, surv[c], med, mn, reps);
        ++measured;
      }
      pf[c] = (double)n * n * n / 3.0 / med / 1e9;
    }
    size_t bi = 0;
    for (size_t c = 1; c < surv.size(); ++c)
      if (pf[c] > pf[bi] || (pf[c] == pf[bi] && surv[c] < surv[bi])) bi = c;
    table.push_back(CEntry{n, surv[bi], pf[bi]});
    std::vector<int> keep(surv.size());
    qr_tune_payg((int)surv.size(), surv.data(), pf.data(), keep.data());  // Property 6.1
    std::vector<int> nx;
    for (size_t c = 0; c < surv.size(); ++c)
      if (keep[c]) nx.push_back(surv[c]);
    surv = nx;
  }
  const double total = since(t_start);
  if (seconds_out) {
    seconds_out[0] = total;
    seconds_out[1] = step1_s;
    seconds_out[2] = step2_s;
    seconds_out[3] = measured;
  }
  {
    std::lock_guard<std::mutex> lock(g_ctmu);
    g_ctab = table;
  }
  if (table_path && table_path[0]) {
    FILE* f = fopen(table_path, "w");
    if (!f) return -5;
    fprintf(f, "{\n  \"factorization\": \"cholesky\",\n  \"heuristic\": %d,\n  \"reps\": %d,\n  \"seconds\": %.3f,\n"
               "  \"step1_seconds\": %.3f,\n  \"step2_seconds\": %.3f,\n  \"entries\": [\n",
            heuristic, reps, total, step1_s, step2_s);
    for (size_t i = 0; i < table.size(); ++i)
      fprintf(f, "    {\"n\": %lld, \"nb\": %d, \"gflops\": %.4f}%s\n", (long long)table[i].n, table[i].nb,
              table[i].gflops, i + 1 < table.size() ? "," : "");
    fprintf(f, "  ]\n}\n");
    fclose(f);
  }
  return 0;
}

int chol_load_table(const char* path) {
  if (!path) return -1;
  FILE* f = fopen(path, "r");
  if (!f) return -1;
  std::string s;
  char buf[4096];
  size_t r;
  while ((r = fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, r);
  fclose(f);
  std::vector<CEntry> t;
  size_t p = s.find("\"entries\"");
  if (p == std::string::npos) return -1;
  while ((p = s.find("{\"n\":", p)) != std::string::npos) {
    CEntry e;
    long long n;
    if (sscanf(s.c_str() + p, "{\"n\": %lld, \"nb\": %d, \"gflops\": %lf", &n, &e.nb, &e.gflops) != 3) return -1;
    e.n = n;
    t.push_back(e);
    ++p;
  }
  std::lock_guard<std::mutex> lock(g_ctmu);
  g_ctab = t;
  return 0;
}

int chol_lookup(int64_t n, int* nb) {
  if (n < 0) return -1;
  if (!nb) return -2;
  chol_table_lookup(n, nb);
  return 0;
}

}  // extern "C"
