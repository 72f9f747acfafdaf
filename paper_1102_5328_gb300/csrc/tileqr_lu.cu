// Tile LU factorization with incremental (pairwise) pivoting on the
// persistent DAG scheduler: the other factorization the paper names for its
// tile framework and tuning method (Secs. 1 and 7; the paper tunes QR only).
// The DAG is the flat-tree tile QR's with the LU task kernels in place of
// the QR ones:
//   GETRF(k)       A_kk = L_kk U_kk, partial pivoting inside the tile
//   GESSM(k, j)    A_kj <- the same swaps and eliminations           (j > k)
//   TSTRF(i, k)    [U_kk; A_ik] = pairwise-pivoted LU: U_kk updated,
//                  A_ik <- its multipliers                          (i > k)
//   SSSSM(i, j, k) [A_kj; A_ij] <- TSTRF(i, k)'s swaps and eliminations
// Column c of GETRF takes the largest |entry| of rows c.. of the tile (first
// on ties); column c of TSTRF swaps in the largest |entry| of A_ik's column
// when it exceeds |U_kk(c, c)| strictly (first on ties). Swaps move columns
// c.. only, so every stored multiplier column is the one its step used (the
// factors are a sequence of elementary transformations; the upper triangle
// is U). Pivot records, caller-owned int32, tile (i, k) at
// d_piv[(k * NT + i) * NB + c]: GETRF the tile row swapped with c (c when
// none), TSTRF the row of A_ik swapped with U_kk's row c (-1 when none).
// A tile's counter counts the operations applied to it in program order; a
// task waits (bounded, acquire) for the counts it needs and publishes with a
// release increment, as the QR and Cholesky kernels do. FP64 on the CUDA
// cores: the FP64 pipe bounds every task (SSSSM keeps its bottom tile in
// registers, 16 entries a thread, and streams one column a step).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "layout.cuh"
#include "listsched.h"
#include "sched.cuh"
#include "tileqr_internal.h"

using namespace tqr;

// nb for an order n from the LU tuning table (closest tuned order, ties to
// the smaller); 64 when nothing is tuned (returns 1 then).
int lu_table_lookup(int64_t n, int* nb);

namespace {

constexpr int LT = 256;     // threads per CTA
constexpr int LMAX = 64;    // largest NB
constexpr int LLD = 65;     // staged tile leading dimension (odd: column walks change banks)
constexpr size_t kLSmemBytes = 2 * (size_t)LMAX * LLD * sizeof(double);

enum { LU_GETRF = 0, LU_GESSM = 1, LU_TSTRF = 2, LU_SSSSM = 3 };

__device__ __forceinline__ void stage_in(double* S, const double* g, int NB) {
  for (int e = threadIdx.x; e < NB * NB; e += LT) {
    const int c = e / NB, r = e - c * NB;
    S[r + c * LLD] = __ldcg(g + e);
  }
}

__device__ __forceinline__ void stage_out(double* g, const double* S, int NB) {
  for (int e = threadIdx.x; e < NB * NB; e += LT) {
    const int c = e / NB, r = e - c * NB;
    __stcg(g + e, S[r + c * LLD]);
  }
}

// A zero pivot: the status bit and the smallest such global column (kept as
// INT_MAX - column under atomicMax).
__device__ void record_zero_pivot(DevCtl* ctl, int* first_zero, int64_t col) {
  atomicOr(&ctl->status, QR_DEV_SINGULAR);
  atomicMax(first_zero, INT_MAX - (int)(col < INT_MAX - 1 ? col : INT_MAX - 1));
}

// Warp 0: the first row of [r0, r1) with the largest |S(r, c)|; r1 when
// none compares (all NaN).
__device__ __forceinline__ int warp_argmax(const double* S, int c, int r0, int r1, double* best) {
  const int lane = threadIdx.x & 31;
  double bv = -1.0;
  int bi = r1;
  for (int r = r0 + lane; r < r1; r += 32) {
    const double v = fabs(S[r + c * LLD]);
    if (v > bv) {
      bv = v;
      bi = r;
    }
  }
  for (int off = 16; off; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, bv, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (ov > bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  *best = bv;
  return bi;
}

struct LSm {
  double* s1;
  double* s2;
  int* piv;     // [LMAX]
  int* pick;    // one word: the column's pivot decision
};

// GETRF of the nk x nk tile T (tile layout, ld NB) in shared memory.
__device__ void getrf_task(double* T, int NB, int nk, int* piv_out, int64_t gcol0, DevCtl* ctl, int* first_zero,
                           const LSm& sm) {
  double* S = sm.s1;
  stage_in(S, T, NB);
  __syncthreads();
  for (int c = 0; c < nk; ++c) {
    if (threadIdx.x < 32) {
      double bv;
      int p = warp_argmax(S, c, c, nk, &bv);
      if (p >= nk) p = c;
      if (threadIdx.x == 0) {
        *sm.pick = p;
        sm.piv[c] = p;
      }
    }
    __syncthreads();
    const int p = *sm.pick;
    if (p != c)
      for (int j = c + threadIdx.x; j < nk; j += LT) {
        const double t = S[c + j * LLD];
        S[c + j * LLD] = S[p + j * LLD];
        S[p + j * LLD] = t;
      }
    __syncthreads();
    const double d = S[c + c * LLD];
    if (d == 0.0) {
      if (threadIdx.x == 0) record_zero_pivot(ctl, first_zero, gcol0 + c);
      continue;  // uniform: every thread read the same d
    }
    for (int r = c + 1 + threadIdx.x; r < nk; r += LT) S[r + c * LLD] /= d;
    __syncthreads();
    const int rows = nk - c - 1, cols = nk - c - 1;
    for (int e = threadIdx.x; e < rows * cols; e += LT) {
      const int jj = e / rows, rr = e - jj * rows;
      const int r = c + 1 + rr, j = c + 1 + jj;
      S[r + j * LLD] = fma(-S[r + c * LLD], S[c + j * LLD], S[r + j * LLD]);
    }
    __syncthreads();
  }
  stage_out(T, S, NB);
  for (int c = threadIdx.x; c < nk; c += LT) piv_out[c] = sm.piv[c];
}

// GESSM: X (nk x nj, tile layout) <- the swaps and eliminations of GETRF(k)
// (multipliers in the strictly lower triangle of Lt, records piv_in).
__device__ void gessm_task(double* X, const double* Lt, int NB, int nk, int nj, const int* piv_in, const LSm& sm) {
  double* S = sm.s1;
  double* L = sm.s2;
  stage_in(S, X, NB);
  // the strictly lower triangle only: TSTRF tasks of the same step rewrite
  // the upper one meanwhile
  for (int e = threadIdx.x; e < NB * NB; e += LT) {
    const int c = e / NB, r = e - c * NB;
    L[r + c * LLD] = r > c ? __ldcg(Lt + e) : 0.0;
  }
  for (int c = threadIdx.x; c < nk; c += LT) sm.piv[c] = __ldcg(piv_in + c);
  __syncthreads();
  for (int c = 0; c < nk; ++c) {
    const int p = sm.piv[c];
    if (p != c) {
      for (int j = threadIdx.x; j < nj; j += LT) {
        const double t = S[c + j * LLD];
        S[c + j * LLD] = S[p + j * LLD];
        S[p + j * LLD] = t;
      }
      __syncthreads();
    }
    const int rows = nk - c - 1;
    for (int e = threadIdx.x; e < rows * nj; e += LT) {
      const int j = e / rows, r = c + 1 + (e - j * rows);
      S[r + j * LLD] = fma(-L[r + c * LLD], S[c + j * LLD], S[r + j * LLD]);
    }
    __syncthreads();
  }
  stage_out(X, S, NB);
}

// TSTRF: [U; B] with U the upper triangle of Ut (nk x nk; its strictly lower
// part, GETRF's multipliers, is neither read nor written) and B (ni x nk).
__device__ void tstrf_task(double* Ut, double* Bt, int NB, int ni, int nk, int* piv_out, int64_t gcol0, DevCtl* ctl,
                           int* first_zero, const LSm& sm) {
  double* U = sm.s1;
  double* B = sm.s2;
  stage_in(U, Ut, NB);
  stage_in(B, Bt, NB);
  __syncthreads();
  for (int c = 0; c < nk; ++c) {
    if (threadIdx.x < 32) {
      double bv;
      const int r = warp_argmax(B, c, 0, ni, &bv);
      if (threadIdx.x == 0) {
        const int pick = (r < ni && bv > fabs(U[c + c * LLD])) ? r : -1;
        *sm.pick = pick;
        sm.piv[c] = pick;
      }
    }
    __syncthreads();
    const int r = *sm.pick;
    if (r >= 0) {
      for (int j = c + threadIdx.x; j < nk; j += LT) {
        const double t = U[c + j * LLD];
        U[c + j * LLD] = B[r + j * LLD];
        B[r + j * LLD] = t;
      }
      __syncthreads();
    }
    const double d = U[c + c * LLD];
    if (d == 0.0) {
      if (threadIdx.x == 0) record_zero_pivot(ctl, first_zero, gcol0 + c);
      continue;
    }
    for (int rr = threadIdx.x; rr < ni; rr += LT) B[rr + c * LLD] /= d;
    __syncthreads();
    const int cols = nk - c - 1;
    for (int e = threadIdx.x; e < ni * cols; e += LT) {
      const int jj = e / ni, rr = e - jj * ni;
      const int j = c + 1 + jj;
      B[rr + j * LLD] = fma(-B[rr + c * LLD], U[c + j * LLD], B[rr + j * LLD]);
    }
    __syncthreads();
  }
  // U's upper triangle only: GESSM tasks of the same step read the lower one
  for (int e = threadIdx.x; e < NB * NB; e += LT) {
    const int c = e / NB, r = e - c * NB;
    if (r <= c) __stcg(Ut + e, U[r + c * LLD]);
  }
  stage_out(Bt, B, NB);
  for (int c = threadIdx.x; c < nk; c += LT) piv_out[c] = sm.piv[c];
}

// SSSSM: [X; Y] (X nk x nj, Y ni x nj) <- TSTRF(i, k)'s swaps and
// eliminations (multipliers Lt, ni x nk; records piv_in). Y lives in
// registers: thread (tx, ty) of 16 x 16 holds rows tx + 16 a, columns
// ty + 16 b, a, b < 4; X and the multipliers are staged in shared memory.
__device__ void ssssm_task(double* Xt, double* Yt, const double* Lt, int NB, int nk, const int* piv_in,
                           const LSm& sm) {
  double* X = sm.s1;
  double* L = sm.s2;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  stage_in(X, Xt, NB);
  stage_in(L, Lt, NB);
  for (int c = threadIdx.x; c < nk; c += LT) sm.piv[c] = __ldcg(piv_in + c);
  double y[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = tx + 16 * a, col = ty + 16 * b;
      y[a][b] = (r < NB && col < NB) ? __ldcg(Yt + r + (size_t)col * NB) : 0.0;
    }
  __syncthreads();
  for (int c = 0; c < nk; ++c) {
    const int r = sm.piv[c];
    if (r >= 0) {
      // the owners of Y's row r exchange it with X's row c (each column once)
      if ((r & 15) == tx) {
        const int ra = r >> 4;  // selects with constant indices keep y in registers
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int col = ty + 16 * b;
          if (col < NB) {
            const double xv = X[c + col * LLD];
            const double t = ra == 0 ? y[0][b] : (ra == 1 ? y[1][b] : (ra == 2 ? y[2][b] : y[3][b]));
            y[0][b] = ra == 0 ? xv : y[0][b];
            y[1][b] = ra == 1 ? xv : y[1][b];
            y[2][b] = ra == 2 ? xv : y[2][b];
            y[3][b] = ra == 3 ? xv : y[3][b];
            X[c + col * LLD] = t;
          }
        }
      }
      __syncthreads();
    }
    double l[4], u[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) l[a] = (tx + 16 * a < NB) ? L[tx + 16 * a + c * LLD] : 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b) u[b] = (ty + 16 * b < NB) ? X[c + (ty + 16 * b) * LLD] : 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) y[a][b] = fma(-l[a], u[b], y[a][b]);
  }
  __syncthreads();
  stage_out(Xt, X, NB);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = tx + 16 * a, col = ty + 16 * b;
      if (r < NB && col < NB) __stcg(Yt + r + (size_t)col * NB, y[a][b]);
    }
}

struct LuArgs {
  double* W;
  int* piv;
  int64_t n;
  int NB, NT;
  const uint64_t* tasks;
  int64_t ntasks;
  unsigned* cnt;  // NT x NT
  DevCtl* ctl;
  int* first_zero;
  uint64_t timeout_ns;
  TraceRec* trace;
  int64_t trace_cap;
};

__global__ void __launch_bounds__(LT, 2) persistent_lu(LuArgs a) {
  extern __shared__ __align__(16) double lsm_raw[];
  __shared__ int s_piv[LMAX];
  __shared__ int s_pick;
  __shared__ int64_t s_ticket;
  __shared__ int s_ok;
  LSm sm;
  sm.s1 = lsm_raw;
  sm.s2 = lsm_raw + LMAX * LLD;
  sm.piv = s_piv;
  sm.pick = &s_pick;
  const int NB = a.NB, NT = a.NT;
  const size_t te = (size_t)NB * NB;
  auto tile = [&](int i, int j) { return a.W + ((size_t)j * NT + i) * te; };
  auto pv = [&](int i, int k) { return a.piv + ((size_t)k * NT + i) * NB; };
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
        case LU_GETRF: ok = wait_ge(ctr(k, k), 1, (unsigned)k, a.ctl, to); break;
        case LU_GESSM:
          ok = wait_ge(ctr(k, k), 1, (unsigned)k + 1, a.ctl, to) && wait_ge(ctr(k, j), 1, (unsigned)k, a.ctl, to);
          break;
        case LU_TSTRF:
          ok = wait_ge(ctr(k, k), 1, (unsigned)i, a.ctl, to) && wait_ge(ctr(i, k), 1, (unsigned)k, a.ctl, to);
          break;
        default:
          ok = wait_ge(ctr(i, k), 1, (unsigned)k + 1, a.ctl, to) && wait_ge(ctr(k, j), 1, (unsigned)i, a.ctl, to) &&
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
      case LU_GETRF: getrf_task(tile(k, k), NB, nk, pv(k, k), (int64_t)k * NB, a.ctl, a.first_zero, sm); break;
      case LU_GESSM: gessm_task(tile(k, j), tile(k, k), NB, nk, dim_of(j), pv(k, k), sm); break;
      case LU_TSTRF:
        tstrf_task(tile(k, k), tile(i, k), NB, dim_of(i), nk, pv(i, k), (int64_t)k * NB, a.ctl, a.first_zero, sm);
        break;
      default: ssssm_task(tile(k, j), tile(i, j), tile(i, k), NB, nk, pv(i, k), sm); break;
    }
    // publish: every thread's stores precede thread 0's fence and release
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      switch (type) {
        case LU_GETRF: red_release_add(ctr(k, k), 1u); break;
        case LU_GESSM: red_release_add(ctr(k, j), 1u); break;
        case LU_TSTRF:
          red_release_add(ctr(k, k), 1u);
          red_release_add(ctr(i, k), 1u);
          break;
        default:
          red_release_add(ctr(k, j), 1u);
          red_release_add(ctr(i, j), 1u);
          break;
      }
      trace_put(a.trace, a.trace_cap, t, type, t_take, t_ready);
    }
  }
}

// ---------------------------------------------------------------------------
// Host: layout, the ticket order, launch.
size_t al256l(size_t x) { return (x + 255) & ~(size_t)255; }

int64_t lu_task_count(int NT) {
  int64_t c = 0;
  for (int k = 0; k < NT; ++k) {
    const int64_t r = NT - k - 1;
    c += 1 + 2 * r + r * r;
  }
  return c;
}

struct LLayout {
  int NT;
  int64_t ntasks;
  size_t off_cnt, off_tasks, off_tiles, bytes;
};

LLayout lu_layout(int64_t n, int nb) {
  LLayout L;
  L.NT = (int)((n + nb - 1) / nb);
  L.ntasks = lu_task_count(L.NT);
  L.off_cnt = 256;  // DevCtl at 0, the first zero pivot at 64
  L.off_tasks = al256l(L.off_cnt + (size_t)L.NT * L.NT * 4);
  L.off_tiles = al256l(L.off_tasks + (size_t)L.ntasks * 8);
  L.bytes = al256l(L.off_tiles + (size_t)L.NT * L.NT * nb * nb * 8);
  return L;
}

std::mutex g_lmu;
std::map<std::pair<int, int>, std::vector<uint64_t>> g_lorders;  // (NT, workers) -> ticket order (host copy)

// Program order (k-major, topological) with direct predecessors (the last
// task that wrote each tile a task reads or writes), then the list schedule
// for the kernel's workers. Costs in NB^3 multiply-adds: GETRF 1/3 weighted
// 4x for its serial column chain, GESSM 1/2, TSTRF 1/2 weighted 4x, SSSSM 1.
const std::vector<uint64_t>& lu_order(int NT, int workers) {
  auto key = std::make_pair(NT, workers);
  auto it = g_lorders.find(key);
  if (it != g_lorders.end()) return it->second;
  std::vector<uint64_t> code;
  std::vector<double> w;
  std::vector<int64_t> poff{0};
  std::vector<int32_t> pred;
  std::map<std::pair<int, int>, int32_t> last;
  auto writer = [&](int i, int j) {
    auto f = last.find(std::make_pair(i, j));
    return f == last.end() ? -1 : f->second;
  };
  auto add = [&](int type, int i, int j, int k, double cost, std::initializer_list<int32_t> deps) {
    std::vector<int32_t> d;
    for (int32_t x : deps)
      if (x >= 0 && std::find(d.begin(), d.end(), x) == d.end()) d.push_back(x);
    pred.insert(pred.end(), d.begin(), d.end());
    code.push_back(encode_task(type, 0, i, j, k));
    w.push_back(cost);
    poff.push_back((int64_t)pred.size());
    return (int32_t)(code.size() - 1);
  };
  for (int k = 0; k < NT; ++k) {
    const int32_t g = add(LU_GETRF, k, k, k, 4.0 / 3.0, {writer(k, k)});
    last[{k, k}] = g;
    for (int j = k + 1; j < NT; ++j) last[{k, j}] = add(LU_GESSM, k, j, k, 0.5, {g, writer(k, j)});
    for (int i = k + 1; i < NT; ++i) {
      const int32_t ts = add(LU_TSTRF, i, k, k, 2.0, {writer(k, k), writer(i, k)});
      last[{k, k}] = ts;
      last[{i, k}] = ts;
      for (int j = k + 1; j < NT; ++j) {
        const int32_t s = add(LU_SSSSM, i, j, k, 1.0, {ts, writer(k, j), writer(i, j)});
        last[{k, j}] = s;
        last[{i, j}] = s;
      }
    }
  }
  const std::vector<int64_t> idx = list_schedule(w, poff, pred, workers);
  std::vector<uint64_t> order(code.size());
  for (size_t t = 0; t < idx.size(); ++t) order[t] = code[idx[t]];
  return g_lorders.emplace(key, std::move(order)).first->second;
}

int lu_grid(int* grid_out, int* workers) {
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
  if ((e = cudaFuncSetAttribute(persistent_lu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLSmemBytes)) !=
      cudaSuccess)
    return (int)e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_lu, LT, kLSmemBytes)) != cudaSuccess)
    return (int)e;
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

int lu_args_check(int64_t n, int nb) {
  if (n < 0) return -1;
  if (nb < 8 || nb > LMAX) return -4;
  if ((n + nb - 1) / nb > 65535) return -1;
  return 0;
}

int lu_impl(int64_t n, double* A, int64_t lda, int nb, int* d_piv, void* scratch, int64_t scratch_bytes,
            void* stream) {
  if (n < 0) return -1;
  if (!A && n > 0) return -2;
  if (lda < std::max<int64_t>(n, 1)) return -3;
  if (nb == 0) lu_table_lookup(n, &nb);
  if (int rc = lu_args_check(n, nb)) return rc;
  if (n == 0) return 0;
  if (!d_piv) return -5;
  if (!scratch) return -6;
  cudaStream_t st = (cudaStream_t)stream;
  const LLayout L = lu_layout(n, nb);
  if (scratch_bytes < (int64_t)L.bytes) return -7;
  int grid = 0, workers = 0;
  int rc = lu_grid(&grid, &workers);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_lmu);
  const std::vector<uint64_t>& order = lu_order(L.NT, workers);
  char* base = (char*)scratch;
  cudaError_t e = cudaMemcpyAsync(base + L.off_tasks, order.data(), order.size() * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return (int)e;  // cached orders are never freed: the host copy outlives the copy
  double* W = (double*)(base + L.off_tiles);
  const int64_t nzero = (int64_t)(L.off_cnt / 4) + (int64_t)L.NT * L.NT;
  cm_to_tiles<double><<<1184, 256, 0, st>>>(A, lda, n, n, W, nb, L.NT, L.NT, (unsigned*)base, nzero);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  LuArgs la;
  la.W = W; la.piv = d_piv; la.n = n; la.NB = nb; la.NT = L.NT;
  la.tasks = (const uint64_t*)(base + L.off_tasks); la.ntasks = (int64_t)order.size();
  la.cnt = (unsigned*)(base + L.off_cnt); la.ctl = (DevCtl*)base; la.first_zero = (int*)(base + 64);
  la.timeout_ns = (uint64_t)qr_get_option(QR_OPT_WAIT_TIMEOUT_US) * 1000ull;
  {
    void* tb = nullptr;
    int64_t tcap = 0;
    qr_trace_target(&tb, &tcap);
    la.trace = (TraceRec*)tb;
    la.trace_cap = tcap;
  }
  persistent_lu<<<grid, LT, kLSmemBytes, st>>>(la);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  tiles_to_cm<double><<<1184, 256, 0, st>>>(W, A, lda, n, n, nb, L.NT);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  return 0;
}

// ---------------------------------------------------------------------------
// The empirical NB tuner of the LU, Secs. 5–6 applied to its one tuning
// parameter: Step 1 times the dominant task (SSSSM, about NT^3 / 3 of them)
// on a device-filling batch for every NB of the grid {16, 24, ..., 64}; the
// upper hull of (NB, GFLOP/s) and Heuristic 0/1/2 (qr_tune_preselect)
// preselect; Step 2 times the factorization for the survivors at each
// order, ascending, and prunes with Property 6.1 (qr_tune_payg); untuned
// orders take the closest tuned one.
__global__ void __launch_bounds__(LT, 2) ssssm_batch(double* X, double* Y, const double* L, const int* piv, int NB) {
  extern __shared__ __align__(16) double bsm_raw[];
  __shared__ int s_piv[LMAX];
  __shared__ int s_pick;
  LSm sm;
  sm.s1 = bsm_raw;
  sm.s2 = bsm_raw + LMAX * LLD;
  sm.piv = s_piv;
  sm.pick = &s_pick;
  const size_t te = (size_t)NB * NB;
  ssssm_task(X + blockIdx.x * te, Y + blockIdx.x * te, L, NB, NB, piv, sm);
}

__device__ __forceinline__ double lu_hash_unit(uint64_t x) {
  // SplitMix64 finalizer (Steele, Lea, Flood 2014) -> uniform in [0, 1)
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void lu_fill(double* p, int64_t cnt, uint64_t seed) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
    p[e] = lu_hash_unit(seed * 0x100000001B3ull + (uint64_t)e) - 0.5;
}

// Step-1 pivot records: every other column swaps with a row of the tile
// below, the others keep U's row (random matrices swap about that often).
__global__ void lu_fill_piv(int* piv, int NB) {
  for (int c = threadIdx.x; c < NB; c += blockDim.x) piv[c] = (c & 1) ? -1 : (c * 7) % NB;
}

int lu_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    sms = 152;
  }
  return sms;
}

int64_t lu_step1_bytes(int nb) { return (int64_t)(1 + 4 * (int64_t)lu_sms()) * nb * nb * 8 + 256 + 4 * LMAX; }

int lu_step1_run(int nb, int launches, double* sec, void* work, int64_t wbytes, cudaStream_t st) {
  const int nbatch = 2 * lu_sms();
  if (lu_step1_bytes(nb) > wbytes) return -7;
  const size_t te = (size_t)nb * nb;
  int* piv = (int*)work;
  double* L = (double*)((char*)work + 256 + 4 * LMAX);
  double* X = L + te;
  double* Y = X + nbatch * te;
  lu_fill<<<1024, 256, 0, st>>>(L, (int64_t)(1 + 2 * nbatch) * te, 23);
  lu_fill_piv<<<1, 64, 0, st>>>(piv, nb);
  cudaError_t e = cudaFuncSetAttribute(ssssm_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLSmemBytes);
  if (e != cudaSuccess) return (int)e;
  ssssm_batch<<<nbatch, LT, kLSmemBytes, st>>>(X, Y, L, piv, nb);  // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  if (launches <= 0) {  // as many launches as fill ~30 ms, 3 to the paper's 50
    cudaEventRecord(e0, st);
    ssssm_batch<<<nbatch, LT, kLSmemBytes, st>>>(X, Y, L, piv, nb);
    cudaEventRecord(e1, st);
    float ms1 = 1.f;
    if ((e = cudaEventSynchronize(e1)) == cudaSuccess) e = cudaEventElapsedTime(&ms1, e0, e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return (int)e;
    }
    launches = std::max(3, std::min(50, (int)std::ceil(30.0 / std::max(ms1, 1e-3f))));
  }
  cudaEventRecord(e0, st);
  for (int l = 0; l < launches; ++l) ssssm_batch<<<nbatch, LT, kLSmemBytes, st>>>(X, Y, L, piv, nb);
  cudaEventRecord(e1, st);
  float ms = 0.f;
  if ((e = cudaEventSynchronize(e1)) == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return (int)e;
  *sec = ms * 1e-3 / launches;
  return 0;
}

// reps timed factorizations of a fresh uniform matrix of order n (CUDA
// events around each call; the refill is outside them); median and minimum
// seconds. work holds A, the pivot records, then the scratch.
int time_lu(int64_t n, int nb, int reps, void* work, int64_t wbytes, cudaStream_t st, double* med, double* mn) {
  const size_t a_bytes = al256l((size_t)n * n * 8);
  const LLayout L = lu_layout(n, nb);
  const size_t p_bytes = al256l((size_t)L.NT * L.NT * nb * 4);
  if ((int64_t)(a_bytes + p_bytes + L.bytes) > wbytes) return -7;
  double* A = (double*)work;
  int* piv = (int*)((char*)work + a_bytes);
  void* scr = (char*)work + a_bytes + p_bytes;
  std::vector<double> ts;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int warm = n * n <= 4000000 ? 1 : 0;
  int rc = 0;
  for (int r = 1 - warm; r < reps + 1; ++r) {
    lu_fill<<<1184, 256, 0, st>>>(A, n * n, (uint64_t)n * 131 + 11);
    cudaEventRecord(e0, st);
    rc = lu_impl(n, A, n, nb, piv, scr, (int64_t)L.bytes, st);
    cudaEventRecord(e1, st);
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      rc = (int)e;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    int stat = 0;
    if ((e = cudaMemcpy(&stat, scr, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) {
      rc = (int)e;
      break;
    }
    if (stat) {
      rc = 1000 + stat;
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

struct LEntry {
  int64_t n;
  int nb;
  double gflops;
};
std::mutex g_ltmu;
std::vector<LEntry> g_ltab;

void lu_append_log(const char* path, int kind, int64_t n, int nb, double sec, double smin, int reps) {
  if (!path || !path[0]) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"kind\": %d, \"n\": %lld, \"nb\": %d, \"seconds\": %.9g, \"min\": %.9g, \"reps\": %d}\n", kind,
          (long long)n, nb, sec, smin, reps);
  fclose(f);
}

void lu_read_log(const char* path, std::map<std::tuple<int, int64_t, int>, double>* seen) {
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

bool lu_nb_ok(int nb) { return nb >= 8 && nb <= LMAX; }

}  // namespace

extern "C" {

int lu_workspace(int64_t n, int nb, int64_t* piv_elems, int64_t* scratch_bytes) {
  if (nb == 0) lu_table_lookup(n, &nb);
  if (int rc = lu_args_check(n, nb)) return rc;
  const LLayout L = lu_layout(std::max<int64_t>(n, 1), nb);
  if (piv_elems) *piv_elems = (int64_t)L.NT * L.NT * nb;
  if (scratch_bytes) *scratch_bytes = (int64_t)L.bytes;
  return 0;
}

int64_t lu_task_count_n(int64_t n, int nb) {
  if (nb == 0) lu_table_lookup(n, &nb);
  if (lu_args_check(n, nb)) return -1;
  return lu_task_count((int)((n + nb - 1) / nb));
}

int lu_factor_d(int64_t n, double* d_A, int64_t lda, int nb, int* d_piv, void* d_scratch, int64_t scratch_bytes,
                void* stream) {
  return lu_impl(n, d_A, lda, nb, d_piv, d_scratch, scratch_bytes, stream);
}

int lu_status(const void* d_scratch, int* status, int64_t* first_zero_col, void* stream) {
  if (!d_scratch) return -1;
  if (!status) return -2;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return (int)e;
  int words[2] = {0, 0};
  if ((e = cudaMemcpy(&words[0], d_scratch, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) return (int)e;
  if ((e = cudaMemcpy(&words[1], (const char*)d_scratch + 64, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return (int)e;
  *status = words[0];
  if (first_zero_col) *first_zero_col = words[1] > 0 ? (int64_t)(INT_MAX - words[1]) : -1;
  return 0;
}

int lu_step1_workspace(int nb, int64_t* bytes) {
  if (!lu_nb_ok(nb)) return -1;
  if (!bytes) return -2;
  *bytes = lu_step1_bytes(nb);
  return 0;
}

int lu_step1_time(int nb, int launches, double* seconds_per_launch, double* gflops, void* d_work, int64_t work_bytes,
                  void* stream) {
  if (!lu_nb_ok(nb)) return -1;
  if (!seconds_per_launch) return -3;
  if (!d_work) return -5;
  double s = 0;
  const int rc = lu_step1_run(nb, launches, &s, d_work, work_bytes, (cudaStream_t)stream);
  if (rc) return rc;
  *seconds_per_launch = s;
  if (gflops) *gflops = 2.0 * lu_sms() * 2.0 * nb * (double)nb * nb / s / 1e9;
  return 0;
}

int lu_time_factor(int64_t n, int nb, int reps, double* median_s, double* min_s, void* d_work, int64_t work_bytes,
                   void* stream) {
  if (n < 1) return -1;
  if (!lu_nb_ok(nb)) return -2;
  if (reps < 1) return -3;
  if (!median_s || !min_s) return -4;
  if (!d_work) return -6;
  return time_lu(n, nb, reps, d_work, work_bytes, (cudaStream_t)stream, median_s, min_s);
}

int lu_tune_workspace(int64_t max_n, int64_t* bytes) {
  if (max_n < 1 || (max_n + 7) / 8 > 65535) return -1;
  if (!bytes) return -2;
  int64_t best = lu_step1_bytes(LMAX);
  for (int nb = 16; nb <= LMAX; nb += 8) {
    const LLayout L = lu_layout(max_n, nb);
    best = std::max<int64_t>(best, (int64_t)(al256l((size_t)max_n * max_n * 8) +
                                              al256l((size_t)L.NT * L.NT * nb * 4) + L.bytes));
  }
  *bytes = best;
  return 0;
}

int lu_tune(const int64_t* ns, int nshapes, int heuristic, int reps, const char* table_path, const char* log_path,
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
  lu_read_log(log_path, &seen);
  std::vector<int> grid;
  for (int nb = 16; nb <= LMAX; nb += 8) grid.push_back(nb);
  std::vector<int> ibs(grid.size(), 1);
  std::vector<double> perf(grid.size());
  double step1_s = 0, step2_s = 0;
  int measured = 0;
  for (size_t g = 0; g < grid.size(); ++g) {
    double s = 0, gf = 0;
    auto it = seen.find(std::make_tuple(21, (int64_t)0, grid[g]));
    if (it != seen.end()) {
      s = it->second;
    } else {
      const auto t0 = std::chrono::steady_clock::now();
      int rc = lu_step1_time(grid[g], 0, &s, &gf, d_work, work_bytes, stream);
      if (rc) return rc;
      step1_s += since(t0);
      lu_append_log(log_path, 21, 0, grid[g], s, s, 0);
    }
    perf[g] = 2.0 * lu_sms() * 2.0 * grid[g] * (double)grid[g] * grid[g] / s / 1e9;
  }
  std::vector<int> snb(grid.size()), sib(grid.size());
  const int k = qr_tune_preselect((int)grid.size(), grid.data(), ibs.data(), perf.data(), heuristic, 8, 8, snb.data(),
                                  sib.data());
  if (k < 1) return -8;
  std::vector<int> surv(snb.begin(), snb.begin() + k);
  std::vector<int64_t> order(ns, ns + nshapes);
  std::sort(order.begin(), order.end());
  std::vector<LEntry> table;
  for (int64_t n : order) {
    std::vector<double> pf(surv.size());
    for (size_t c = 0; c < surv.size(); ++c) {
      double med = 0, mn = 0;
      auto it = seen.find(std::make_tuple(22, n, surv[c]));
      if (it != seen.end()) {
        med = it->second;
      } else {
        const auto t0 = std::chrono::steady_clock::now();
        int rc = time_lu(n, surv[c], reps, d_work, work_bytes, st, &med, &mn);
        if (rc) return rc;
        step2_s += since(t0);
        lu_append_log(log_path, 22, n, surv[c], med, mn, reps);
        ++measured;
      }
      pf[c] = 2.0 * (double)n * n * n / 3.0 / med / 1e9;
    }
    size_t bi = 0;
    for (size_t c = 1; c < surv.size(); ++c)
      if (pf[c] > pf[bi] || (pf[c] == pf[bi] && surv[c] < surv[bi])) bi = c;
    table.push_back(LEntry{n, surv[bi], pf[bi]});
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
    std::lock_guard<std::mutex> lock(g_ltmu);
    g_ltab = table;
  }
  if (table_path && table_path[0]) {
    FILE* f = fopen(table_path, "w");
    if (!f) return -5;
    fprintf(f, "{\n  \"factorization\": \"lu\",\n  \"heuristic\": %d,\n  \"reps\": %d,\n  \"seconds\": %.3f,\n"
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

int lu_load_table(const char* path) {
  if (!path) return -1;
  FILE* f = fopen(path, "r");
  if (!f) return -1;
  std::string s;
  char buf[4096];
  size_t r;
  while ((r = fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, r);
  fclose(f);
  std::vector<LEntry> t;
  size_t p = s.find("\"entries\"");
  if (p == std::string::npos) return -1;
  while ((p = s.find("{\"n\":", p)) != std::string::npos) {
    LEntry e;
    long long n;
    if (sscanf(s.c_str() + p, "{\"n\": %lld, \"nb\": %d, \"gflops\": %lf", &n, &e.nb, &e.gflops) != 3) return -1;
    if (!lu_nb_ok(e.nb)) return -1;
    e.n = n;
    t.push_back(e);
    ++p;
  }
  std::lock_guard<std::mutex> lock(g_ltmu);
  g_ltab = t;
  return 0;
}

int lu_lookup(int64_t n, int* nb) {
  if (n < 0) return -1;
  if (!nb) return -2;
  lu_table_lookup(n, nb);
  return 0;
}

int lu_clear_table(void) {
  std::lock_guard<std::mutex> lock(g_ltmu);
  g_ltab.clear();
  return 0;
}

}  // extern "C"

int lu_table_lookup(int64_t n, int* nb) {
  std::lock_guard<std::mutex> lock(g_ltmu);
  if (g_ltab.empty()) {
    *nb = LMAX;  // built-in default when nothing is tuned
    return 1;
  }
  const LEntry* best = &g_ltab[0];
  for (const LEntry& e : g_ltab) {
    const int64_t d = std::llabs(e.n - n), db = std::llabs(best->n - n);
    if (d < db || (d == db && e.n < best->n)) best = &e;
  }
  *nb = best->nb;
  return 0;
}
