// Tile QR factorization: layout conversion, the persistent DAG scheduler and
// the C-ABI entry points qr_workspace / qr_factor_{d,s} / qr_status.
//
// Sec. 2.1 of the paper: the matrix is cut into tiles of order NB and QR is
// a DAG of GEQRT, TSQRT, UNMQR and TSMQR tasks. Its multicore runtime
// schedules the DAG statically over cores; here one persistent kernel keeps
// every SM resident and hands out tasks through a global ticket counter in a
// topological order computed on the host (earliest-start-time order of the
// DAG, which pulls panel tasks of later steps forward - a look-ahead). A task
// waits on per-tile progress counters (acquire loads with a time limit), runs
// on its CTA, and publishes its tiles with a release increment.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "layout.cuh"
#include "listsched.h"
#include "sched.cuh"
#include "tile_kernels.cuh"
#include "tileqr_internal.h"

using namespace tqr;

namespace {

std::mutex g_mu;
int64_t g_wait_timeout_us = 20LL * 1000 * 1000;
std::atomic<void*> g_trace{nullptr};
std::atomic<int64_t> g_trace_cap{0};
int g_ctas_per_sm = 0;
int g_split = 0;
int g_order = 1;  // ticket order of the flat tree: 0 earliest start time, 1 list schedule
int g_wpanel = 150;  // list-schedule cost of GEQRT/TSQRT, percent of their flops
int g_wunmqr = 100;  // list-schedule cost of UNMQR, percent of its flops
// measured task costs (GEQRT, UNMQR, TSQRT, TSMQR service times, any unit)
// per (precision, NB, IB), installed by qr_set_task_costs; they replace the
// flop-count weights of the list schedule for that configuration
std::map<std::tuple<int, int, int>, std::array<double, 4>> g_costs;
int g_grid_limit = 0;
int g_sm_budget = 0;  // QR_OPT_SM_BUDGET: SMs' worth of persistent CTAs (0 = all)
int64_t g_drop_task = -1;
int g_record = 0;
int g_ls_refine = 0;     // QR_OPT_LS_REFINE
int g_gmres_max = 50;    // QR_OPT_GMRES_MAX
int g_gmres_tol_exp = 6;  // QR_OPT_GMRES_TOL_EXP
int g_tune_ib_tol = 0;    // QR_OPT_TUNE_IB_TOL (1/1000)
cudaEvent_t g_ev[2] = {nullptr, nullptr};
bool g_ev_pending = false;

struct Layout {
  int64_t m, n;
  int NB, IB, MT, NT, S;
  int64_t ntasks;
  size_t off_cnt, off_tasks, off_tiles, bytes;
  int64_t t_elems;
};

// Column chunks per update task. FP64: from NB = 128 on, two chunks run as
// separate tasks on two CTAs (measured on the GB300: N = 10000 at NB = 128
// 1076 -> 1094 GFLOP/s, N = 8000 1028 -> 1068; the chain of panel tasks and
// the start and end of the run get twice the parallel work, and a chunk
// costs what the same columns cost inside one task); NB = 64 keeps one (a
// 32-column chunk leaves three quarters of the CTA idle). FP32 tasks are
// latency-bound and keep one chunk up to NB = 160.
int auto_split(int NB, size_t esz) {
  if (g_split > 0) return g_split;
  if (NB <= (esz == 8 ? 96 : 160)) return 1;
  if (NB <= 320) return 2;
  return 4;
}

int64_t count_tasks(int MT, int NT, int S) {
  int64_t c = 0;
  const int K = std::min(MT, NT);
  for (int k = 0; k < K; ++k) {
    c += 1 + (int64_t)(NT - k - 1) * S;
    c += (int64_t)(MT - k - 1) * (1 + (int64_t)(NT - k - 1) * S);
  }
  return c;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout make_layout(int64_t m, int64_t n, int nb, int ib, size_t esz) {
  Layout L;
  L.m = m; L.n = n; L.NB = nb; L.IB = ib;
  L.MT = (int)((m + nb - 1) / nb);
  L.NT = (int)((n + nb - 1) / nb);
  L.S = std::min(auto_split(nb, esz), nb);
  L.ntasks = count_tasks(L.MT, L.NT, L.S);
  size_t off = 256;  // status words
  L.off_cnt = off;
  off = align256(off + (size_t)L.MT * L.NT * L.S * sizeof(unsigned));
  L.off_tasks = off;
  off = align256(off + (size_t)L.ntasks * sizeof(uint64_t));
  L.off_tiles = off;
  off = align256(off + (size_t)L.MT * L.NT * nb * nb * esz);
  L.bytes = off;
  L.t_elems = (int64_t)L.MT * L.NT * ib * nb;
  return L;
}

// ---------------------------------------------------------------------------
// Host: the task order. Program order first (k-major flat tree), then the
// earliest start time of every task in an unbounded-processor schedule with
// flop weights, then a stable sort on it. Dependencies always start strictly
// earlier, so the result is a topological order.
struct SchedKey {
  int MT, NT, S, order, workers;
  double wG, wU, wT, wM;
  bool operator<(const SchedKey& o) const {
    return std::tie(MT, NT, S, order, workers, wG, wU, wT, wM) <
           std::tie(o.MT, o.NT, o.S, o.order, o.workers, o.wG, o.wU, o.wT, o.wM);
  }
};

int device_sms() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  return sms;
}

// Persistent workers the list schedule plans for: two CTAs per SM of the SM
// budget (g_mu held by the caller).
int workers_locked() {
  const int sms = device_sms();
  return 2 * (g_sm_budget > 0 ? std::min(g_sm_budget, sms) : sms);
}
struct Sched {
  uint64_t* host = nullptr;  // pinned
  int64_t n = 0;
};
std::map<SchedKey, Sched> g_sched;

// List-schedule weights of the four task types for a configuration: the
// measured costs when installed, else flop counts (units of NB^3) with the
// panel tasks weighted up by QR_OPT_PANEL_WEIGHT and UNMQR by
// QR_OPT_UNMQR_WEIGHT (their level-2 and triangular parts run below the
// update's rate).
std::array<double, 4> task_weights(int prec, int nb, int ib, int S) {
  auto it = g_costs.find(std::make_tuple(prec, nb, ib));
  if (it != g_costs.end()) return it->second;
  const double ap = g_wpanel / 100.0, au = g_wunmqr / 100.0;
  return {4.0 / 3.0 * ap, 2.0 * au / S, 2.0 * ap, 4.0 / S};
}

const Sched& get_schedule(int MT, int NT, int S, const std::array<double, 4>& w) {
  SchedKey key{MT, NT, S, g_order, workers_locked(), w[0], w[1], w[2], w[3]};
  auto it = g_sched.find(key);
  if (it != g_sched.end()) return it->second;
  const int K = std::min(MT, NT);
  std::vector<uint64_t> code;
  std::vector<double> est;
  code.reserve(count_tasks(MT, NT, S));
  est.reserve(code.capacity());
  std::vector<double> fin((size_t)MT * NT * S, 0.0);
  auto F = [&](int i, int j, int s) -> double& { return fin[((size_t)j * MT + i) * S + s]; };
  // direct predecessors (last writers of the touched tile chunks) for the
  // list-scheduled order
  std::vector<int32_t> lastw((size_t)MT * NT * S, -1);
  auto LW = [&](int i, int j, int s) -> int32_t& { return lastw[((size_t)j * MT + i) * S + s]; };
  std::vector<int64_t> poff(1, 0);
  std::vector<int32_t> pred;
  std::vector<double> wt;
  std::vector<int32_t> cur;
  auto dep = [&](int i, int j, int s) {
    const int32_t p = LW(i, j, s);
    if (p >= 0 && std::find(cur.begin(), cur.end(), p) == cur.end()) cur.push_back(p);
  };
  auto close = [&](double w) {
    for (int32_t p : cur) pred.push_back(p);
    poff.push_back((int64_t)pred.size());
    wt.push_back(w);
    cur.clear();
  };
  const double wG = w[0], wU = w[1], wT = w[2], wM = w[3];
  for (int k = 0; k < K; ++k) {
    {
      double st = 0;
      for (int s = 0; s < S; ++s) {
        st = std::max(st, F(k, k, s));
        dep(k, k, s);
      }
      close(wG);
      for (int s = 0; s < S; ++s) {
        F(k, k, s) = st + wG;
        LW(k, k, s) = (int32_t)code.size();
      }
      code.push_back(encode_task(TASK_GEQRT, 0, k, k, k));
      est.push_back(st);
    }
    const double fin_geqrt = F(k, k, 0);
    const int32_t geqrt_id = (int32_t)code.size() - 1;
    for (int j = k + 1; j < NT; ++j)
      for (int s = 0; s < S; ++s) {
        double st = std::max(fin_geqrt, F(k, j, s));
        cur.push_back(geqrt_id);
        dep(k, j, s);
        close(wU);
        F(k, j, s) = st + wU;
        LW(k, j, s) = (int32_t)code.size();
        code.push_back(encode_task(TASK_UNMQR, s, k, j, k));
        est.push_back(st);
      }
    for (int i = k + 1; i < MT; ++i) {
      double st = 0;
      for (int s = 0; s < S; ++s) {
        st = std::max(st, std::max(F(k, k, s), F(i, k, s)));
        dep(k, k, s);
        dep(i, k, s);
      }
      close(wT);
      const int32_t ts_id = (int32_t)code.size();
      for (int s = 0; s < S; ++s) {
        F(k, k, s) = F(i, k, s) = st + wT;
        LW(k, k, s) = LW(i, k, s) = ts_id;
      }
      code.push_back(encode_task(TASK_TSQRT, 0, i, k, k));
      est.push_back(st);
      const double fin_v = st + wT;
      for (int j = k + 1; j < NT; ++j)
        for (int s = 0; s < S; ++s) {
          double st2 = std::max(fin_v, std::max(F(k, j, s), F(i, j, s)));
          cur.push_back(ts_id);
          dep(k, j, s);
          dep(i, j, s);
          close(wM);
          F(k, j, s) = F(i, j, s) = st2 + wM;
          LW(k, j, s) = LW(i, j, s) = (int32_t)code.size();
          code.push_back(encode_task(TASK_TSMQR, s, i, j, k));
          est.push_back(st2);
        }
    }
  }
  std::vector<int64_t> idx;
  if (g_order == 1) {
    idx = list_schedule(wt, poff, pred, workers_locked());
  } else {
    idx.resize(code.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return est[a] < est[b]; });
  }
  Sched sc;
  sc.n = (int64_t)code.size();
  if (cudaHostAlloc((void**)&sc.host, sizeof(uint64_t) * std::max<int64_t>(sc.n, 1), cudaHostAllocDefault) !=
      cudaSuccess) {
    cudaGetLastError();
    sc.host = (uint64_t*)malloc(sizeof(uint64_t) * std::max<int64_t>(sc.n, 1));
  }
  for (int64_t t = 0; t < sc.n; ++t) sc.host[t] = code[idx[t]];
  return g_sched.emplace(key, sc).first->second;
}

// ---------------------------------------------------------------------------
// Device: the persistent scheduler.
template <typename S>
struct FactorArgs {
  S* W;
  S* T;
  int64_t m, n;
  int NB, IB, MT, NT, S_;
  const uint64_t* tasks;
  int64_t ntasks;
  unsigned* cnt;
  DevCtl* ctl;
  uint64_t timeout_ns;
  TraceRec* trace;
  int64_t trace_cap;
  int tc;  // TC_* precision of the UNMQR/TSMQR products (FP32 tiles)
};

template <typename S>
__global__ void __launch_bounds__(NTHREADS, 2) persistent_qr(FactorArgs<S> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem<S> sm = carve<S>(reinterpret_cast<S*>(smem_raw));
  __shared__ int64_t s_ticket;
  __shared__ int s_ok;
  const int NB = a.NB, MT = a.MT, Sp = a.S_;
  const size_t tile_elems = (size_t)NB * NB;
  auto tile = [&](int i, int j) { return a.W + ((size_t)j * MT + i) * tile_elems; };
  auto tfac = [&](int i, int k) { return a.T + ((size_t)k * MT + i) * (size_t)a.IB * NB; };
  auto ctr = [&](int i, int j, int s) { return a.cnt + ((size_t)j * MT + i) * Sp + s; };
  auto rows_of = [&](int i) { return (int)min((int64_t)NB, a.m - (int64_t)i * NB); };
  auto cols_of = [&](int j) { return (int)min((int64_t)NB, a.n - (int64_t)j * NB); };
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
    uint64_t t_take = 0, t_ready = 0;
    if (threadIdx.x == 0) {
      if (a.trace) t_take = globaltimer();
      bool ok = true;
      const uint64_t to = a.timeout_ns;
      switch (type) {
        case TASK_GEQRT: ok = wait_ge(ctr(k, k, 0), Sp, (unsigned)k, a.ctl, to); break;
        case TASK_UNMQR:
          ok = wait_ge(ctr(k, k, 0), 1, (unsigned)k + 1, a.ctl, to) &&
               wait_ge(ctr(k, j, sch), 1, (unsigned)k, a.ctl, to);
          break;
        case TASK_TSQRT:
          ok = wait_ge(ctr(k, k, 0), Sp, (unsigned)i, a.ctl, to) &&
               wait_ge(ctr(i, k, 0), Sp, (unsigned)k, a.ctl, to);
          break;
        default:
          ok = wait_ge(ctr(i, k, 0), 1, (unsigned)k + 1, a.ctl, to) &&
               wait_ge(ctr(k, j, sch), 1, (unsigned)i, a.ctl, to) &&
               wait_ge(ctr(i, j, sch), 1, (unsigned)k, a.ctl, to);
          break;
      }
      s_ok = ok;
      if (a.trace) t_ready = globaltimer();
    }
    __syncthreads();
    if (!s_ok) break;
    const int rk = rows_of(k), ck = cols_of(k);
    switch (type) {
      case TASK_GEQRT:
        geqrt<S>(tile(k, k), NB, rk, ck, a.IB, tfac(k, k), sm, &a.ctl->status);
        break;
      case TASK_UNMQR: {
        const int cj = cols_of(j);
        const int c0 = (int)((int64_t)sch * cj / Sp), c1 = (int)((int64_t)(sch + 1) * cj / Sp);
        unmqr<S>(tile(k, k), NB, tfac(k, k), a.IB, rk, ck, tile(k, j), NB, c0, c1, sm, a.tc);
        break;
      }
      case TASK_TSQRT:
        tsqrt<S>(tile(k, k), NB, tile(i, k), NB, rows_of(i), ck, a.IB, tfac(i, k), sm, &a.ctl->status);
        break;
      default: {
        const int cj = cols_of(j);
        const int c0 = (int)((int64_t)sch * cj / Sp), c1 = (int)((int64_t)(sch + 1) * cj / Sp);
        tsmqr<S>(tile(i, k), NB, tfac(i, k), a.IB, rows_of(i), ck, tile(k, j), NB, tile(i, j), NB, c0, c1, sm,
                 false, a.tc);
        break;
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      switch (type) {
        case TASK_GEQRT:
          for (int s = 0; s < Sp; ++s) red_release_add(ctr(k, k, s), 1u);
          break;
        case TASK_UNMQR: red_release_add(ctr(k, j, sch), 1u); break;
        case TASK_TSQRT:
          for (int s = 0; s < Sp; ++s) {
            red_release_add(ctr(k, k, s), 1u);
            red_release_add(ctr(i, k, s), 1u);
          }
          break;
        default:
          red_release_add(ctr(k, j, sch), 1u);
          red_release_add(ctr(i, j, sch), 1u);
          break;
      }
      trace_put(a.trace, a.trace_cap, t, type, t_take, t_ready);
    }
  }
}

template <typename S>
int persistent_grid(int* grid_out, size_t smem) {
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  e = cudaFuncSetAttribute(persistent_qr<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_qr<S>, NTHREADS, smem);
  if (e != cudaSuccess) return (int)e;
  if (occ < 1) return (int)cudaErrorInvalidConfiguration;
  int per = occ;
  if (g_ctas_per_sm > 0) per = std::min(per, g_ctas_per_sm);
  int grid = sms * per;
  if (g_sm_budget > 0) grid = std::min(grid, std::min(g_sm_budget, sms) * per);
  if (g_grid_limit > 0) grid = std::min(grid, g_grid_limit);
  *grid_out = grid;
  return 0;
}

template <typename S>
int factor_impl(int64_t m, int64_t n, S* A, int64_t lda, int nb, int ib, S* T, void* scratch,
                int64_t scratch_bytes, void* stream, int tc = TC_NONE) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (!A && m * n > 0) return -3;
  if (lda < std::max<int64_t>(m, 1)) return -4;
  if (nb == 0) {
    if (qr_table_lookup(m, n, (int)sizeof(S), &nb, &ib) != 0) return -5;
  }
  if (nb < 8 || nb > 512) return -5;
  if (ib < 1 || ib > nb || ib > 256) return -6;
  if (m == 0 || n == 0) return 0;
  if (!T) return -7;
  if (!scratch) return -8;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_mu);
  const Layout L = make_layout(m, n, nb, ib, sizeof(S));
  if (scratch_bytes < (int64_t)L.bytes) return -9;
  if (L.MT > 65535 || L.NT > 65535) return -1;
  const Sched& sc = get_schedule(L.MT, L.NT, L.S, task_weights(sizeof(S) == 8 ? QR_PREC_F64 : QR_PREC_F32, nb, ib, L.S));
  char* base = (char*)scratch;
  DevCtl* ctl = (DevCtl*)base;
  unsigned* cnt = (unsigned*)(base + L.off_cnt);
  uint64_t* dtasks = (uint64_t*)(base + L.off_tasks);
  S* W = (S*)(base + L.off_tiles);
  int64_t ntasks = sc.n;
  cudaError_t e;
  if (g_drop_task >= 0 && g_drop_task < sc.n) {
    // test hook: a task list with one task missing (host-made fault)
    if (g_drop_task > 0)
      e = cudaMemcpyAsync(dtasks, sc.host, sizeof(uint64_t) * g_drop_task, cudaMemcpyHostToDevice, st);
    else
      e = cudaSuccess;
    if (e == cudaSuccess && g_drop_task + 1 < sc.n)
      e = cudaMemcpyAsync(dtasks + g_drop_task, sc.host + g_drop_task + 1,
                          sizeof(uint64_t) * (sc.n - g_drop_task - 1), cudaMemcpyHostToDevice, st);
    ntasks = sc.n - 1;
  } else {
    e = cudaMemcpyAsync(dtasks, sc.host, sizeof(uint64_t) * sc.n, cudaMemcpyHostToDevice, st);
  }
  if (e != cudaSuccess) return (int)e;
  const int64_t nzero = (int64_t)(L.off_cnt / sizeof(unsigned)) + (int64_t)L.MT * L.NT * L.S;
  cm_to_tiles<S><<<1184, 256, 0, st>>>(A, lda, m, n, W, nb, L.MT, L.NT, (unsigned*)base, nzero);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  // the staged tensor-core updates take more shared memory (two CTAs per SM still fit)
  const size_t smem = (sizeof(S) == 4 && tc != TC_NONE) ? std::max<size_t>(smem_elems<S>() * sizeof(S), TC_SMEM_BYTES)
                                                       : smem_elems<S>() * sizeof(S);
  int grid = 0;
  int rc = persistent_grid<S>(&grid, smem);
  if (rc) return rc;
  FactorArgs<S> fa;
  fa.W = W; fa.T = T; fa.m = m; fa.n = n; fa.NB = nb; fa.IB = ib; fa.MT = L.MT; fa.NT = L.NT; fa.S_ = L.S;
  fa.tasks = dtasks; fa.ntasks = ntasks; fa.cnt = cnt; fa.ctl = ctl;
  fa.timeout_ns = (uint64_t)g_wait_timeout_us * 1000ull;
  fa.trace = (TraceRec*)g_trace.load(); fa.trace_cap = g_trace_cap.load();
  fa.tc = tc;
  if (g_record) {
    if (!g_ev[0]) {
      if ((e = cudaEventCreate(&g_ev[0])) != cudaSuccess) return (int)e;
      if ((e = cudaEventCreate(&g_ev[1])) != cudaSuccess) return (int)e;
    }
    cudaEventRecord(g_ev[0], st);
  }
  persistent_qr<S><<<grid, NTHREADS, smem, st>>>(fa);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  if (g_record) {
    cudaEventRecord(g_ev[1], st);
    g_ev_pending = true;
  }
  tiles_to_cm<S><<<1184, 256, 0, st>>>(W, A, lda, m, n, nb, L.MT);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  return 0;
}

// ---------------------------------------------------------------------------
// Allocation-free variant (qr_factor_d_noalloc). Its scratch -- status word,
// ticket, progress counters, task list and tile-layout copy of A -- lives in
// this fixed device array instead of a caller buffer. Host code must not pass
// the symbol itself to a kernel (on the host it names a stand-in, not device
// memory); the device address comes from cudaGetSymbolAddress, once per
// device, on the first call made with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[QR_NOALLOC_SCRATCH_BYTES];

// The array's device address belongs to one CUDA context. It is looked up
// once per context and cached under the context's unique id (cuCtxGetId,
// reached through the runtime's driver entry points, so the library does not
// link libcuda): a context created anew on the same device, for instance
// after cudaDeviceReset, gets a fresh lookup instead of a stale address.
struct NoallocSlot {
  unsigned long long ctx_id;
  void* ptr;
};
constexpr int kNoallocSlots = 64;
NoallocSlot g_noalloc_slot[kNoallocSlots] = {};
int g_noalloc_next = 0;

typedef CUresult(CUDAAPI* CtxGetCurrentFn)(CUcontext*);
typedef CUresult(CUDAAPI* CtxGetIdFn)(CUcontext, unsigned long long*);

// Id of the context current on this thread; false if none is current (the
// runtime makes its primary context current on its first device call).
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_cur || !get_id) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f)
      return false;
    get_cur = (CtxGetCurrentFn)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f)
      return false;
    get_id = (CtxGetIdFn)f;
  }
  CUcontext ctx = nullptr;
  if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_noalloc_scratch in the current context (0 or a CUDA
// error code).
int noalloc_scratch_address(void** out) {
  unsigned long long id = 0;
  if (current_context_id(&id)) {
    for (int i = 0; i < kNoallocSlots; ++i)
      if (g_noalloc_slot[i].ptr && g_noalloc_slot[i].ctx_id == id) {
        *out = g_noalloc_slot[i].ptr;
        return 0;
      }
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return (int)e;
  // the lookup has made the runtime's context current if none was
  if (current_context_id(&id)) {
    g_noalloc_slot[g_noalloc_next] = NoallocSlot{id, p};
    g_noalloc_next = (g_noalloc_next + 1) % kNoallocSlots;
  }
  *out = p;
  return 0;
}

// Program (k-major) order of the flat-tree DAG, written by the device: one
// thread per elimination step, each computing its own offset.
__global__ void gen_program_order(int MT, int NT, int S, uint64_t* tasks) {
  const int K = min(MT, NT);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  int64_t off = 0;
  for (int kk = 0; kk < k; ++kk)
    off += 1 + (int64_t)(NT - kk - 1) * S + (int64_t)(MT - kk - 1) * (1 + (int64_t)(NT - kk - 1) * S);
  tasks[off++] = encode_task(TASK_GEQRT, 0, k, k, k);
  for (int j = k + 1; j < NT; ++j)
    for (int s = 0; s < S; ++s) tasks[off++] = encode_task(TASK_UNMQR, s, k, j, k);
  for (int i = k + 1; i < MT; ++i) {
    tasks[off++] = encode_task(TASK_TSQRT, 0, i, k, k);
    for (int j = k + 1; j < NT; ++j)
      for (int s = 0; s < S; ++s) tasks[off++] = encode_task(TASK_TSMQR, s, i, j, k);
  }
}

__global__ void copy_status(const DevCtl* ctl, int* out) { *out = ctl->status; }

int factor_noalloc_impl(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* T, int* d_status,
                        void* stream) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (!A && m * n > 0) return -3;
  if (lda < std::max<int64_t>(m, 1)) return -4;
  if (nb == 0) {
    if (qr_table_lookup(m, n, 8, &nb, &ib) != 0) return -5;
  }
  if (nb < 8 || nb > 512) return -5;
  if (ib < 1 || ib > nb || ib > 256) return -6;
  if (m == 0 || n == 0) return 0;
  if (!T) return -7;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_mu);
  const Layout L = make_layout(m, n, nb, ib, sizeof(double));
  // too large for the fixed scratch (this bound also keeps MT, NT small)
  if (L.bytes > (size_t)QR_NOALLOC_SCRATCH_BYTES || L.MT > 65535 || L.NT > 65535) return QR_NOALLOC_TOO_LARGE;
  void* scratch = nullptr;
  int rc0 = noalloc_scratch_address(&scratch);
  if (rc0) return rc0;
  cudaError_t e;
  char* base = (char*)scratch;
  DevCtl* ctl = (DevCtl*)base;
  unsigned* cnt = (unsigned*)(base + L.off_cnt);
  uint64_t* dtasks = (uint64_t*)(base + L.off_tasks);
  double* W = (double*)(base + L.off_tiles);
  const int K = std::min(L.MT, L.NT);
  gen_program_order<<<(K + 127) / 128, 128, 0, st>>>(L.MT, L.NT, L.S, dtasks);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  // the status word, ticket and every progress counter start at zero
  const int64_t nzero = (int64_t)(L.off_cnt / sizeof(unsigned)) + (int64_t)L.MT * L.NT * L.S;
  cm_to_tiles<double><<<1184, 256, 0, st>>>(A, lda, m, n, W, nb, L.MT, L.NT, (unsigned*)base, nzero);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  int grid = 0;
  int rc = persistent_grid<double>(&grid, smem_elems<double>() * sizeof(double));
  if (rc) return rc;
  FactorArgs<double> fa;
  fa.W = W; fa.T = T; fa.m = m; fa.n = n; fa.NB = nb; fa.IB = ib; fa.MT = L.MT; fa.NT = L.NT; fa.S_ = L.S;
  fa.tasks = dtasks; fa.ntasks = L.ntasks; fa.cnt = cnt; fa.ctl = ctl;
  fa.timeout_ns = (uint64_t)g_wait_timeout_us * 1000ull;
  fa.trace = (TraceRec*)g_trace.load(); fa.trace_cap = g_trace_cap.load();
  fa.tc = TC_NONE;
  persistent_qr<double><<<grid, NTHREADS, smem_elems<double>() * sizeof(double), st>>>(fa);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  tiles_to_cm<double><<<1184, 256, 0, st>>>(W, A, lda, m, n, nb, L.MT);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  if (d_status) {
    copy_status<<<1, 1, 0, st>>>(ctl, d_status);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  }
  return 0;
}

}  // namespace

int qr_prepare_schedule(int64_t m, int64_t n, int nb, int ib, int prec) {
  if (m < 1 || n < 1 || n > m || nb < 8 || nb > 512) return -1;
  std::lock_guard<std::mutex> lock(g_mu);
  const Layout L = make_layout(m, n, nb, ib, prec == QR_PREC_F32 ? 4 : 8);
  if (L.MT > 65535 || L.NT > 65535) return -1;
  get_schedule(L.MT, L.NT, L.S, task_weights(prec, nb, ib, L.S));
  return 0;
}

// ---------------------------------------------------------------------------
std::array<double, 4> qr_task_weights(int prec, int nb, int ib, int S) {
  std::lock_guard<std::mutex> lock(g_mu);
  return task_weights(prec, nb, ib, S);
}

void qr_trace_target(void** buf, int64_t* cap) {
  *buf = g_trace.load();
  *cap = g_trace_cap.load();
}

extern "C" {

int qr_workspace(int64_t m, int64_t n, int nb, int ib, int prec, int64_t* t_elems, int64_t* scratch_bytes) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (nb == 0) {
    if (qr_table_lookup(m, n, prec == QR_PREC_F32 ? 4 : 8, &nb, &ib) != 0) return -3;
  }
  if (nb < 8 || nb > 512) return -3;
  if (ib < 1 || ib > nb || ib > 256) return -4;
  if (prec != QR_PREC_F64 && prec != QR_PREC_F32) return -5;
  std::lock_guard<std::mutex> lock(g_mu);
  const Layout L = make_layout(std::max<int64_t>(m, 1), std::max<int64_t>(n, 1), nb, ib,
                               prec == QR_PREC_F64 ? 8 : 4);
  if (t_elems) *t_elems = L.t_elems;
  if (scratch_bytes) *scratch_bytes = (int64_t)L.bytes;
  return 0;
}

int64_t qr_task_count(int64_t m, int64_t n, int nb, int ib, int prec) {
  if (m <= 0 || n <= 0 || nb < 8) return 0;
  std::lock_guard<std::mutex> lock(g_mu);
  const Layout L = make_layout(m, n, nb, ib, prec == QR_PREC_F32 ? 4 : 8);
  return L.ntasks;
}

int qr_factor_d(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* T, void* scratch,
                int64_t scratch_bytes, void* stream) {
  return factor_impl<double>(m, n, A, lda, nb, ib, T, scratch, scratch_bytes, stream);
}

int qr_factor_s(int64_t m, int64_t n, float* A, int64_t lda, int nb, int ib, float* T, void* scratch,
                int64_t scratch_bytes, void* stream) {
  return factor_impl<float>(m, n, A, lda, nb, ib, T, scratch, scratch_bytes, stream);
}

static_assert(TC_NONE == 0 && TC_TF32 == 1 && TC_BF16X3 == 2, "tc_of_prec maps onto the TC_* values");

int qr_factor_mixed_s(int64_t m, int64_t n, float* A, int64_t lda, int nb, int ib, int p, int prec, float* T,
                      void* scratch, int64_t scratch_bytes, void* stream) {
  if (prec != QR_PREC_F32 && prec != QR_PREC_TF32 && prec != QR_PREC_BF16X3) return -8;
  const int tc = tc_of_prec(prec);
  if (p < 1 || p > 4096) return -7;
  if (p == 1) return factor_impl<float>(m, n, A, lda, nb, ib, T, scratch, scratch_bytes, stream, tc);
  return qr_factor_p_tc_s(m, n, A, lda, nb, ib, p, T, scratch, scratch_bytes, stream, tc);
}

int qr_factor_d_noalloc(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, double* T, int* d_status,
                        void* stream) {
  return factor_noalloc_impl(m, n, A, lda, nb, ib, T, d_status, stream);
}

int qr_status(const void* scratch, int* status, void* stream) {
  if (!scratch) return -1;
  if (!status) return -2;
  DevCtl h;
  cudaError_t e = cudaMemcpyAsync(&h, scratch, sizeof(DevCtl), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return (int)e;
  *status = h.status;
  return 0;
}

int qr_set_task_costs(int prec, int nb, int ib, const double* costs) {
  if (prec != QR_PREC_F64 && prec != QR_PREC_F32) return -1;
  if (nb < 8 || nb > 512) return -2;
  if (ib < 1 || ib > nb || ib > 256) return -3;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!costs) {
    g_costs.erase(std::make_tuple(prec, nb, ib));
    return 0;
  }
  for (int q = 0; q < 4; ++q)
    if (!(costs[q] > 0.0) || !std::isfinite(costs[q])) return -4;
  g_costs[std::make_tuple(prec, nb, ib)] = {costs[0], costs[1], costs[2], costs[3]};
  return 0;
}

int qr_set_trace(void* d_buf, int64_t capacity) {
  if (capacity < 0) return -2;
  if (d_buf && ((uintptr_t)d_buf & 31)) return -1;
  g_trace_cap.store(d_buf ? capacity : 0);
  g_trace.store(d_buf);
  return 0;
}

int qr_last_kernel_ms(float* ms) {
  if (!ms) return -1;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ev_pending) return -2;
  cudaError_t e = cudaEventSynchronize(g_ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, g_ev[0], g_ev[1]);
  return e == cudaSuccess ? 0 : (int)e;
}

int qr_set_option(int opt, int64_t value) {
  std::lock_guard<std::mutex> lock(g_mu);
  switch (opt) {
    case QR_OPT_RECORD_EVENTS:
      g_record = value ? 1 : 0;
      return 0;
    case QR_OPT_WAIT_TIMEOUT_US:
      if (value <= 0) return -2;
      g_wait_timeout_us = value;
      return 0;
    case QR_OPT_CTAS_PER_SM:
      if (value < 0) return -2;
      g_ctas_per_sm = (int)value;
      return 0;
    case QR_OPT_SPLIT:
      if (value < 0 || value > 64) return -2;
      g_split = (int)value;  // schedules are cached per split count
      return 0;
    case QR_OPT_GRID_LIMIT:
      if (value < 0) return -2;
      g_grid_limit = (int)value;
      return 0;
    case QR_OPT_DROP_TASK:
      g_drop_task = value;
      return 0;
    case QR_OPT_ORDER:
      if (value != 0 && value != 1) return -2;
      g_order = (int)value;
      return 0;
    case QR_OPT_PANEL_WEIGHT:
      if (value < 10 || value > 10000) return -2;
      g_wpanel = (int)value;
      return 0;
    case QR_OPT_UNMQR_WEIGHT:
      if (value < 10 || value > 10000) return -2;
      g_wunmqr = (int)value;
      return 0;
    case QR_OPT_SM_BUDGET:
      if (value < 0 || value > 1 << 20) return -2;
      g_sm_budget = (int)value;  // schedules are cached per worker count
      return 0;
    case QR_OPT_LS_REFINE:
      if (value < 0 || value > 2) return -2;
      g_ls_refine = (int)value;
      return 0;
    case QR_OPT_GMRES_MAX:
      if (value < 1 || value > QR_GMRES_MAX_DIM) return -2;
      g_gmres_max = (int)value;
      return 0;
    case QR_OPT_GMRES_TOL_EXP:
      if (value < 1 || value > 16) return -2;
      g_gmres_tol_exp = (int)value;
      return 0;
    case QR_OPT_TUNE_IB_TOL:
      if (value < 0 || value > 500) return -2;
      g_tune_ib_tol = (int)value;
      return 0;
  }
  return -1;
}

int64_t qr_get_option(int opt) {
  std::lock_guard<std::mutex> lock(g_mu);
  switch (opt) {
    case QR_OPT_WAIT_TIMEOUT_US: return g_wait_timeout_us;
    case QR_OPT_CTAS_PER_SM: return g_ctas_per_sm;
    case QR_OPT_SPLIT: return g_split;
    case QR_OPT_GRID_LIMIT: return g_grid_limit;
    case QR_OPT_DROP_TASK: return g_drop_task;
    case QR_OPT_RECORD_EVENTS: return g_record;
    case QR_OPT_ORDER: return g_order;
    case QR_OPT_PANEL_WEIGHT: return g_wpanel;
    case QR_OPT_UNMQR_WEIGHT: return g_wunmqr;
    case QR_OPT_SM_BUDGET: return g_sm_budget;
    case QR_OPT_LS_REFINE: return g_ls_refine;
    case QR_OPT_GMRES_MAX: return g_gmres_max;
    case QR_OPT_GMRES_TOL_EXP: return g_gmres_tol_exp;
    case QR_OPT_TUNE_IB_TOL: return g_tune_ib_tol;
  }
  return INT64_MIN;
}

}  // extern "C"
