// Tile QR with p domains per panel (CAQR-style reduction tree) and the
// matching application of Q: qr_workspace_p, qr_factor_p_{d,s},
// qr_apply_workspace_p, qr_apply_qt_p_{d,s}.
//
// The paper names a third tunable for tall-skinny matrices: the number p of
// domains of the panel (Sec. 7, communication-avoiding QR). In the flat tree
// of Sec. 2.1 the panel of step k is one chain GEQRT(k) -> TSQRT(k+1) -> ...
// -> TSQRT(MT-1), MT - k tasks long. With p domains the tile rows k..MT-1 are
// cut into ranges of ceil(MT/p) rows that slide down with the panel; each
// runs its own flat tree (GEQRT on the domain's first tile, TSQRT down the
// domain, with UNMQR/TSMQR updates), and the triangles left at the domain
// heads are merged pairwise by a binary tree of triangle-on-triangle steps
// (TTQRT, with TTMQR updates). The chain shrinks to about MT/p + log2 p
// tasks. p = 1 is the flat tree.
//
// Dependencies are explicit: a host pass over the program order records,
// for every task, how many earlier writes each tile (column chunk) it touches
// must have completed; the persistent kernel waits for those counts. The
// task list is sorted by earliest start time in an unbounded-processor
// schedule (a topological order with look-ahead), as for the flat tree.
//
// Storage: a domain head's tile keeps its GEQRT reflectors below the
// diagonal; its triangle, once merged into another head, is replaced by the
// TTQRT reflectors (upper triangular). T factors: T1 for GEQRT/TSQRT of
// tile (i, k), T2 for the TTQRT that eliminated head tile (i, k), each
// IB x NB per tile.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <numeric>
#include <queue>
#include <tuple>
#include <vector>

#include "layout.cuh"
#include "listsched.h"
#include "sched.cuh"
#include "tile_kernels.cuh"
#include "tileqr_internal.h"

using namespace tqr;

namespace {

enum DagType { D_GEQRT = 0, D_UNMQR = 1, D_TSQRT = 2, D_TSMQR = 3, D_TTQRT = 4, D_TTMQR = 5 };

struct __align__(16) TaskRec {
  int8_t type;
  int8_t pad0;
  uint16_t s;     // column chunk (updates)
  int32_t i;      // bottom tile row (TSQRT/TSMQR: eliminated row; TTQRT/TTMQR: eliminated head)
  int32_t h;      // top tile row (domain head / surviving head)
  int32_t j;      // updated tile column (updates)
  int32_t k;      // elimination step
  uint16_t cv;    // writes the reflector tile must have seen (updates)
  uint16_t ctop;  // writes the top tile (chunk) must have seen
  uint16_t cbot;  // writes the bottom tile (chunk) must have seen
  uint16_t pad1;
  int32_t pad2;
};
static_assert(sizeof(TaskRec) == 32, "task record is 32 bytes");

std::mutex g_tmu2;

// Domain heads of step k: the tile rows [k, MT) cut into ranges of
// B = ceil(MT / p) rows starting at the panel, so the domains slide down
// with the panel. A head of step k+1 is then the second row of a domain of
// step k, which receives its last update of step k early (the first link of
// that domain's chain) instead of waiting for the merge tree -- the steps
// pipeline as in the flat tree. Fewer than p domains remain once
// MT - k < (p - 1) B. A ragged last tile row shorter than the panel is never
// a head (a head runs GEQRT, which needs rows >= columns); it joins the
// domain before it.
std::vector<int> domain_heads(int k, int MT, int p, bool last_short) {
  const int B = std::max(1, (MT + p - 1) / p);
  std::vector<int> h;
  for (int r = k; r < MT; r += B) h.push_back(r);
  if (last_short && h.size() > 1 && h.back() == MT - 1) h.pop_back();
  return h;
}

struct Dag {
  std::vector<TaskRec> tasks;  // execution (ticket) order
};

int sched_workers() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  const int64_t budget = qr_get_option(QR_OPT_SM_BUDGET);
  return 2 * (budget > 0 ? (int)std::min<int64_t>(budget, sms) : sms);  // two persistent CTAs per SM of the budget
}

struct DagKey {
  int MT, NT, S, P, last_short, workers;
  double w0, w1, w2, w3;  // list-schedule weights (factorization DAGs)
  bool operator<(const DagKey& o) const {
    return std::tie(MT, NT, S, P, last_short, workers, w0, w1, w2, w3) <
           std::tie(o.MT, o.NT, o.S, o.P, o.last_short, o.workers, o.w0, o.w1, o.w2, o.w3);
  }
};
std::map<DagKey, Dag> g_dags;

// Factorization DAG.
// w: list-schedule costs of GEQRT, UNMQR, TSQRT, TSMQR (qr_task_weights);
// the triangle-on-triangle tasks count half of their TS counterparts.
const Dag& factor_dag(int MT, int NT, int S, int P, bool last_short, const std::array<double, 4>& w) {
  DagKey key{MT, NT, S, P, last_short ? 1 : 0, sched_workers(), w[0], w[1], w[2], w[3]};
  auto it = g_dags.find(key);
  if (it != g_dags.end()) return it->second;
  const int K = std::min(MT, NT);
  std::vector<uint16_t> wc((size_t)MT * NT * S, 0);
  std::vector<double> fin((size_t)MT * NT * S, 0.0);
  auto W = [&](int i, int j, int s) -> uint16_t& { return wc[((size_t)j * MT + i) * S + s]; };
  auto F = [&](int i, int j, int s) -> double& { return fin[((size_t)j * MT + i) * S + s]; };
  std::vector<TaskRec> prog;
  std::vector<double> est, wt;
  std::vector<int64_t> poff(1, 0);
  std::vector<int32_t> pred;
  std::vector<int32_t> lastw((size_t)MT * NT * S, -1);
  auto LW = [&](int i, int j, int s) -> int32_t& { return lastw[((size_t)j * MT + i) * S + s]; };
  // direct predecessors of the task about to be appended: the last writers
  // of the listed (tile, chunk) pairs; then the task becomes the last writer
  // of the chunks it writes
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
  auto rec = [&](int type, int s, int i, int h, int j, int k) {
    TaskRec t{};
    t.type = (int8_t)type;
    t.s = (uint16_t)s;
    t.i = i;
    t.h = h;
    t.j = j;
    t.k = k;
    return t;
  };
  const double wG = w[0], wU = w[1], wT = w[2], wM = w[3], wTT = 0.5 * w[2], wMT = 0.5 * w[3];
  auto panel1 = [&](int type, int h, int k, double w) {  // GEQRT on (h,k)
    TaskRec t = rec(type, 0, h, h, k, k);
    t.ctop = W(h, k, 0);
    double st = 0;
    for (int s = 0; s < S; ++s) {
      st = std::max(st, F(h, k, s));
      dep(h, k, s);
    }
    close(w);
    for (int s = 0; s < S; ++s) {
      ++W(h, k, s);
      F(h, k, s) = st + w;
      LW(h, k, s) = (int32_t)prog.size();
    }
    prog.push_back(t);
    est.push_back(st);
  };
  auto panel2 = [&](int type, int top, int bot, int k, double w) {  // TSQRT / TTQRT
    TaskRec t = rec(type, 0, bot, top, k, k);
    t.ctop = W(top, k, 0);
    t.cbot = W(bot, k, 0);
    double st = 0;
    for (int s = 0; s < S; ++s) {
      st = std::max(st, std::max(F(top, k, s), F(bot, k, s)));
      dep(top, k, s);
      dep(bot, k, s);
    }
    close(w);
    for (int s = 0; s < S; ++s) {
      ++W(top, k, s);
      ++W(bot, k, s);
      F(top, k, s) = F(bot, k, s) = st + w;
      LW(top, k, s) = LW(bot, k, s) = (int32_t)prog.size();
    }
    prog.push_back(t);
    est.push_back(st);
  };
  auto upd1 = [&](int h, int j, int k, int s) {  // UNMQR: V (h,k), C (h,j)
    TaskRec t = rec(D_UNMQR, s, h, h, j, k);
    t.cv = W(h, k, 0);
    t.ctop = W(h, j, s);
    const double st = std::max(F(h, k, 0), F(h, j, s));
    dep(h, k, 0);
    dep(h, j, s);
    close(wU);
    ++W(h, j, s);
    F(h, j, s) = st + wU;
    LW(h, j, s) = (int32_t)prog.size();
    prog.push_back(t);
    est.push_back(st);
  };
  auto upd2 = [&](int type, int top, int bot, int j, int k, int s, double w) {  // TSMQR / TTMQR: V (bot,k)
    TaskRec t = rec(type, s, bot, top, j, k);
    t.cv = W(bot, k, 0);
    t.ctop = W(top, j, s);
    t.cbot = W(bot, j, s);
    const double st = std::max(F(bot, k, 0), std::max(F(top, j, s), F(bot, j, s)));
    dep(bot, k, 0);
    dep(top, j, s);
    dep(bot, j, s);
    close(w);
    ++W(top, j, s);
    ++W(bot, j, s);
    F(top, j, s) = F(bot, j, s) = st + w;
    LW(top, j, s) = LW(bot, j, s) = (int32_t)prog.size();
    prog.push_back(t);
    est.push_back(st);
  };
  for (int k = 0; k < K; ++k) {
    std::vector<int> hs = domain_heads(k, MT, P, last_short);
    hs.push_back(MT);
    const int nd = (int)hs.size() - 1;
    for (int d = 0; d < nd; ++d) {
      const int h = hs[d];
      panel1(D_GEQRT, h, k, wG);
      for (int j = k + 1; j < NT; ++j)
        for (int s = 0; s < S; ++s) upd1(h, j, k, s);
      for (int i = h + 1; i < hs[d + 1]; ++i) {
        panel2(D_TSQRT, h, i, k, wT);
        for (int j = k + 1; j < NT; ++j)
          for (int s = 0; s < S; ++s) upd2(D_TSMQR, h, i, j, k, s, wM);
      }
    }
    for (int step = 1; step < nd; step *= 2)
      for (int d = 0; d + step < nd; d += 2 * step) {
        const int a = hs[d], b = hs[d + step];
        panel2(D_TTQRT, a, b, k, wTT);
        for (int j = k + 1; j < NT; ++j)
          for (int s = 0; s < S; ++s) upd2(D_TTMQR, a, b, j, k, s, wMT);
      }
  }
  const std::vector<int64_t> idx = list_schedule(wt, poff, pred, sched_workers());
  Dag dag;
  dag.tasks.resize(prog.size());
  for (size_t t = 0; t < idx.size(); ++t) dag.tasks[t] = prog[idx[t]];
  return g_dags.emplace(key, std::move(dag)).first->second;
}

// Q application DAG over C's row blocks (column chunks S). Program order is
// the factorization's update order for Q^T, reversed for Q.
const Dag& apply_dag(int MT, int NT, int S, int P, bool last_short, int tr) {
  DagKey key{MT, NT, S, -P - 1 - 1000 * tr, last_short ? 1 : 0, 0, 0.0, 0.0, 0.0, 0.0};
  auto it = g_dags.find(key);
  if (it != g_dags.end()) return it->second;
  const int K = std::min(MT, NT);
  struct Op {
    int type, top, bot, k;
  };
  std::vector<Op> ops;
  for (int k = 0; k < K; ++k) {
    std::vector<int> hs = domain_heads(k, MT, P, last_short);
    hs.push_back(MT);
    const int nd = (int)hs.size() - 1;
    for (int d = 0; d < nd; ++d) {
      ops.push_back({D_UNMQR, hs[d], hs[d], k});
      for (int i = hs[d] + 1; i < hs[d + 1]; ++i) ops.push_back({D_TSMQR, hs[d], i, k});
    }
    for (int step = 1; step < nd; step *= 2)
      for (int d = 0; d + step < nd; d += 2 * step) ops.push_back({D_TTMQR, hs[d], hs[d + step], k});
  }
  if (!tr) std::reverse(ops.begin(), ops.end());
  std::vector<uint16_t> wc((size_t)MT * S, 0);
  std::vector<double> fin((size_t)MT * S, 0.0);
  std::vector<TaskRec> prog;
  std::vector<double> est, wt;
  std::vector<int64_t> poff(1, 0);
  std::vector<int32_t> pred;
  std::vector<int32_t> lastw((size_t)MT * S, -1);
  for (const Op& o : ops)
    for (int s = 0; s < S; ++s) {
      {
        const int32_t p1 = lastw[(size_t)o.top * S + s];
        if (p1 >= 0) pred.push_back(p1);
        if (o.type != D_UNMQR) {
          const int32_t p2 = lastw[(size_t)o.bot * S + s];
          if (p2 >= 0 && p2 != p1) pred.push_back(p2);
        }
        poff.push_back((int64_t)pred.size());
        wt.push_back(o.type == D_TSMQR ? 2.0 : 1.0);
        lastw[(size_t)o.top * S + s] = (int32_t)prog.size();
        if (o.type != D_UNMQR) lastw[(size_t)o.bot * S + s] = (int32_t)prog.size();
      }
      TaskRec t{};
      t.type = (int8_t)o.type;
      t.s = (uint16_t)s;
      t.h = o.top;
      t.i = o.bot;
      t.j = -1;
      t.k = o.k;
      t.ctop = wc[(size_t)o.top * S + s];
      double st = fin[(size_t)o.top * S + s];
      if (o.type != D_UNMQR) {
        t.cbot = wc[(size_t)o.bot * S + s];
        st = std::max(st, fin[(size_t)o.bot * S + s]);
        ++wc[(size_t)o.bot * S + s];
      }
      ++wc[(size_t)o.top * S + s];
      const double w = o.type == D_TSMQR ? 2.0 : 1.0;
      fin[(size_t)o.top * S + s] = st + w;
      if (o.type != D_UNMQR) fin[(size_t)o.bot * S + s] = st + w;
      prog.push_back(t);
      est.push_back(st);
    }
  const std::vector<int64_t> idx = list_schedule(wt, poff, pred, sched_workers());
  Dag dag;
  dag.tasks.resize(prog.size());
  for (size_t t = 0; t < idx.size(); ++t) dag.tasks[t] = prog[idx[t]];
  return g_dags.emplace(key, std::move(dag)).first->second;
}

int split_for(int NB) {
  const int64_t o = qr_get_option(QR_OPT_SPLIT);
  if (o > 0) return std::min<int>((int)o, NB);
  if (NB <= 160) return 1;
  if (NB <= 320) return 2;
  return 4;
}

struct PLayout {
  int MT, NT, S, P;
  bool last_short;
  int64_t ntasks;
  size_t off_cnt, off_tasks, off_tiles, bytes;
  int64_t t_elems;
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

PLayout p_layout(int64_t m, int64_t n, int nb, int ib, int p, size_t esz, bool with_tasks) {
  PLayout L;
  L.MT = (int)((m + nb - 1) / nb);
  L.NT = (int)((n + nb - 1) / nb);
  L.S = split_for(nb);
  L.P = std::max(1, p);
  const int64_t last_rows = m - (int64_t)(L.MT - 1) * nb;
  L.last_short = last_rows < std::min<int64_t>(nb, n);
  L.ntasks = with_tasks ? (int64_t)factor_dag(L.MT, L.NT, L.S, L.P, L.last_short,
                                               qr_task_weights(esz == 8 ? QR_PREC_F64 : QR_PREC_F32, nb, ib, L.S))
                                     .tasks.size()
                        : 0;
  size_t off = 256;
  L.off_cnt = off;
  off = al256(off + (size_t)L.MT * L.NT * L.S * 4);
  L.off_tasks = off;
  off = al256(off + (size_t)L.ntasks * sizeof(TaskRec));
  L.off_tiles = off;
  off = al256(off + (size_t)L.MT * L.NT * nb * nb * esz);
  L.bytes = off;
  L.t_elems = 2 * (int64_t)L.MT * L.NT * ib * nb;  // T1 and T2
  return L;
}

template <typename S>
struct DagArgs {
  S* W;
  S* T1;
  S* T2;
  int64_t m, n;
  int NB, IB, MT, NT, S_;
  const TaskRec* tasks;
  int64_t ntasks;
  unsigned* cnt;
  DevCtl* ctl;
  uint64_t timeout_ns;
  TraceRec* trace;
  int64_t trace_cap;
  int tc;  // TC_* precision of the UNMQR/TSMQR products (FP32 tiles)
};

template <typename S>
__global__ void __launch_bounds__(NTHREADS, 2) persistent_qr_dag(DagArgs<S> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem<S> sm = carve<S>(reinterpret_cast<S*>(smem_raw));
  __shared__ int64_t s_ticket;
  __shared__ int s_ok;
  __shared__ TaskRec s_task;
  const int NB = a.NB, MT = a.MT, Sp = a.S_;
  const size_t tile_elems = (size_t)NB * NB;
  auto tile = [&](int i, int j) { return a.W + ((size_t)j * MT + i) * tile_elems; };
  auto t1 = [&](int i, int k) { return a.T1 + ((size_t)k * MT + i) * (size_t)a.IB * NB; };
  auto t2 = [&](int i, int k) { return a.T2 + ((size_t)k * MT + i) * (size_t)a.IB * NB; };
  auto ctr = [&](int i, int j, int s) { return a.cnt + ((size_t)j * MT + i) * Sp + s; };
  auto rows_of = [&](int i) { return (int)min((int64_t)NB, a.m - (int64_t)i * NB); };
  auto cols_of = [&](int j) { return (int)min((int64_t)NB, a.n - (int64_t)j * NB); };
  for (;;) {
    if (threadIdx.x == 0) {
      int64_t t = -1;
      if (!((volatile int*)&a.ctl->abort)[0]) t = (int64_t)atomicAdd(&a.ctl->ticket, 1u);
      s_ticket = t;
      if (t >= 0 && t < a.ntasks) s_task = a.tasks[t];
    }
    __syncthreads();
    const int64_t tk = s_ticket;
    if (tk < 0 || tk >= a.ntasks) break;
    const TaskRec t = s_task;
    const int type = t.type, i = t.i, h = t.h, j = t.j, k = t.k, sc = t.s;
    uint64_t t_take = 0, t_ready = 0;
    if (threadIdx.x == 0) {
      if (a.trace) t_take = globaltimer();
      bool ok = true;
      const uint64_t to = a.timeout_ns;
      switch (type) {
        case D_GEQRT: ok = wait_ge(ctr(h, k, 0), Sp, t.ctop, a.ctl, to); break;
        case D_TSQRT:
        case D_TTQRT:
          ok = wait_ge(ctr(h, k, 0), Sp, t.ctop, a.ctl, to) && wait_ge(ctr(i, k, 0), Sp, t.cbot, a.ctl, to);
          break;
        case D_UNMQR:
          ok = wait_ge(ctr(h, k, 0), 1, t.cv, a.ctl, to) && wait_ge(ctr(h, j, sc), 1, t.ctop, a.ctl, to);
          break;
        default:  // TSMQR / TTMQR
          ok = wait_ge(ctr(i, k, 0), 1, t.cv, a.ctl, to) && wait_ge(ctr(h, j, sc), 1, t.ctop, a.ctl, to) &&
               wait_ge(ctr(i, j, sc), 1, t.cbot, a.ctl, to);
          break;
      }
      s_ok = ok;
      if (a.trace) t_ready = globaltimer();
    }
    __syncthreads();
    if (!s_ok) break;
    const int ck = cols_of(k);
    int c0 = 0, c1 = 0;
    if (type == D_UNMQR || type == D_TSMQR || type == D_TTMQR) {
      const int cj = cols_of(j);
      c0 = (int)((int64_t)sc * cj / Sp);
      c1 = (int)((int64_t)(sc + 1) * cj / Sp);
    }
    switch (type) {
      case D_GEQRT: geqrt<S>(tile(h, k), NB, rows_of(h), ck, a.IB, t1(h, k), sm, &a.ctl->status); break;
      case D_UNMQR:
        unmqr<S>(tile(h, k), NB, t1(h, k), a.IB, rows_of(h), ck, tile(h, j), NB, c0, c1, sm, a.tc);
        break;
      case D_TSQRT:
        tsqrt<S>(tile(h, k), NB, tile(i, k), NB, rows_of(i), ck, a.IB, t1(i, k), sm, &a.ctl->status, false);
        break;
      case D_TSMQR:
        tsmqr<S>(tile(i, k), NB, t1(i, k), a.IB, rows_of(i), ck, tile(h, j), NB, tile(i, j), NB, c0, c1, sm, false,
                 a.tc);
        break;
      case D_TTQRT:
        tsqrt<S>(tile(h, k), NB, tile(i, k), NB, rows_of(i), ck, a.IB, t2(i, k), sm, &a.ctl->status, true);
        break;
      default:  // D_TTMQR
        tsmqr<S>(tile(i, k), NB, t2(i, k), a.IB, rows_of(i), ck, tile(h, j), NB, tile(i, j), NB, c0, c1, sm, true);
        break;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      switch (type) {
        case D_GEQRT:
          for (int s = 0; s < Sp; ++s) red_release_add(ctr(h, k, s), 1u);
          break;
        case D_TSQRT:
        case D_TTQRT:
          for (int s = 0; s < Sp; ++s) {
            red_release_add(ctr(h, k, s), 1u);
            red_release_add(ctr(i, k, s), 1u);
          }
          break;
        case D_UNMQR: red_release_add(ctr(h, j, sc), 1u); break;
        default:
          red_release_add(ctr(h, j, sc), 1u);
          red_release_add(ctr(i, j, sc), 1u);
          break;
      }
      trace_put(a.trace, a.trace_cap, tk, type, t_take, t_ready);
    }
  }
}

template <typename S>
int factor_p_impl(int64_t m, int64_t n, S* A, int64_t lda, int nb, int ib, int p, S* T, void* scratch,
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
  if (p < 1 || p > 4096) return -7;
  if (m == 0 || n == 0) return 0;
  if (!T) return -8;
  if (!scratch) return -9;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_tmu2);
  if ((m + nb - 1) / nb > 65535) return -1;
  const PLayout L = p_layout(m, n, nb, ib, p, sizeof(S), true);
  if (scratch_bytes < (int64_t)L.bytes) return -10;
  const Dag& dag = factor_dag(L.MT, L.NT, L.S, L.P, L.last_short,
                             qr_task_weights(sizeof(S) == 8 ? QR_PREC_F64 : QR_PREC_F32, nb, ib, L.S));
  char* base = (char*)scratch;
  cudaError_t e = cudaMemcpyAsync(base + L.off_tasks, dag.tasks.data(), dag.tasks.size() * sizeof(TaskRec),
                                  cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return (int)e;  // cached DAGs are never freed: the host copy outlives the copy
  S* W = (S*)(base + L.off_tiles);
  const int64_t nzero = (int64_t)(L.off_cnt / 4) + (int64_t)L.MT * L.NT * L.S;
  cm_to_tiles<S><<<1184, 256, 0, st>>>(A, lda, m, n, W, nb, L.MT, L.NT, (unsigned*)base, nzero);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the staged tensor-core updates take more shared memory (two CTAs per SM still fit)
  const size_t smem = (sizeof(S) == 4 && tc != TC_NONE) ? std::max<size_t>(smem_elems<S>() * sizeof(S), TC_SMEM_BYTES)
                                                       : smem_elems<S>() * sizeof(S);
  e = cudaFuncSetAttribute(persistent_qr_dag<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_qr_dag<S>, NTHREADS, smem);
  if (e != cudaSuccess) return (int)e;
  if (occ < 1) return (int)cudaErrorInvalidConfiguration;
  int per = occ;
  const int64_t cps = qr_get_option(QR_OPT_CTAS_PER_SM);
  if (cps > 0) per = std::min<int>(per, (int)cps);
  int grid = sms * per;
  const int64_t budget = qr_get_option(QR_OPT_SM_BUDGET);
  if (budget > 0) grid = std::min<int64_t>(grid, std::min<int64_t>(budget, sms) * per);
  const int64_t gl = qr_get_option(QR_OPT_GRID_LIMIT);
  if (gl > 0) grid = std::min<int>(grid, (int)gl);
  DagArgs<S> da;
  da.W = W; da.T1 = T; da.T2 = T + (size_t)L.MT * L.NT * ib * nb; da.m = m; da.n = n; da.NB = nb; da.IB = ib;
  da.MT = L.MT; da.NT = L.NT; da.S_ = L.S; da.tasks = (const TaskRec*)(base + L.off_tasks);
  da.ntasks = (int64_t)dag.tasks.size(); da.cnt = (unsigned*)(base + L.off_cnt); da.ctl = (DevCtl*)base;
  da.timeout_ns = (uint64_t)qr_get_option(QR_OPT_WAIT_TIMEOUT_US) * 1000ull;
  {
    void* tb = nullptr;
    int64_t tcap = 0;
    qr_trace_target(&tb, &tcap);
    da.trace = (TraceRec*)tb;
    da.trace_cap = tcap;
  }
  da.tc = sizeof(S) == 4 ? tc : TC_NONE;
  persistent_qr_dag<S><<<grid, NTHREADS, smem, st>>>(da);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  tiles_to_cm<S><<<1184, 256, 0, st>>>(W, A, lda, m, n, nb, L.MT);
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  return 0;
}

// ---------------------------------------------------------------------------
// Q application over C's row blocks with explicit dependencies.
template <typename S>
struct ApplyDagArgs {
  const S* A;
  int64_t lda;
  const S* T1;
  const S* T2;
  int64_t m, n;
  int NB, IB, MT, NT, S_;
  S* C;
  int64_t ldc, nrhs;
  const TaskRec* tasks;
  int64_t ntasks;
  unsigned* cnt;
  DevCtl* ctl;
  uint64_t timeout_ns;
  TraceRec* trace;
  int64_t trace_cap;
};

__global__ void zero_u32(unsigned* p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0u;
}

template <typename S, bool TR>
__global__ void __launch_bounds__(NTHREADS, 2) persistent_apply_dag(ApplyDagArgs<S> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem<S> sm = carve<S>(reinterpret_cast<S*>(smem_raw));
  __shared__ int64_t s_ticket;
  __shared__ int s_ok;
  __shared__ TaskRec s_task;
  const int NB = a.NB, MT = a.MT, Sp = a.S_;
  auto tileA = [&](int i, int j) { return a.A + (size_t)i * NB + (size_t)j * NB * a.lda; };
  auto t1 = [&](int i, int k) { return a.T1 + ((size_t)k * MT + i) * (size_t)a.IB * NB; };
  auto t2 = [&](int i, int k) { return a.T2 + ((size_t)k * MT + i) * (size_t)a.IB * NB; };
  auto rows_of = [&](int i) { return (int)min((int64_t)NB, a.m - (int64_t)i * NB); };
  auto cols_of = [&](int j) { return (int)min((int64_t)NB, a.n - (int64_t)j * NB); };
  auto ctr = [&](int r, int s) { return a.cnt + (size_t)r * Sp + s; };
  for (;;) {
    if (threadIdx.x == 0) {
      int64_t t = -1;
      if (!((volatile int*)&a.ctl->abort)[0]) t = (int64_t)atomicAdd(&a.ctl->ticket, 1u);
      s_ticket = t;
      if (t >= 0 && t < a.ntasks) s_task = a.tasks[t];
    }
    __syncthreads();
    const int64_t tk = s_ticket;
    if (tk < 0 || tk >= a.ntasks) break;
    const TaskRec t = s_task;
    const int type = t.type, i = t.i, h = t.h, k = t.k, sc = t.s;
    uint64_t t_take = 0, t_ready = 0;
    if (threadIdx.x == 0 && a.trace) t_take = globaltimer();
    const int c0 = (int)((int64_t)sc * a.nrhs / Sp), c1 = (int)((int64_t)(sc + 1) * a.nrhs / Sp);
    const int ck = cols_of(k);
    S* Ch = a.C + (size_t)h * NB;
    // few right-hand sides: stage the whole task in shared memory once; the
    // reflectors and T are final (written by the factorization), so they are
    // staged before the wait for the task's rows of C
    const int rw = type == D_UNMQR ? rows_of(h) : (type == D_TSMQR ? rows_of(i) : min(rows_of(i), ck));
    const bool nar = narrow_fits(rw, ck, a.IB, c1 - c0);
    const S* tf = type == D_UNMQR ? t1(h, k) : (type == D_TSMQR ? t1(i, k) : t2(i, k));
    if (nar) {
      if (type == D_UNMQR)
        narrow_stage_vt<S, false>(tileA(h, k), (int)a.lda, tf, a.IB, ck, a.IB, rw, sm);
      else
        narrow_stage_vt<S, true>(tileA(i, k), (int)a.lda, tf, a.IB, ck, a.IB, rw, sm, type == D_TTMQR);
    }
    if (threadIdx.x == 0) {
      bool ok = wait_ge(ctr(h, sc), 1, t.ctop, a.ctl, a.timeout_ns);
      if (ok && type != D_UNMQR) ok = wait_ge(ctr(i, sc), 1, t.cbot, a.ctl, a.timeout_ns);
      s_ok = ok;
      if (a.trace) t_ready = globaltimer();
    }
    __syncthreads();
    if (!s_ok) break;
    if (type == D_UNMQR) {
      if (nar)
        apply_narrow<S, false, TR>(tileA(h, k), (int)a.lda, t1(h, k), a.IB, ck, a.IB, nullptr, 0, Ch, (int)a.ldc, rw,
                                   c0, c1, sm, false, true);
      else
        apply_qt<S, false, TR>(tileA(h, k), (int)a.lda, t1(h, k), a.IB, false, 0, ck, a.IB, nullptr, 0, Ch,
                               (int)a.ldc, rw, c0, c1, sm);
    } else {
      const bool tri = type == D_TTMQR;
      if (nar)
        apply_narrow<S, true, TR>(tileA(i, k), (int)a.lda, tf, a.IB, ck, a.IB, Ch, (int)a.ldc, a.C + (size_t)i * NB,
                                  (int)a.ldc, rw, c0, c1, sm, tri, true);
      else
        apply_qt<S, true, TR>(tileA(i, k), (int)a.lda, tf, a.IB, false, 0, ck, a.IB, Ch, (int)a.ldc,
                              a.C + (size_t)i * NB, (int)a.ldc, rw, c0, c1, sm, tri);
    }
    // publish: the barrier orders every thread's C writes before thread
    // 0's fence and release (cumulative), one fence per task
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      red_release_add(ctr(h, sc), 1u);
      if (type != D_UNMQR) red_release_add(ctr(i, sc), 1u);
      trace_put(a.trace, a.trace_cap, tk, type, t_take, t_ready);
    }
  }
}

template <typename S, bool TR>
int launch_apply_dag(const ApplyDagArgs<S>& aa, cudaStream_t st) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = smem_elems<S>() * sizeof(S);
  cudaError_t e =
      cudaFuncSetAttribute(persistent_apply_dag<S, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_apply_dag<S, TR>, NTHREADS, smem);
  if (e != cudaSuccess) return (int)e;
  if (occ < 1) return (int)cudaErrorInvalidConfiguration;
  const int64_t grid = std::min<int64_t>((int64_t)sms * occ, aa.ntasks);
  persistent_apply_dag<S, TR><<<(unsigned)grid, NTHREADS, smem, st>>>(aa);
  e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

int apply_split_p(int64_t nrhs) { return (int)std::max<int64_t>(1, (nrhs + 63) / 64); }

struct APLayout {
  int MT, NT, S;
  bool last_short;
  size_t off_cnt, off_tasks, bytes;
};

APLayout ap_layout(int64_t m, int64_t n, int64_t nrhs, int nb, int p, int64_t ntasks) {
  APLayout L;
  L.MT = (int)((m + nb - 1) / nb);
  L.NT = (int)((n + nb - 1) / nb);
  L.S = apply_split_p(nrhs);
  L.last_short = (m - (int64_t)(L.MT - 1) * nb) < std::min<int64_t>(nb, n);
  L.off_cnt = 256;
  L.off_tasks = al256(L.off_cnt + (size_t)L.MT * L.S * 4);
  L.bytes = al256(L.off_tasks + (size_t)ntasks * sizeof(TaskRec));
  (void)p;
  return L;
}

template <typename S>
int apply_p_impl(int64_t m, int64_t n, int64_t nrhs, const S* A, int64_t lda, int nb, int ib, int p, const S* T,
                 S* C, int64_t ldc, int trans, void* scratch, int64_t scratch_bytes, void* stream) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (nrhs < 0) return -3;
  if (lda < std::max<int64_t>(m, 1)) return -5;
  if (nb == 0) {
    if (qr_table_lookup(m, n, (int)sizeof(S), &nb, &ib) != 0) return -6;
  }
  if (nb < 8 || nb > 512) return -6;
  if (ib < 1 || ib > nb || ib > 256) return -7;
  if (p < 1 || p > 4096) return -8;
  if (ldc < std::max<int64_t>(m, 1)) return -11;
  if (trans != 0 && trans != 1) return -12;
  if (m == 0 || n == 0 || nrhs == 0) return 0;
  if (!A) return -4;
  if (!T) return -9;
  if (!C) return -10;
  if (!scratch) return -13;
  if (lda > INT32_MAX || ldc > INT32_MAX) return -5;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_tmu2);
  APLayout L0 = ap_layout(m, n, nrhs, nb, p, 0);
  const Dag& dag = apply_dag(L0.MT, L0.NT, L0.S, p, L0.last_short, trans);
  const APLayout L = ap_layout(m, n, nrhs, nb, p, (int64_t)dag.tasks.size());
  if (scratch_bytes < (int64_t)L.bytes) return -14;
  char* base = (char*)scratch;
  cudaError_t e = cudaMemcpyAsync(base + L.off_tasks, dag.tasks.data(), dag.tasks.size() * sizeof(TaskRec),
                                  cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return (int)e;
  zero_u32<<<64, 256, 0, st>>>((unsigned*)base, (int64_t)(L.off_tasks / 4));
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  ApplyDagArgs<S> aa;
  aa.A = A; aa.lda = lda; aa.T1 = T; aa.T2 = T + (size_t)L.MT * L.NT * ib * nb; aa.m = m; aa.n = n; aa.NB = nb;
  aa.IB = ib; aa.MT = L.MT; aa.NT = L.NT; aa.S_ = L.S; aa.C = C; aa.ldc = ldc; aa.nrhs = nrhs;
  aa.tasks = (const TaskRec*)(base + L.off_tasks); aa.ntasks = (int64_t)dag.tasks.size();
  aa.cnt = (unsigned*)(base + L.off_cnt); aa.ctl = (DevCtl*)base;
  aa.timeout_ns = (uint64_t)qr_get_option(QR_OPT_WAIT_TIMEOUT_US) * 1000ull;
  {
    void* tb = nullptr;
    int64_t tc = 0;
    qr_trace_target(&tb, &tc);
    aa.trace = (TraceRec*)tb;
    aa.trace_cap = tc;
  }
  return trans ? launch_apply_dag<S, true>(aa, st) : launch_apply_dag<S, false>(aa, st);
}

}  // namespace

extern "C" {

int qr_workspace_p(int64_t m, int64_t n, int nb, int ib, int p, int prec, int64_t* t_elems, int64_t* scratch_bytes) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (nb == 0) {
    if (qr_table_lookup(m, n, prec == QR_PREC_F32 ? 4 : 8, &nb, &ib) != 0) return -3;
  }
  if (nb < 8 || nb > 512) return -3;
  if (ib < 1 || ib > nb || ib > 256) return -4;
  if (p < 1 || p > 4096) return -5;
  if (prec != QR_PREC_F64 && prec != QR_PREC_F32) return -6;
  std::lock_guard<std::mutex> lock(g_tmu2);
  if ((std::max<int64_t>(m, 1) + nb - 1) / nb > 65535) return -1;
  const PLayout L = p_layout(std::max<int64_t>(m, 1), std::max<int64_t>(n, 1), nb, ib, p,
                             prec == QR_PREC_F64 ? 8 : 4, true);
  if (t_elems) *t_elems = L.t_elems;
  if (scratch_bytes) *scratch_bytes = (int64_t)L.bytes;
  return 0;
}

int qr_factor_p_d(int64_t m, int64_t n, double* A, int64_t lda, int nb, int ib, int p, double* T, void* scratch,
                  int64_t scratch_bytes, void* stream) {
  return factor_p_impl<double>(m, n, A, lda, nb, ib, p, T, scratch, scratch_bytes, stream);
}

int qr_factor_p_s(int64_t m, int64_t n, float* A, int64_t lda, int nb, int ib, int p, float* T, void* scratch,
                  int64_t scratch_bytes, void* stream) {
  return factor_p_impl<float>(m, n, A, lda, nb, ib, p, T, scratch, scratch_bytes, stream);
}

int qr_apply_workspace_p(int64_t m, int64_t n, int64_t nrhs, int nb, int p, int64_t* bytes) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (nrhs < 1) return -3;
  if (nb == 0) {
    int ib = 0;
    if (qr_table_lookup(m, n, 8, &nb, &ib) != 0) return -4;
  }
  if (nb < 8 || nb > 512) return -4;
  if (p < 1 || p > 4096) return -5;
  if (!bytes) return -6;
  std::lock_guard<std::mutex> lock(g_tmu2);
  const APLayout L0 = ap_layout(m, n, nrhs, nb, p, 0);
  size_t nt = 0;
  for (int tr = 0; tr < 2; ++tr) nt = std::max(nt, apply_dag(L0.MT, L0.NT, L0.S, p, L0.last_short, tr).tasks.size());
  *bytes = (int64_t)ap_layout(m, n, nrhs, nb, p, (int64_t)nt).bytes;
  return 0;
}

int qr_apply_qt_p_d(int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda, int nb, int ib, int p,
                    const double* T, double* C, int64_t ldc, int trans, void* scratch, int64_t scratch_bytes,
                    void* stream) {
  return apply_p_impl<double>(m, n, nrhs, A, lda, nb, ib, p, T, C, ldc, trans, scratch, scratch_bytes, stream);
}

int qr_apply_qt_p_s(int64_t m, int64_t n, int64_t nrhs, const float* A, int64_t lda, int nb, int ib, int p,
                    const float* T, float* C, int64_t ldc, int trans, void* scratch, int64_t scratch_bytes,
                    void* stream) {
  return apply_p_impl<float>(m, n, nrhs, A, lda, nb, ib, p, T, C, ldc, trans, scratch, scratch_bytes, stream);
}

}  // extern "C"

int qr_factor_p_tc_s(int64_t m, int64_t n, float* A, int64_t lda, int nb, int ib, int p, float* T, void* scratch,
                     int64_t scratch_bytes, void* stream, int tc) {
  return factor_p_impl<float>(m, n, A, lda, nb, ib, p, T, scratch, scratch_bytes, stream, tc);
}
