// Host-side list scheduling of a task DAG (shared by the persistent
// schedulers): turns a topological program order into a ticket order.
#pragma once
#include <algorithm>
#include <cstdint>
#include <functional>
#include <queue>
#include <utility>
#include <vector>

namespace tqr {

// Ticket order from a list-scheduling simulation with the kernel's number of
// persistent CTAs as workers: tasks start when their predecessors have
// finished, the ready task with the longest path to the end (bottom level)
// first. With few workers the order follows what the GPU can actually run,
// so CTAs rarely hold a ticket whose dependencies are far in the future.
// prog order is topological; pred_off/pred list the direct predecessors.
inline std::vector<int64_t> list_schedule(const std::vector<double>& w, const std::vector<int64_t>& pred_off,
                                   const std::vector<int32_t>& pred, int workers) {
  const int64_t T = (int64_t)w.size();
  std::vector<int64_t> nsucc(T + 1, 0);
  for (int64_t t = 0; t < T; ++t)
    for (int64_t e = pred_off[t]; e < pred_off[t + 1]; ++e) ++nsucc[pred[e] + 1];
  for (int64_t t = 0; t < T; ++t) nsucc[t + 1] += nsucc[t];
  std::vector<int32_t> succ(pred.size());
  std::vector<int64_t> fill(nsucc.begin(), nsucc.end() - 1);
  std::vector<int32_t> indeg(T, 0);
  for (int64_t t = 0; t < T; ++t)
    for (int64_t e = pred_off[t]; e < pred_off[t + 1]; ++e) {
      succ[fill[pred[e]]++] = (int32_t)t;
      ++indeg[t];
    }
  std::vector<double> bl(T, 0.0);
  for (int64_t t = T - 1; t >= 0; --t) {
    double mx = 0.0;
    for (int64_t e = nsucc[t]; e < nsucc[t + 1]; ++e) mx = std::max(mx, bl[succ[e]]);
    bl[t] = w[t] + mx;
  }
  auto rcmp = [&](int64_t a, int64_t b) { return bl[a] < bl[b] || (bl[a] == bl[b] && a > b); };
  std::priority_queue<int64_t, std::vector<int64_t>, decltype(rcmp)> ready(rcmp);
  typedef std::pair<double, int64_t> Ev;
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> running;
  for (int64_t t = 0; t < T; ++t)
    if (indeg[t] == 0) ready.push(t);
  std::vector<int64_t> order;
  order.reserve(T);
  double now = 0.0;
  int busy = 0;
  while ((int64_t)order.size() < T) {
    while (busy < workers && !ready.empty()) {
      const int64_t t = ready.top();
      ready.pop();
      order.push_back(t);
      running.push(Ev(now + w[t], t));
      ++busy;
    }
    if (running.empty()) break;  // only if the graph had a cycle
    now = running.top().first;
    while (!running.empty() && running.top().first <= now) {
      const int64_t t = running.top().second;
      running.pop();
      --busy;
      for (int64_t e = nsucc[t]; e < nsucc[t + 1]; ++e)
        if (--indeg[succ[e]] == 0) ready.push(succ[e]);
    }
  }
  if ((int64_t)order.size() < T) {  // never expected: fall back to program order (topological)
    order.resize(T);
    for (int64_t t = 0; t < T; ++t) order[t] = t;
  }
  return order;
}

}  // namespace tqr
