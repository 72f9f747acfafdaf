// The empirical NB/IB autotuner (Secs. 5–6 of the paper), on the GPU.
//
// Step 1 (Sec. 5): time the update kernel that dominates the factorization
// (TSMQR, the paper's DSSRFB, O(NT^3) calls) for every (NB, IB) of the grid:
// 50 back-to-back launches of a device-filling batch of independent tile
// tasks, same data every call ("No Flush", the mode the paper reports).
// Then Property 5.1 keeps the best IB per NB, Property 5.2's upper convex
// hull of (NB, performance) is formed, and Heuristic 0/1/2 preselects at
// most 8 pairs.
// Step 2 (Sec. 6): time the whole factorization for the preselected pairs at
// each benchmarked order N, ascending, 6 runs each (median), and prune as
// you go with Property 6.1. Untuned orders use the closest tuned one
// (Sec. 6.1). The decision table is written to JSON and every measurement is
// appended to a JSONL log, which a later run reads to skip what is measured.
//
// Optionally (use_model = k > 0) a small MLP cost model (tileqr_mlp.cu),
// trained on the Step-2 timings gathered so far, ranks the survivors at each
// new order from the third one on; only the k it ranks best are measured
// (more when the ranking or the predictions prove unreliable), and the
// measurement always decides. The final model, fitted to every Step-2
// timing, is saved with the table and proposes pairs for untuned shapes.
// Step 1 can also run as MultCallFlushLRU (every launch on operands that are
// not in L2), the variant the paper leaves out of scope (Sec. 5).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "tile_kernels.cuh"
#include "tileqr_internal.h"

using namespace tqr;

namespace {

// ---------------------------------------------------------------------------
// Pure host rules (also exported for the CPU tests).
struct Pt {
  double x, y;
};

double cross(const Pt& o, const Pt& a, const Pt& b) { return (a.x - o.x) * (b.y - o.y) - (a.y - o.y) * (b.x - o.x); }

// Upper hull, left to right, both end points, collinear middle points dropped.
std::vector<Pt> upper_hull(std::vector<Pt> p) {
  std::sort(p.begin(), p.end(), [](const Pt& a, const Pt& b) { return a.x < b.x || (a.x == b.x && a.y < b.y); });
  std::vector<Pt> h;
  for (const Pt& q : p) {
    while (h.size() >= 2 && cross(h[h.size() - 2], h.back(), q) >= 0) h.pop_back();
    h.push_back(q);
  }
  return h;
}

std::vector<double> steepness(const std::vector<Pt>& h) {
  std::vector<double> s;
  Pt prev{0.0, 0.0};
  for (const Pt& q : h) {
    s.push_back((q.y - prev.y) / (q.x - prev.x));
    prev = q;
  }
  return s;
}

// Property 5.1 then the hull then H0/H1/H2. Returns selected NBs (ascending).
std::vector<int> select_nbs(const std::map<int, std::pair<int, double>>& best, int heuristic, int max_sel, int nseg,
                            int nb_lo, int nb_hi) {
  std::vector<Pt> pts;
  for (auto& kv : best) pts.push_back({(double)kv.first, kv.second.second});
  std::vector<Pt> h = upper_hull(pts);
  std::vector<double> st = steepness(h);
  std::vector<int> out;
  if (heuristic == 0) {
    for (auto& q : h) out.push_back((int)q.x);
  } else if (heuristic == 1) {
    std::vector<int> idx(h.size());
    for (size_t i = 0; i < h.size(); ++i) idx[i] = (int)i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return st[a] > st[b] || (st[a] == st[b] && h[a].x < h[b].x); });
    for (int i = 0; i < (int)idx.size() && i < max_sel; ++i) out.push_back((int)h[idx[i]].x);
  } else {
    const double w = (double)(nb_hi - nb_lo) / nseg;
    for (int s = 0; s < nseg; ++s) {
      const double a = nb_lo + s * w, b = nb_lo + (s + 1) * w;
      int bi = -1;
      for (int i = 0; i < (int)h.size(); ++i) {
        const bool inside = (h[i].x >= a && h[i].x < b) || (s == nseg - 1 && h[i].x == (double)nb_hi);
        if (inside && (bi < 0 || st[i] > st[bi])) bi = i;
      }
      if (bi >= 0) out.push_back((int)h[bi].x);
    }
  }
  std::sort(out.begin(), out.end());
  if ((int)out.size() > max_sel && heuristic != 0) out.resize(max_sel);
  return out;
}

std::vector<std::pair<int, int>> grid_pairs(int nb_lo, int nb_hi, int step, int ib_min) {
  std::vector<std::pair<int, int>> g;
  for (int nb = nb_lo; nb <= nb_hi; nb += step)
    for (int ib = ib_min; ib <= nb / 2; ++ib)
      if (nb % ib == 0) g.push_back({nb, ib});
  return g;
}

// ---------------------------------------------------------------------------
// Table (decision tree of Sec. 7: tuned at install time, read at call time).
struct Entry {
  int64_t m, n;
  int nb, ib;
  double gflops;
  int p;    // panel domains (1 = flat tree; tuned for tall-skinny shapes)
  int sms;  // SM budget the entry was tuned for (0 = the whole GPU)
};
std::mutex g_tmu;
std::vector<Entry> g_table[2];  // [0] fp64, [1] fp32

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    sms = 152;
  }
  return sms;
}

// The closest tuned configuration (Sec. 6.1), one dimension after the other
// as the paper's example reads (N = 1800 on 5 cores -> the point tuned for
// N = 2000 on 4 cores): first the closest SM budget among the entries (ties
// to the smaller), then among that budget's entries the closest shape,
// distance |m - m_i| + |n - n_i| (ties to the smaller shape). sms <= 0 and
// entries' sms = 0 both mean the whole GPU.
int lookup_entry(const std::vector<Entry>& t, int64_t m, int64_t n, int sms, int* nb, int* ib, int* pd) {
  if (t.empty()) return 1;
  int dev_sms = -1;
  auto eff = [&](int b) {
    if (b > 0) return b;
    if (dev_sms < 0) dev_sms = device_sm_count();
    return dev_sms;
  };
  const int want = eff(sms);
  int bsel = -1;
  for (const Entry& e : t) {
    const int b = eff(e.sms);
    if (bsel < 0 || std::abs(b - want) < std::abs(bsel - want) || (std::abs(b - want) == std::abs(bsel - want) && b < bsel))
      bsel = b;
  }
  int64_t best = INT64_MAX, bsum = INT64_MAX;
  int bi = -1;
  for (int i = 0; i < (int)t.size(); ++i) {
    if (eff(t[i].sms) != bsel) continue;
    const int64_t d = std::llabs(t[i].m - m) + std::llabs(t[i].n - n);
    const int64_t s = t[i].m + t[i].n;
    if (d < best || (d == best && s < bsum)) {
      best = d;
      bsum = s;
      bi = i;
    }
  }
  *nb = t[bi].nb;
  *ib = t[bi].ib;
  if (pd) *pd = t[bi].p;
  return 0;
}

// --- minimal JSON table writer/reader (flat, fixed schema) -----------------
bool write_table(const char* path, int prec, const std::vector<Entry>& t, const std::string& extra) {
  FILE* f = fopen(path, "w");
  if (!f) return false;
  fprintf(f, "{\n  \"prec\": \"%s\",\n%s  \"entries\": [\n", prec ? "fp32" : "fp64", extra.c_str());
  for (size_t i = 0; i < t.size(); ++i)
    fprintf(f, "    {\"m\": %lld, \"n\": %lld, \"nb\": %d, \"ib\": %d, \"p\": %d, \"gflops\": %.4f, \"sms\": %d}%s\n",
            (long long)t[i].m, (long long)t[i].n, t[i].nb, t[i].ib, t[i].p, t[i].gflops, t[i].sms,
            i + 1 < t.size() ? "," : "");
  fprintf(f, "  ]\n}\n");
  fclose(f);
  return true;
}

bool read_table(const char* path, int* prec, std::vector<Entry>* t, std::string* text = nullptr) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  std::string s;
  char buf[4096];
  size_t r;
  while ((r = fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, r);
  fclose(f);
  *prec = (s.find("\"prec\": \"fp32\"") != std::string::npos) ? 1 : 0;
  if (text) *text = s;
  size_t p = s.find("\"entries\"");
  if (p == std::string::npos) return false;
  t->clear();
  while ((p = s.find("{\"m\":", p)) != std::string::npos) {
    Entry e;
    long long m, n;
    e.p = 1;
    e.sms = 0;
    if (sscanf(s.c_str() + p, "{\"m\": %lld, \"n\": %lld, \"nb\": %d, \"ib\": %d, \"p\": %d, \"gflops\": %lf", &m,
               &n, &e.nb, &e.ib, &e.p, &e.gflops) != 6 &&
        sscanf(s.c_str() + p, "{\"m\": %lld, \"n\": %lld, \"nb\": %d, \"ib\": %d, \"gflops\": %lf", &m, &n, &e.nb,
               &e.ib, &e.gflops) != 5)
      return false;
    if (e.p < 1) e.p = 1;
    {
      const size_t close = s.find('}', p);
      const size_t k = s.find("\"sms\": ", p);
      if (k != std::string::npos && k < close) e.sms = std::max(0, atoi(s.c_str() + k + 7));
    }
    e.m = m;
    e.n = n;
    t->push_back(e);
    ++p;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Device helpers for Step 1 and Step 2 inputs.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  // SplitMix64 finalizer (Steele, Lea, Flood 2014)
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

template <typename S>
__global__ void fill_uniform(S* p, int64_t n, uint64_t seed, double lo, double hi) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double u = (double)(mix64(seed * 0x100000001B3ull + (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
    p[i] = (S)(lo + (hi - lo) * u);
  }
}

// Step-1 kernel: CTA b applies one TSMQR (V, T shared) to its own tile pair;
// tc (FP32 tiles) selects the tensor-core update of the mixed precisions.
template <typename S>
__global__ void __launch_bounds__(NTHREADS, 2)
    tsmqr_batch(const S* V, const S* T, S* C1, S* C2, int NB, int IB, int tc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem<S> sm = carve<S>(reinterpret_cast<S*>(smem_raw));
  const size_t te = (size_t)NB * NB;
  tsmqr<S>(V, NB, T, IB, NB, NB, C1 + blockIdx.x * te, NB, C2 + blockIdx.x * te, NB, 0, NB, sm, false, tc);
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

int64_t step1_bytes(int nb, int nbatch, size_t esz) {
  // V, T (NB x NB each, generous) + two tiles per task
  return (int64_t)((2 + 2 * (size_t)nbatch) * nb * nb * esz) + 4096;
}

int64_t l2_bytes() {
  int dev = 0, l2 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  return l2 > 0 ? l2 : (128ll << 20);
}

// MultCallFlushLRU: every launch works on its own copy of the operands
// (V, T and the tile pairs), the copies taken in turn, and there are enough
// of them that the ones a launch reads were last touched more than two L2
// capacities of traffic ago: each launch finds its data in HBM, not in L2.
int step1_flush_sets(int nb, int nbatch, size_t esz) {
  const int64_t set = step1_bytes(nb, nbatch, esz);
  return (int)std::max<int64_t>(2, (2 * l2_bytes() + set - 1) / set + 1);
}

int64_t step1_flush_bytes(int nb, int nbatch, size_t esz) {
  return (int64_t)step1_flush_sets(nb, nbatch, esz) * step1_bytes(nb, nbatch, esz);
}

// Extra workspace of the flushed Step 1 over the plain one, largest over the grid.
int64_t step1_flush_extra(size_t esz) {
  int64_t best = 0;
  const int nbatch = 2 * sm_count();
  for (int nb = 64; nb <= 512; nb += 32)
    best = std::max(best, step1_flush_bytes(nb, nbatch, esz) - step1_bytes(512, nbatch, esz));
  return best;
}

// One operand set of the Step-1 batch: V, T, then the nbatch tile pairs.
template <typename S>
struct Step1Set {
  S *V, *T, *C1, *C2;
};
template <typename S>
Step1Set<S> step1_set(void* work, int nb, int nbatch, int k) {
  const size_t te = (size_t)nb * nb;
  Step1Set<S> o;
  o.V = (S*)((char*)work + (size_t)k * step1_bytes(nb, nbatch, sizeof(S)));
  o.T = o.V + te;
  o.C1 = o.T + te;
  o.C2 = o.C1 + (size_t)nbatch * te;
  return o;
}

// flush = 0: "No Flush", every launch on the same data (the mode the paper
// reports, Sec. 5). flush = 1: MultCallFlushLRU, launch l on operand set
// l mod nsets (step1_flush_sets), so its data is never in L2.
template <typename S>
int step1_time(int nb, int ib, int nbatch, int launches, int flush, double* sec, void* work, int64_t wbytes,
               cudaStream_t st, int tc = TC_NONE) {
  const int nsets = flush ? step1_flush_sets(nb, nbatch, sizeof(S)) : 1;
  if ((int64_t)nsets * step1_bytes(nb, nbatch, sizeof(S)) > wbytes) return -7;
  const size_t te = (size_t)nb * nb;
  for (int k = 0; k < nsets; ++k) {
    const Step1Set<S> o = step1_set<S>(work, nb, nbatch, k);
    fill_uniform<S><<<1024, 256, 0, st>>>(o.V, (int64_t)te, 11 + 16 * k, -0.05, 0.05);
    fill_uniform<S><<<1024, 256, 0, st>>>(o.T, (int64_t)te, 12 + 16 * k, 0.0, 0.05);
    fill_uniform<S><<<1024, 256, 0, st>>>(o.C1, (int64_t)(2 * nbatch * te), 13 + 16 * k, -0.5, 0.5);
  }
  const size_t smem = (sizeof(S) == 4 && tc != TC_NONE) ? std::max<size_t>(smem_elems<S>() * sizeof(S), TC_SMEM_BYTES)
                                                       : smem_elems<S>() * sizeof(S);
  cudaError_t e = cudaFuncSetAttribute(tsmqr_batch<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  int cur = 0;
  auto launch = [&]() {
    const Step1Set<S> o = step1_set<S>(work, nb, nbatch, cur);
    cur = (cur + 1) % nsets;
    tsmqr_batch<S><<<nbatch, NTHREADS, smem, st>>>(o.V, o.T, o.C1, o.C2, nb, ib, tc);
  };
  launch();  // warm-up
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  if (launches <= 0) {
    // adaptive count: time one launch, then take as many as fill ~30 ms
    // (at least 3, at most the paper's 50)
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms1 = 1.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms1, e0, e1);
    if (e != cudaSuccess) return (int)e;
    launches = (int)std::ceil(30.0 / std::max(ms1, 1e-3f));
    launches = std::max(3, std::min(50, launches));
  }
  cudaEventRecord(e0, st);
  for (int l = 0; l < launches; ++l) launch();
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return (int)e;
  *sec = ms * 1e-3 / launches;
  return 0;
}

// Step-2 timing of qr_factor at (m, n, nb, ib): reps runs, returns median and
// min seconds. The matrix is regenerated on the device before every run.
template <typename S>
int time_factor(int64_t m, int64_t n, int nb, int ib, int pd, int reps, void* work, int64_t wbytes, cudaStream_t st,
                double* med, double* mn) {
  int64_t t_el = 0, sb = 0;
  int rc = pd > 1 ? qr_workspace_p(m, n, nb, ib, pd, sizeof(S) == 8 ? QR_PREC_F64 : QR_PREC_F32, &t_el, &sb)
                  : qr_workspace(m, n, nb, ib, sizeof(S) == 8 ? QR_PREC_F64 : QR_PREC_F32, &t_el, &sb);
  if (rc) return rc;
  const size_t a_bytes = ((size_t)m * n * sizeof(S) + 255) & ~(size_t)255;
  const size_t t_bytes = ((size_t)t_el * sizeof(S) + 255) & ~(size_t)255;
  if ((int64_t)(a_bytes + t_bytes + sb) > wbytes) return -7;
  S* A = (S*)work;
  S* T = (S*)((char*)work + a_bytes);
  void* scr = (char*)work + a_bytes + t_bytes;
  std::vector<double> ts;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // the task order is built (and cached) on the host outside the timed runs;
  // small problems also get one untimed warm-up run
  qr_prepare_schedule(m, n, nb, ib, sizeof(S) == 8 ? QR_PREC_F64 : QR_PREC_F32);
  const int warm = (m * n <= 4000000) ? 1 : 0;
  for (int r = 1 - warm; r < reps + 1; ++r) {
    fill_uniform<S><<<1184, 256, 0, st>>>(A, m * n, (uint64_t)(m * 31 + n), -0.5, 0.5);
    cudaEventRecord(e0, st);
    if (pd > 1)
      rc = sizeof(S) == 8 ? qr_factor_p_d(m, n, (double*)A, m, nb, ib, pd, (double*)T, scr, sb, st)
                          : qr_factor_p_s(m, n, (float*)A, m, nb, ib, pd, (float*)T, scr, sb, st);
    else
      rc = sizeof(S) == 8 ? qr_factor_d(m, n, (double*)A, m, nb, ib, (double*)T, scr, sb, st)
                          : qr_factor_s(m, n, (float*)A, m, nb, ib, (float*)T, scr, sb, st);
    cudaEventRecord(e1, st);
    if (rc) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { rc = (int)e; break; }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    int status = 0;
    qr_status(scr, &status, st);
    if (status) { rc = 1000 + status; break; }
    if (r > 0) ts.push_back(ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  std::sort(ts.begin(), ts.end());
  *med = ts[ts.size() / 2];
  if (ts.size() % 2 == 0) *med = 0.5 * (ts[ts.size() / 2 - 1] + ts[ts.size() / 2]);
  *mn = ts.front();
  return 0;
}

double qr_flops_d(int64_t m, int64_t n) { return 2.0 * m * (double)n * n - 2.0 * (double)n * n * n / 3.0; }

// --- the learned cost model inside the search --------------------------------
// The tuner's own Step-2 timings train the MLP of tileqr_mlp.cu (features
// (log m, log n, NB/512, IB/256), standardized over the training set; target
// log seconds, centred). Its device buffers sit at the start of the tuner's
// workspace (kModelBytes); the factorization timings use the rest.
constexpr int kModelCap = 4096;  // training samples at most
constexpr int64_t kModelBytes = QR_MODEL_WORK_BYTES;
constexpr int kModelSteps = 3000;
constexpr float kModelLr = 1e-3f;
constexpr double kModelTrust = 0.25;  // |log t_measured - log t_predicted| allowed before falling back

struct Model {
  bool ok = false;
  float mean[4] = {0, 0, 0, 0}, sd[4] = {1, 1, 1, 1};
  float ymean = 0.f;
  std::vector<float> params;
  std::vector<std::pair<int, int>> pairs;  // candidate (NB, IB) pairs it was trained on
};
Model g_model[2];  // [0] fp64, [1] fp32 (guarded by g_tmu)

struct Sample {
  int64_t m, n;
  int nb, ib;
  double sec;
};

void raw_features(int64_t m, int64_t n, int nb, int ib, float* f) {
  f[0] = (float)std::log((double)m);
  f[1] = (float)std::log((double)n);
  f[2] = (float)(nb / 512.0);
  f[3] = (float)(ib / 256.0);
}

// Initial weights: each Linear(in, out) draws W and b uniform in
// [-1/sqrt(in), 1/sqrt(in)] from a SplitMix64 stream (fixed seed).
std::vector<float> model_init(uint64_t seed) {
  std::vector<float> p(QR_MLP_NPARAMS);
  const int fin[3] = {4, 64, 64}, fout[3] = {64, 64, 1};
  uint64_t x = seed;
  auto next = [&x]() {
    x += 0x9E3779B97F4A7C15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  size_t o = 0;
  for (int l = 0; l < 3; ++l) {
    const double b = 1.0 / std::sqrt((double)fin[l]);
    for (int e = 0; e < fin[l] * fout[l] + fout[l]; ++e) p[o++] = (float)(-b + 2.0 * b * next());
  }
  return p;
}

struct ModelDev {
  float *P, *M, *V, *G, *X, *Y, *out, *work;
};
ModelDev model_dev(void* base) {
  float* f = (float*)base;
  ModelDev d;
  d.P = f;
  d.M = d.P + QR_MLP_NPARAMS;
  d.V = d.M + QR_MLP_NPARAMS;
  d.G = d.V + QR_MLP_NPARAMS;
  d.X = d.G + QR_MLP_NPARAMS + 1;
  d.Y = d.X + 4 * kModelCap;
  d.out = d.Y + kModelCap;
  d.work = d.out + kModelCap;
  return d;
}

// Fits the model to the samples from the same initial weights every time
// (full batch, Adam); synchronous.
int model_fit(const std::vector<Sample>& data, const std::vector<std::pair<int, int>>& pairs, void* base,
              cudaStream_t st, Model* md) {
  const int ns = (int)std::min<size_t>(data.size(), kModelCap);
  if (ns < 2) return -1;
  std::vector<float> X(4 * (size_t)ns), Y(ns);
  double mu[4] = {0, 0, 0, 0}, sq[4] = {0, 0, 0, 0}, ym = 0;
  for (int s = 0; s < ns; ++s) {
    raw_features(data[s].m, data[s].n, data[s].nb, data[s].ib, &X[4 * s]);
    for (int i = 0; i < 4; ++i) mu[i] += X[4 * s + i];
    ym += std::log(data[s].sec);
  }
  Model m;
  for (int i = 0; i < 4; ++i) mu[i] /= ns;
  for (int s = 0; s < ns; ++s)
    for (int i = 0; i < 4; ++i) sq[i] += (X[4 * s + i] - mu[i]) * (X[4 * s + i] - mu[i]);
  for (int i = 0; i < 4; ++i) {
    m.mean[i] = (float)mu[i];
    const double sd = std::sqrt(sq[i] / ns);
    m.sd[i] = sd > 0 ? (float)sd : 1.f;
  }
  m.ymean = (float)(ym / ns);
  for (int s = 0; s < ns; ++s) {
    for (int i = 0; i < 4; ++i) X[4 * s + i] = (X[4 * s + i] - m.mean[i]) / m.sd[i];
    Y[s] = (float)std::log(data[s].sec) - m.ymean;
  }
  m.params = model_init(0x5EED0001ull);
  const ModelDev d = model_dev(base);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d.P, m.params.data(), sizeof(float) * QR_MLP_NPARAMS, cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemsetAsync(d.M, 0, sizeof(float) * 2 * QR_MLP_NPARAMS, st)) ||
      (e = cudaMemcpyAsync(d.X, X.data(), sizeof(float) * X.size(), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(d.Y, Y.data(), sizeof(float) * ns, cudaMemcpyHostToDevice, st)))
    return (int)e;
  int rc = qr_mlp_train(ns, d.X, d.Y, d.P, d.M, d.V, kModelSteps, kModelLr, d.G, d.work, st);
  if (rc) return rc;
  if ((e = cudaMemcpyAsync(m.params.data(), d.P, sizeof(float) * QR_MLP_NPARAMS, cudaMemcpyDeviceToHost, st)))
    return (int)e;
  if ((e = cudaStreamSynchronize(st))) return (int)e;
  m.pairs = pairs;
  m.ok = true;
  *md = m;
  return 0;
}

// Predicted seconds of each (NB, IB) at (m, n); synchronous.
int model_predict(const Model& md, int64_t m, int64_t n, const std::vector<std::pair<int, int>>& pairs, void* base,
                  cudaStream_t st, std::vector<double>* sec) {
  const int np = (int)pairs.size();
  if (np == 0 || np > kModelCap) return -1;
  std::vector<float> X(4 * (size_t)np), out(np);
  for (int s = 0; s < np; ++s) {
    raw_features(m, n, pairs[s].first, pairs[s].second, &X[4 * s]);
    for (int i = 0; i < 4; ++i) X[4 * s + i] = (X[4 * s + i] - md.mean[i]) / md.sd[i];
  }
  const ModelDev d = model_dev(base);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d.P, md.params.data(), sizeof(float) * QR_MLP_NPARAMS, cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(d.X, X.data(), sizeof(float) * X.size(), cudaMemcpyHostToDevice, st)))
    return (int)e;
  int rc = qr_mlp_forward(np, d.X, d.P, d.out, st);
  if (rc) return rc;
  if ((e = cudaMemcpyAsync(out.data(), d.out, sizeof(float) * np, cudaMemcpyDeviceToHost, st)) ||
      (e = cudaStreamSynchronize(st)))
    return (int)e;
  sec->resize(np);
  for (int s = 0; s < np; ++s) (*sec)[s] = std::exp((double)out[s] + md.ymean);
  return 0;
}

std::string model_json(const Model& md) {
  std::string s = "  \"model\": {\"mean\": [";
  char b[64];
  for (int i = 0; i < 4; ++i) {
    snprintf(b, sizeof(b), "%s%.9g", i ? ", " : "", md.mean[i]);
    s += b;
  }
  s += "], \"sd\": [";
  for (int i = 0; i < 4; ++i) {
    snprintf(b, sizeof(b), "%s%.9g", i ? ", " : "", md.sd[i]);
    s += b;
  }
  snprintf(b, sizeof(b), "], \"ymean\": %.9g, \"pairs\": [", md.ymean);
  s += b;
  for (size_t i = 0; i < md.pairs.size(); ++i) {
    snprintf(b, sizeof(b), "%s[%d, %d]", i ? ", " : "", md.pairs[i].first, md.pairs[i].second);
    s += b;
  }
  s += "], \"params\": [";
  for (size_t i = 0; i < md.params.size(); ++i) {
    snprintf(b, sizeof(b), "%s%.9g", i ? ", " : "", md.params[i]);
    s += b;
  }
  s += "]},\n";
  return s;
}

// Parses the "model" object written by model_json; false if absent or malformed.
bool parse_model(const std::string& s, Model* md) {
  size_t p = s.find("\"model\": {");
  if (p == std::string::npos) return false;
  Model m;
  auto read_floats = [&](const char* key, float* out, size_t count, size_t* pos) {
    size_t q = s.find(key, *pos);
    if (q == std::string::npos) return false;
    q = s.find('[', q);
    if (q == std::string::npos) return false;
    const char* c = s.c_str() + q + 1;
    for (size_t i = 0; i < count; ++i) {
      char* end = nullptr;
      out[i] = strtof(c, &end);
      if (end == c) return false;
      c = end;
      while (*c == ',' || *c == ' ' || *c == '\n') ++c;
    }
    *pos = (size_t)(c - s.c_str());
    return true;
  };
  size_t pos = p;
  if (!read_floats("\"mean\"", m.mean, 4, &pos) || !read_floats("\"sd\"", m.sd, 4, &pos)) return false;
  size_t q = s.find("\"ymean\": ", pos);
  if (q == std::string::npos) return false;
  m.ymean = strtof(s.c_str() + q + 9, nullptr);
  q = s.find("\"pairs\": [", q);
  if (q == std::string::npos) return false;
  q += 10;
  while (true) {
    int a, b;
    while (q < s.size() && (s[q] == ' ' || s[q] == ',')) ++q;
    if (q >= s.size() || s[q] != '[') break;
    if (sscanf(s.c_str() + q, "[%d, %d]", &a, &b) != 2) return false;
    m.pairs.push_back({a, b});
    q = s.find(']', q) + 1;
  }
  m.params.resize(QR_MLP_NPARAMS);
  pos = q;
  if (!read_floats("\"params\"", m.params.data(), QR_MLP_NPARAMS, &pos)) return false;
  if (m.pairs.empty()) return false;
  m.ok = true;
  *md = m;
  return true;
}

// --- resumable JSONL log ------------------------------------------------------
struct LogKey {
  // 1 = step 1, 2 = step 2 (p = 1), 3 = domain sweep of a tall shape,
  // 4 = the model's predicted seconds (not reused), 5 = step 1 (MultCallFlushLRU)
  int kind;
  int64_t m, n;
  int nb, ib;
  int p;
  int sms;  // SM budget of a Step-2 timing (0 = the whole GPU; Step 1 is always 0)
  bool operator<(const LogKey& o) const {
    return std::tie(kind, m, n, nb, ib, p, sms) < std::tie(o.kind, o.m, o.n, o.nb, o.ib, o.p, o.sms);
  }
};

void read_log(const char* path, std::map<LogKey, double>* seen) {
  if (!path || !path[0]) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    int kind, nb, ib;
    long long m, n;
    double sec;
    if (sscanf(line, "{\"kind\": %d, \"m\": %lld, \"n\": %lld, \"nb\": %d, \"ib\": %d, \"seconds\": %lf", &kind, &m,
               &n, &nb, &ib, &sec) == 6) {
      int pd = 1, sb = 0;
      const char* pp = strstr(line, "\"p\": ");
      if (pp) pd = atoi(pp + 5);
      const char* ps = strstr(line, "\"sms\": ");
      if (ps) sb = atoi(ps + 7);
      (*seen)[LogKey{kind, m, n, nb, ib, pd, sb}] = sec;
    }
  }
  fclose(f);
}

void append_log(const char* path, int kind, int64_t m, int64_t n, int nb, int ib, double sec, double smin,
                int reps, int pd = 1, int sms = 0) {
  if (!path || !path[0]) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"kind\": %d, \"m\": %lld, \"n\": %lld, \"nb\": %d, \"ib\": %d, \"seconds\": %.9g, \"min\": %.9g, "
             "\"reps\": %d, \"p\": %d, \"sms\": %d}\n",
          kind, (long long)m, (long long)n, nb, ib, sec, smin, reps, pd, sms);
  fclose(f);
}

}  // namespace

// ---------------------------------------------------------------------------
int qr_table_lookup(int64_t m, int64_t n, int elem_bytes, int* nb, int* ib, int* pd) {
  const int sms = (int)qr_get_option(QR_OPT_SM_BUDGET);  // read before g_tmu: never both locks at once
  std::lock_guard<std::mutex> lock(g_tmu);
  const int p = elem_bytes == 4 ? 1 : 0;
  if (pd) *pd = 1;
  if (lookup_entry(g_table[p], m, n, sms, nb, ib, pd) == 0) return 0;
  if (p == 1 && lookup_entry(g_table[0], m, n, sms, nb, ib, pd) == 0) return 0;
  *nb = 128;  // built-in default when nothing is loaded
  *ib = 16;
  return 0;
}

extern "C" {

int qr_load_table(const char* path) {
  if (!path) return -1;
  int prec = 0;
  std::vector<Entry> t;
  std::string text;
  if (!read_table(path, &prec, &t, &text)) return -1;
  Model md;
  const bool has_model = parse_model(text, &md);
  std::lock_guard<std::mutex> lock(g_tmu);
  g_table[prec] = t;
  g_model[prec] = has_model ? md : Model();
  return 0;
}

int qr_clear_tables(void) {
  std::lock_guard<std::mutex> lock(g_tmu);
  g_table[0].clear();
  g_table[1].clear();
  g_model[0] = Model();
  g_model[1] = Model();
  return 0;
}

int qr_model_propose(int64_t m, int64_t n, int prec, int* nb, int* ib, double* seconds, void* d_work,
                     int64_t work_bytes, void* stream) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (prec != QR_PREC_F64 && prec != QR_PREC_F32) return -3;
  if (!nb) return -4;
  if (!ib) return -5;
  if (!d_work) return -7;
  if (work_bytes < kModelBytes) return -8;
  Model md;
  {
    std::lock_guard<std::mutex> lock(g_tmu);
    md = g_model[prec == QR_PREC_F32 ? 1 : 0];
  }
  if (!md.ok) return 1;  // no trained model for this precision
  std::vector<double> sec;
  int rc = model_predict(md, m, n, md.pairs, d_work, (cudaStream_t)stream, &sec);
  if (rc) return rc;
  size_t bi = 0;
  for (size_t c = 1; c < sec.size(); ++c)
    if (sec[c] < sec[bi]) bi = c;
  *nb = md.pairs[bi].first;
  *ib = md.pairs[bi].second;
  if (seconds) *seconds = sec[bi];
  return 0;
}

int qr_lookup(int64_t m, int64_t n, int prec, int* nb, int* ib) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (prec != QR_PREC_F64 && prec != QR_PREC_F32) return -3;
  if (!nb) return -4;
  if (!ib) return -5;
  return qr_table_lookup(m, n, prec == QR_PREC_F32 ? 4 : 8, nb, ib, nullptr);
}

int qr_lookup_sms(int64_t m, int64_t n, int prec, int sms, int* nb, int* ib, int* p) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (prec < QR_PREC_F64 || prec > QR_PREC_BF16X3) return -3;
  if (sms < 0) return -4;
  if (!nb) return -5;
  if (!ib) return -6;
  std::lock_guard<std::mutex> lock(g_tmu);
  const int t = prec == QR_PREC_F64 ? 0 : 1;
  int pd = 1;
  if (lookup_entry(g_table[t], m, n, sms, nb, ib, &pd) != 0 && (t == 0 || lookup_entry(g_table[0], m, n, sms, nb, ib, &pd) != 0)) {
    *nb = 128;
    *ib = 16;
    pd = 1;
  }
  if (p) *p = pd;
  return 0;
}

int qr_lookup_p(int64_t m, int64_t n, int prec, int* nb, int* ib, int* p) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (prec != QR_PREC_F64 && prec != QR_PREC_F32) return -3;
  if (!nb) return -4;
  if (!ib) return -5;
  if (!p) return -6;
  return qr_table_lookup(m, n, prec == QR_PREC_F32 ? 4 : 8, nb, ib, p);
}

int qr_tune_grid(int nb_lo, int nb_hi, int nb_step, int ib_min, int cap, int* nbs, int* ibs) {
  if (nb_lo < 1 || nb_hi < nb_lo || nb_step < 1 || ib_min < 1) return -1;
  auto g = grid_pairs(nb_lo, nb_hi, nb_step, ib_min);
  if (nbs && ibs)
    for (int i = 0; i < (int)g.size() && i < cap; ++i) {
      nbs[i] = g[i].first;
      ibs[i] = g[i].second;
    }
  return (int)g.size();
}

int qr_tune_preselect(int npairs, const int* nb, const int* ib, const double* perf, int heuristic, int max_sel,
                      int nseg, int* sel_nb, int* sel_ib) {
  if (npairs <= 0 || !nb || !ib || !perf) return -1;
  if (heuristic < 0 || heuristic > 2) return -5;
  std::map<int, std::pair<int, double>> best;  // Property 5.1
  int lo = INT32_MAX, hi = 0;
  for (int i = 0; i < npairs; ++i) {
    lo = std::min(lo, nb[i]);
    hi = std::max(hi, nb[i]);
    auto it = best.find(nb[i]);
    if (it == best.end() || perf[i] > it->second.second ||
        (perf[i] == it->second.second && ib[i] < it->second.first))
      best[nb[i]] = {ib[i], perf[i]};
  }
  std::vector<int> sel = select_nbs(best, heuristic, max_sel, nseg, lo, hi);
  for (size_t i = 0; i < sel.size(); ++i) {
    sel_nb[i] = sel[i];
    sel_ib[i] = best[sel[i]].first;
  }
  return (int)sel.size();
}

int qr_tune_payg(int nsurv, const int* nb, const double* perf, int* keep) {
  if (nsurv < 0 || (nsurv > 0 && (!nb || !perf || !keep))) return -1;
  for (int a = 0; a < nsurv; ++a) {
    keep[a] = 1;
    for (int b = 0; b < nsurv; ++b)
      if (nb[b] > nb[a] && perf[b] > perf[a]) keep[a] = 0;  // Property 6.1
  }
  return 0;
}

int64_t qr_tune_nearest(int64_t value, const int64_t* grid, int ngrid) {
  if (ngrid <= 0 || !grid) return -1;
  int64_t best = grid[0];
  for (int i = 1; i < ngrid; ++i) {
    const int64_t d = std::llabs(grid[i] - value), db = std::llabs(best - value);
    if (d < db || (d == db && grid[i] < best)) best = grid[i];
  }
  return best;
}

int qr_step1_workspace(int nb, int prec, int flush, int64_t* bytes) {
  if (nb < 8 || nb > 512) return -1;
  if (prec < QR_PREC_F64 || prec > QR_PREC_BF16X3) return -2;
  if (flush != 0 && flush != 1) return -3;
  if (!bytes) return -4;
  const size_t esz = prec == QR_PREC_F64 ? 8 : 4;
  *bytes = flush ? step1_flush_bytes(nb, 2 * sm_count(), esz) : step1_bytes(nb, 2 * sm_count(), esz);
  return 0;
}

int qr_step1_time(int nb, int ib, int prec, int launches, int flush, double* seconds_per_launch, double* gflops,
                  void* d_work, int64_t work_bytes, void* stream) {
  if (nb < 8 || nb > 512) return -1;
  if (ib < 1 || ib > nb || ib > 256) return -2;
  if (prec < QR_PREC_F64 || prec > QR_PREC_BF16X3) return -3;
  if (flush != 0 && flush != 1) return -5;
  if (!seconds_per_launch) return -6;
  const int nbatch = 2 * sm_count();
  double s = 0;  // launches <= 0: adaptive count (3..50)
  const int rc =
      prec == QR_PREC_F64
          ? step1_time<double>(nb, ib, nbatch, launches, flush, &s, d_work, work_bytes, (cudaStream_t)stream)
          : step1_time<float>(nb, ib, nbatch, launches, flush, &s, d_work, work_bytes, (cudaStream_t)stream,
                              tc_of_prec(prec));
  if (rc) return rc;
  *seconds_per_launch = s;
  if (gflops) *gflops = nbatch * 4.0 * nb * (double)nb * nb / s / 1e9;
  return 0;
}

int qr_tune_workspace(int64_t max_m, int64_t max_n, int prec, int64_t* bytes) {
  if (max_m < 1 || max_n < 1 || max_n > max_m) return -1;
  if (!bytes) return -4;
  const size_t esz = prec == QR_PREC_F32 ? 4 : 8;
  int64_t best = step1_bytes(512, 2 * sm_count(), esz) + step1_flush_extra(esz);
  for (int nb = 64; nb <= 512; nb += 32) {
    int64_t t_el = 0, sb = 0;
    // the domain-tree path (tall-skinny p sweep) needs the larger scratch
    qr_workspace_p(max_m, max_n, nb, std::min(nb / 2, 256), 64, prec, &t_el, &sb);
    const int64_t need = (int64_t)(((size_t)max_m * max_n * esz + 255) & ~(size_t)255) +
                         (int64_t)((t_el * esz + 255) & ~(size_t)255) + sb;
    best = std::max(best, need);
  }
  *bytes = best + kModelBytes;  // the cost model's buffers come first
  return 0;
}

int qr_time_factor(int64_t m, int64_t n, int nb, int ib, int prec, int reps, double* median_s, double* min_s,
                   void* d_work, int64_t work_bytes, void* stream) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (reps < 1) return -6;
  if (!median_s || !min_s) return -7;
  return prec == QR_PREC_F32 ? time_factor<float>(m, n, nb, ib, 1, reps, d_work, work_bytes, (cudaStream_t)stream,
                                                  median_s, min_s)
                             : time_factor<double>(m, n, nb, ib, 1, reps, d_work, work_bytes, (cudaStream_t)stream,
                                                   median_s, min_s);
}

int qr_time_factor_p(int64_t m, int64_t n, int nb, int ib, int p, int prec, int reps, double* median_s, double* min_s,
                     void* d_work, int64_t work_bytes, void* stream) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (p < 1 || p > 4096) return -5;
  if (reps < 1) return -7;
  if (!median_s || !min_s) return -8;
  return prec == QR_PREC_F32 ? time_factor<float>(m, n, nb, ib, p, reps, d_work, work_bytes, (cudaStream_t)stream,
                                                  median_s, min_s)
                             : time_factor<double>(m, n, nb, ib, p, reps, d_work, work_bytes, (cudaStream_t)stream,
                                                   median_s, min_s);
}

int qr_tune(const int64_t* ms, const int64_t* ns, int nshapes, int heuristic, int mode, int use_model, int reps,
            int prec, const char* table_path, const char* log_path, void* d_work, int64_t work_bytes,
            double* seconds_out, void* stream) {
  if (!ms || !ns || nshapes < 1) return -1;
  if (heuristic < 0 || heuristic > 2) return -4;
  if (mode < 0 || mode > 3) return -5;
  if (use_model < 0 || use_model > 8) return -6;
  if (reps < 1) return -7;
  if (prec != QR_PREC_F64 && prec != QR_PREC_F32) return -8;
  if (!d_work) return -11;
  if (work_bytes <= kModelBytes) return -12;
  const bool exhaustive = (mode & 1) != 0;
  const int flush = (mode >> 1) & 1;
  // the SM budget (QR_OPT_SM_BUDGET) every Step-2 timing of this call runs
  // under; 0 = the whole GPU. Step 1 is budget-independent, as in the paper.
  const int budget = (int)std::min<int64_t>(qr_get_option(QR_OPT_SM_BUDGET), sm_count());
  cudaStream_t st = (cudaStream_t)stream;
  void* mwork = d_work;  // the cost model's buffers
  void* fwork = (char*)d_work + kModelBytes;
  const int64_t fbytes = work_bytes - kModelBytes;
  const auto t_start = std::chrono::steady_clock::now();
  auto since = [](std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  };
  std::map<LogKey, double> seen;
  read_log(log_path, &seen);
  auto grid = grid_pairs(64, 512, 32, 8);
  std::vector<std::pair<int, int>> cand;
  double step1_s = 0, model_s = 0;
  const int step1_kind = flush ? 5 : 1;
  if (exhaustive) {
    cand = grid;  // exhaustive search over the grid
  } else {
    std::vector<int> nb(grid.size()), ib(grid.size());
    std::vector<double> perf(grid.size());
    for (size_t g = 0; g < grid.size(); ++g) {
      nb[g] = grid[g].first;
      ib[g] = grid[g].second;
      double s = 0, gf = 0;
      auto it = seen.find(LogKey{step1_kind, 0, 0, nb[g], ib[g], 1, 0});
      if (it != seen.end()) {
        s = it->second;
      } else {
        const auto t0 = std::chrono::steady_clock::now();
        int rc = qr_step1_time(nb[g], ib[g], prec, 0, flush, &s, &gf, fwork, fbytes, stream);
        if (rc) return rc;
        step1_s += since(t0);
        append_log(log_path, step1_kind, 0, 0, nb[g], ib[g], s, s, 0);
      }
      perf[g] = 2.0 * sm_count() * 4.0 * nb[g] * (double)nb[g] * nb[g] / s / 1e9;
    }
    std::vector<int> sn(grid.size()), si(grid.size());
    const int k = qr_tune_preselect((int)grid.size(), nb.data(), ib.data(), perf.data(), heuristic, 8, 8, sn.data(),
                                    si.data());
    // QR_OPT_TUNE_IB_TOL > 0: each preselected NB also brings every other IB
    // whose kernel rate is within that tolerance of its best IB's (ascending
    // IB after the best); 0 is Property 5.1 as the paper states it
    const double tol = (double)qr_get_option(QR_OPT_TUNE_IB_TOL) / 1000.0;
    for (int i = 0; i < k; ++i) {
      cand.push_back({sn[i], si[i]});
      if (tol <= 0) continue;
      double pbest = 0;
      for (size_t g = 0; g < grid.size(); ++g)
        if (nb[g] == sn[i] && ib[g] == si[i]) pbest = perf[g];
      for (size_t g = 0; g < grid.size(); ++g)
        if (nb[g] == sn[i] && ib[g] != si[i] && perf[g] >= (1.0 - tol) * pbest) cand.push_back({nb[g], ib[g]});
    }
  }
  // Step 2: shapes in ascending order of n (then m), PSPAYG between orders
  std::vector<int> order(nshapes);
  for (int i = 0; i < nshapes; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return std::tie(ns[a], ms[a]) < std::tie(ns[b], ms[b]); });
  std::vector<Entry> table;
  std::vector<std::pair<int, int>> surv = cand;
  std::vector<Sample> train;  // Step-2 timings of the orders done so far
  double step2_s = 0;
  int measured = 0, done = 0, squares_done = 0, fallbacks = 0;
  for (int oi : order) {
    const int64_t m = ms[oi], n = ns[oi];
    const size_t ns_ = surv.size();
    std::vector<double> perf(ns_, 0.0), sec(ns_, 0.0);
    std::vector<char> have(ns_, 0);
    auto measure = [&](size_t c) -> int {
      double med = 0, mn = 0;
      auto it = seen.find(LogKey{2, m, n, surv[c].first, surv[c].second, 1, budget});
      if (it != seen.end()) {
        med = it->second;
      } else {
        const auto t0 = std::chrono::steady_clock::now();
        int rc = qr_time_factor(m, n, surv[c].first, surv[c].second, prec, reps, &med, &mn, fwork, fbytes, stream);
        if (rc) return rc;
        step2_s += since(t0);
        append_log(log_path, 2, m, n, surv[c].first, surv[c].second, med, mn, reps, 1, budget);
        ++measured;
      }
      sec[c] = med;
      perf[c] = qr_flops_d(m, n) / med / 1e9;
      have[c] = 1;
      train.push_back(Sample{m, n, surv[c].first, surv[c].second, med});
      return 0;
    };
    // With the model (use_model = k > 0, PSPAYG, square orders from the
    // third square order on): fit it to the timings so far, rank the
    // survivors by predicted time and measure the k best; keep going down the
    // ranking while the last one measured is the fastest so far, and measure
    // every survivor when the model's relative predictions are off: the
    // ratio measured / predicted of a timed pair differs from that of the
    // top-ranked pair by more than the trust margin (the model ranks; the
    // overall scale of an extrapolation to a larger order may drift).
    const bool guided = use_model > 0 && !exhaustive && m == n && squares_done >= 2 && (int)ns_ > use_model &&
                        train.size() >= 4;
    if (!guided) {
      for (size_t c = 0; c < ns_; ++c)
        if (int rc = measure(c)) return rc;
    } else {
      const auto t0 = std::chrono::steady_clock::now();
      Model md;
      std::vector<double> pred;
      int rc = model_fit(train, cand, mwork, st, &md);
      if (!rc) rc = model_predict(md, m, n, surv, mwork, st, &pred);
      if (rc) return rc;
      model_s += since(t0);
      for (size_t c = 0; c < ns_; ++c)
        append_log(log_path, 4, m, n, surv[c].first, surv[c].second, pred[c], pred[c], 0, 1, budget);
      std::vector<size_t> rank(ns_);
      for (size_t c = 0; c < ns_; ++c) rank[c] = c;
      std::stable_sort(rank.begin(), rank.end(), [&](size_t a, size_t b) { return pred[a] < pred[b]; });
      size_t r = 0;
      for (; r < (size_t)use_model; ++r)
        if (int rc2 = measure(rank[r])) return rc2;
      auto fastest = [&]() {
        size_t b = rank[0];
        for (size_t q = 0; q < r; ++q)
          if (sec[rank[q]] < sec[b]) b = rank[q];
        return b;
      };
      while (r < ns_ && fastest() == rank[r - 1])
        if (int rc2 = measure(rank[r++])) return rc2;
      bool trusted = true;
      const double scale = std::log(sec[rank[0]]) - std::log(pred[rank[0]]);
      for (size_t q = 1; q < r; ++q)
        if (std::fabs(std::log(sec[rank[q]]) - std::log(pred[rank[q]]) - scale) > kModelTrust) trusted = false;
      if (!trusted) {
        ++fallbacks;
        for (; r < ns_; ++r)
          if (int rc2 = measure(rank[r])) return rc2;
      }
    }
    size_t bi = ns_;
    for (size_t c = 0; c < ns_; ++c)
      if (have[c] && (bi == ns_ || perf[c] > perf[bi] || (perf[c] == perf[bi] && surv[c].first < surv[bi].first)))
        bi = c;
    Entry ent{m, n, surv[bi].first, surv[bi].second, perf[bi], 1, budget};
    // the paper's third tunable for tall-skinny matrices: the number of
    // panel domains, swept in powers of two with the chosen (NB, IB)
    const int64_t MTs = (m + ent.nb - 1) / ent.nb, NTs = (n + ent.nb - 1) / ent.nb;
    if (m >= 4 * n && MTs >= 4)
      for (int pd = 2; pd <= 64 && pd <= MTs / std::max<int64_t>(NTs, 1) * 2 && pd <= MTs; pd *= 2) {
        double med = 0, mn = 0;
        auto it = seen.find(LogKey{3, m, n, ent.nb, ent.ib, pd, budget});
        if (it != seen.end()) {
          med = it->second;
        } else {
          const auto t0 = std::chrono::steady_clock::now();
          int rc = qr_time_factor_p(m, n, ent.nb, ent.ib, pd, prec, reps, &med, &mn, fwork, fbytes, stream);
          if (rc) return rc;
          step2_s += since(t0);
          append_log(log_path, 3, m, n, ent.nb, ent.ib, med, mn, reps, pd, budget);
          ++measured;
        }
        const double g = qr_flops_d(m, n) / med / 1e9;
        if (g > ent.gflops) {
          ent.gflops = g;
          ent.p = pd;
        }
      }
    table.push_back(ent);
    if (!exhaustive && m == n) {  // prune as you go along the square orders
      // Property 6.1 among the pairs measured at this order; a survivor the
      // model left unmeasured is kept
      std::vector<int> nbv, keep;
      std::vector<double> pv;
      std::vector<size_t> idx;
      for (size_t c = 0; c < ns_; ++c)
        if (have[c]) {
          nbv.push_back(surv[c].first);
          pv.push_back(perf[c]);
          idx.push_back(c);
        }
      keep.resize(nbv.size());
      qr_tune_payg((int)nbv.size(), nbv.data(), pv.data(), keep.data());
      std::vector<char> drop(ns_, 0);
      for (size_t q = 0; q < idx.size(); ++q)
        if (!keep[q]) drop[idx[q]] = 1;
      std::vector<std::pair<int, int>> nx;
      for (size_t c = 0; c < ns_; ++c)
        if (!drop[c]) nx.push_back(surv[c]);
      surv = nx;
    }
    ++done;
    if (m == n) ++squares_done;
  }
  // the final model, fitted to every Step-2 timing, proposes pairs for
  // untuned shapes (qr_model_propose) and is saved with the table
  Model final_model;
  if (use_model > 0 && train.size() >= 4) {
    const auto t0 = std::chrono::steady_clock::now();
    int rc = model_fit(train, cand, mwork, st, &final_model);
    if (rc) return rc;
    model_s += since(t0);
  }
  const double total = since(t_start);
  if (seconds_out) {
    seconds_out[0] = total;
    seconds_out[1] = step1_s;
    seconds_out[2] = step2_s;
    seconds_out[3] = (double)measured;
    seconds_out[4] = model_s;
    seconds_out[5] = (double)fallbacks;
  }
  {
    std::lock_guard<std::mutex> lock(g_tmu);
    g_table[prec == QR_PREC_F32 ? 1 : 0] = table;
    g_model[prec == QR_PREC_F32 ? 1 : 0] = final_model;
  }
  if (table_path && table_path[0]) {
    char extra[768];
    snprintf(extra, sizeof(extra),
             "  \"heuristic\": %d,\n  \"mode\": \"%s\",\n  \"step1\": \"%s\",\n  \"use_model\": %d,\n"
             "  \"reps\": %d,\n  \"seconds\": %.3f,\n  \"step1_seconds\": %.3f,\n  \"step2_seconds\": %.3f,\n"
             "  \"model_seconds\": %.3f,\n  \"factorizations_timed\": %d,\n  \"model_fallbacks\": %d,\n"
             "  \"ib_tol_permille\": %d,\n",
             heuristic, exhaustive ? "exhaustive" : "pspayg", flush ? "multcallflushlru" : "noflush", use_model,
             reps, total, step1_s, step2_s, model_s, measured, fallbacks, (int)qr_get_option(QR_OPT_TUNE_IB_TOL));
    std::string ex = extra;
    if (final_model.ok) ex += model_json(final_model);
    if (!write_table(table_path, prec == QR_PREC_F32 ? 1 : 0, table, ex)) return -9;
  }
  return 0;
}

}  // extern "C"
