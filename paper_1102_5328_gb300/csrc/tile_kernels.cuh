// Device building blocks of the tile Householder QR (flat tree).
//
// The four tile kernels the paper builds its QR from (Sec. 2.1): GEQRT (QR of
// a diagonal tile), TSQRT (QR of a triangle stacked on a square tile), UNMQR
// (the paper's DLARFB: apply GEQRT's Q^T to a tile to its right) and TSMQR
// (the paper's DSSRFB: apply TSQRT's Q^T to a pair of tiles). Inner blocking
// IB (Sec. 2.2) groups the reflectors of a tile into blocks of IB whose
// product is I - V T V^T with T upper triangular (compact WY form).
//
// Execution model: one CTA of NTHREADS threads runs one task. FP64 on this
// GPU issues roughly 2 fused multiply-adds per clock per SM, so every kernel
// is bound by the FP64 pipe, not by memory: the code spends shared memory and
// registers freely to keep that pipe fed and to avoid non-FMA FP64 work.
//
// Memory discipline inside the persistent scheduler: any tile another CTA may
// have written is read with ld.global.cg (L2, bypassing the non-coherent L1)
// and written with st.global.cg, so no SM ever consumes a stale L1 line.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tileqr.h"

namespace tqr {

constexpr int NTHREADS = 256;
constexpr int RPT = 32;          // rows of C held in registers per thread (apply)
constexpr int VS_CAP = 4096;     // elements of the staged V panel
constexpr int PG = 8;            // reflectors per partial-sum group (apply)
constexpr int PART_CAP = PG * NTHREADS;
constexpr int W_CAP = 4096;      // elements of W = T^T V^T C for one chunk
constexpr int PANEL_CAP = PART_CAP + W_CAP;  // level-2 sub-panel (aliases part + W): 6144
constexpr int TS_CAP = 1024;     // sub-block T (<= 32 x 32)
constexpr int RED_CAP = 64;

// Shared-memory carve-up (in elements of S) used by every task.
template <typename S>
struct Smem {
  S* vs;     // [VS_CAP]
  S* part;   // [PART_CAP]
  S* w;      // [W_CAP]
  S* ts;     // [TS_CAP]
  S* red;    // [RED_CAP]
  S* tau;    // [512]
  S* rs;     // [TS_CAP] R sub-block (TSQRT level-2)
};

template <typename S>
__host__ __device__ constexpr size_t smem_elems() {
  return (size_t)VS_CAP + PART_CAP + W_CAP + TS_CAP + RED_CAP + 512 + TS_CAP;
}

template <typename S>
__device__ __forceinline__ Smem<S> carve(S* base) {
  Smem<S> s;
  s.vs = base;
  s.part = s.vs + VS_CAP;
  s.w = s.part + PART_CAP;
  s.ts = s.w + W_CAP;
  s.red = s.ts + TS_CAP;
  s.tau = s.red + RED_CAP;
  s.rs = s.tau + 512;
  return s;
}

// ---------------------------------------------------------------------------
// coherent (L2) global access helpers
template <typename S>
__device__ __forceinline__ S ldg(const S* p) { return __ldcg(p); }
template <typename S>
__device__ __forceinline__ void stg(S* p, S v) { __stcg(p, v); }
// a pointer that may be shared (generic) or global (L2-coherent path)
template <typename S>
__device__ __forceinline__ S ldx(const S* p, bool sm) { return sm ? *p : __ldcg(p); }
template <typename S>
__device__ __forceinline__ void stx(S* p, S v, bool sm) {
  if (sm) *p = v; else __stcg(p, v);
}

// Copy of a rows x cols column-major block from global memory (ld lds,
// L2-coherent loads) into shared memory (ld ldd). Each thread issues U loads
// before its first store, so a thread has U global loads in flight instead
// of one load-store round trip per element. Element (r, c) is read only if
// rd(r, c) (else taken as 0); f(r, c, v) gives the value stored (masks such
// as the unit diagonal).
template <int U, typename S, typename R, typename F>
__device__ __forceinline__ void stage_block(S* dst, int ldd, const S* src, int64_t lds, int rows, int cols, R rd,
                                            F f) {
  const int total = rows * cols;
  for (int base = threadIdx.x; base < total; base += U * NTHREADS) {
    S v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * NTHREADS;
      v[u] = S(0);
      if (idx < total) {
        const int c = idx / rows, r = idx - c * rows;
        if (rd(r, c)) v[u] = __ldcg(src + r + (size_t)c * lds);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int idx = base + u * NTHREADS;
      if (idx < total) {
        const int c = idx / rows, r = idx - c * rows;
        dst[r + (size_t)c * ldd] = f(r, c, v[u]);
      }
    }
  }
}
struct AllRd {
  __device__ bool operator()(int, int) const { return true; }
};
struct Ident {
  template <typename S>
  __device__ S operator()(int, int, S v) const { return v; }
};

template <typename S>
__device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA-wide sum; every thread gets the result. Uses red[0..NTHREADS/32].
template <typename S>
__device__ __forceinline__ S cta_sum(S v, S* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  S t = (threadIdx.x < NTHREADS / 32) ? red[threadIdx.x] : S(0);
  if (wid == 0) {
    t = warp_sum(t);
    if (lane == 0) red[NTHREADS / 32] = t;
  }
  __syncthreads();
  return red[NTHREADS / 32];
}

// Reflectors pc0 .. pc0+pb-1 of a tile V (ld ldv), rows r0 .. r0+nr-1, into
// buf (ld nr) with their masks (GE: zero above the diagonal, unit diagonal;
// TS tri: zero below it); zero past `rows`. GE: four loads in flight per
// thread. TS: one (its later blocks come through the cp.async prefetch of
// apply_qt, and the TS update keeps more registers live).
// TS with use_async (no triangle mask, V and ldv 16-byte aligned): 16-byte
// cp.async copies, zero-filled past `rows`, all in flight at once; the
// caller issues cp.async.wait_all before the barrier that publishes them.
template <typename S, bool TS>
__device__ __forceinline__ void stage_refl(S* buf, const S* V, int ldv, int nr, int r0, int rows, int pc0, int pb,
                                           bool tri, bool use_async = false) {
  if constexpr (TS) {
    if (use_async) {
      constexpr int EPC = 16 / sizeof(S);
      const int half = nr / EPC;  // nr is a multiple of 32, so of EPC
      for (int idx = threadIdx.x; idx < pb * half; idx += NTHREADS) {
        const int p = idx / half, rl = EPC * (idx - (idx / half) * half), r = rl + r0;
        const int valid = r < rows ? min(EPC, rows - r) * (int)sizeof(S) : 0;
        const S* src = V + (valid ? r + (size_t)(pc0 + p) * ldv : 0);
        const unsigned dst = (unsigned)__cvta_generic_to_shared(buf + p * nr + rl);
        const size_t gsrc = __cvta_generic_to_global(src);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(gsrc), "r"(valid) : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      return;  // the caller waits (cp.async.wait_all) before its barrier
    }
    for (int idx = threadIdx.x; idx < pb * nr; idx += NTHREADS) {
      const int p = idx / nr, rl = idx - (idx / nr) * nr;
      const int r = rl + r0, pc = pc0 + p;
      S v = S(0);
      if (r < rows) v = (tri && r > pc) ? S(0) : ldg(V + r + (size_t)pc * ldv);
      buf[p * nr + rl] = v;
    }
  } else {
    stage_block<4>(buf, nr, V + r0 + (size_t)pc0 * ldv, ldv, nr, pb,
                   [=](int rl, int p) { return rl + r0 < rows && rl + r0 > pc0 + p; },
                   [=](int rl, int p, S v) { return rl + r0 == pc0 + p ? S(1) : v; });
  }
}

// ---------------------------------------------------------------------------
// Apply Q_l^T of blocks of reflectors to a range of columns.
//
// GE mode (UNMQR; trailing update inside GEQRT): reflector p of a block that
// starts at row/column l0 is v_p = [0 (rows < l0+p); 1; V(l0+p+1:rows, l0+p)]
// from the tile V; C is one tile whose rows [0, rows) all live in registers.
// TS mode (TSMQR; trailing update inside TSQRT): reflector p is
// [e_{l0+p} (top tile); V(0:rows, l0+p) (bottom tile)], Ctop is the top tile
// and C the bottom tile.
// For each block of ib reflectors: W = Vfull^T Cstack, W <- T_l^T W,
// Cstack -= Vfull W, with T_l the upper-triangular ib x ib factor stored at
// T + l0*ldt (element (q, p) at T[q + (l0+p)*ldt]).
// Blocks run from l0 = lstart to lend in steps of IB.
//
// Thread layout: C's column chunk of width cw is split in G = ceil(rows/RPT)
// row groups; thread (g, c) keeps C(g*RPT : g*RPT+RPT, c) in registers for
// all blocks, so C is read and written once per task.
//
// TR = true applies Q^T (blocks in ascending order, W <- T^T W); TR = false
// applies Q (blocks in descending order, W <- T W).
//
// tri (TS mode only): the bottom reflectors are upper triangular -- the
// triangle-on-triangle case of a tree reduction (TTQRT/TTMQR): V(r, c) is
// taken as zero for r > c, whatever the tile holds there.
template <typename S, bool TS, bool TR = true>
__device__ void apply_qt(const S* __restrict__ V, int ldv, const S* T, int ldt, bool t_smem,
                         int lstart, int lend, int IB, S* Ctop, int ldct, S* C, int ldc, int rows,
                         int c0, int c1, const Smem<S>& sm, bool tri = false) {
  if (c1 <= c0 || lend <= lstart || rows <= 0) return;
  const int tid = threadIdx.x;
  const int G = (rows + RPT - 1) / RPT;
  const int ibmax = min(IB, lend - lstart);
  const int cwmax = min(NTHREADS / G, W_CAP / ibmax);
  const int nchunks = (c1 - c0 + cwmax - 1) / cwmax;
  const int per = (c1 - c0 + nchunks - 1) / nchunks;
  const int nblk = (lend - lstart + IB - 1) / IB;
  // TS blocks whose reflectors fit one staging buffer are double-buffered:
  // while the CTA updates C with block b, cp.async copies block b+1's
  // reflectors into the other buffer (vs and part swap the roles of V stage
  // and partial-sum buffer) and each thread holds part of b+1's T in a
  // register. 16-byte copies need a leading dimension that is a multiple of
  // 16 bytes and a 16-byte aligned V.
  constexpr int EPC = 16 / sizeof(S);  // elements per 16-byte copy
  const bool can_pipe = TS && !tri && (ldv % EPC == 0) && ((reinterpret_cast<uintptr_t>(V) & 15) == 0);
  for (int cs = c0; cs < c1; cs += per) {
    const int cw = min(per, c1 - cs);
    const int g = tid / cw, c = tid - (tid / cw) * cw;
    const bool act = g < G;
    S creg[RPT];
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int r = g * RPT + rr;
      creg[rr] = (act && r < rows) ? ldg(C + r + (size_t)(cs + c) * ldc) : S(0);
    }
    int tsel = 0;           // which half of ts holds the current block's T (t_in_ts)
    int vcur = 0;           // which buffer holds the current block's V (0: vs, 1: part)
    bool staged = false;    // current block's V (and T in ts) already in place
    for (int bi = 0; bi < nblk; ++bi) {
      const int l0 = lstart + (TR ? bi : nblk - 1 - bi) * IB;
      const int ib = min(IB, lend - l0);
      // rows below rlo_al are untouched by this block (GE); whole groups skip
      const int rlo = TS ? 0 : l0;
      const int glo = rlo / RPT;
      const int rlo_al = glo * RPT;
      // triangle-on-triangle: this block's reflectors stop at row l0+ib-1, so
      // the row groups below take no part in it
      const int ghi = (TS && tri) ? min(G, (min(rows, l0 + ib) + RPT - 1) / RPT) : G;
      const int nr = ghi * RPT - rlo_al;  // staged rows, zero-padded past `rows`
      S* vbuf = vcur ? sm.part : sm.vs;
      S* pbuf = vcur ? sm.vs : sm.part;
      const int vcap = vcur ? PART_CAP : VS_CAP;
      int PB = vcap / nr;
      if (PB > ib) PB = ib;
      if (PB < 1) PB = 1;
      const bool myrows = act && g >= glo && g < ghi;
      // T_l in shared memory: half tsel of ts (tsel = 1 only after a T
      // prefetch, which needs ib * ib <= NTHREADS, so the block fits there)
      const bool t_in_ts = !t_smem && ib * ib <= TS_CAP;
      // --- phase A: W = Vfull^T Cstack, V staged PB reflectors at a time
      for (int pp0 = 0; pp0 < ib; pp0 += PB) {
        const int pb = min(PB, ib - pp0);
        if (!staged) {
          __syncthreads();
          stage_refl<S, TS>(vbuf, V, ldv, nr, rlo_al, rows, l0 + pp0, pb, tri, can_pipe);
          if (pp0 == 0 && t_in_ts)
            for (int idx = tid; idx < ib * ib; idx += NTHREADS) {
              const int p = idx / ib, q = idx - (idx / ib) * ib;
              sm.ts[tsel * (TS_CAP / 2) + idx] = (q <= p) ? ldg(T + q + (size_t)(l0 + p) * ldt) : S(0);
            }
          asm volatile("cp.async.wait_all;" ::: "memory");
          __syncthreads();
        }
        for (int pg0 = 0; pg0 < pb; pg0 += PG) {
          const int pgc = min(PG, pb - pg0);
          if (myrows) {
            S acc[PG];
#pragma unroll
            for (int q = 0; q < PG; ++q) acc[q] = S(0);
            const S* vrow = vbuf + (size_t)pg0 * nr + (g * RPT - rlo_al);
            if constexpr (sizeof(S) == 4) {
              // FP32: 16-byte shared loads (4 rows of a reflector) feed 4
              // FMAs each; vbuf, nr and the row offset are multiples of 4
              // elements, and the summation order per reflector is unchanged
#pragma unroll
              for (int r4 = 0; r4 < RPT; r4 += 4) {
#pragma unroll
                for (int q = 0; q < PG; ++q)
                  if (q < pgc) {
                    const float4 v = *reinterpret_cast<const float4*>(vrow + q * nr + r4);
                    acc[q] = fma(v.x, creg[r4], acc[q]);
                    acc[q] = fma(v.y, creg[r4 + 1], acc[q]);
                    acc[q] = fma(v.z, creg[r4 + 2], acc[q]);
                    acc[q] = fma(v.w, creg[r4 + 3], acc[q]);
                  }
              }
            } else {
#pragma unroll
              for (int rr = 0; rr < RPT; ++rr) {
                const S cv = creg[rr];
#pragma unroll
                for (int q = 0; q < PG; ++q)
                  if (q < pgc) acc[q] = fma(vrow[q * nr + rr], cv, acc[q]);
              }
            }
#pragma unroll
            for (int q = 0; q < PG; ++q)
              if (q < pgc) pbuf[(q * G + g) * cw + c] = acc[q];
          }
          __syncthreads();
          // two outputs per thread per pass, both top-row loads issued
          // before either sum (one L2 round trip instead of two)
          for (int o = tid; o < pgc * cw; o += 2 * NTHREADS) {
            const int o2 = o + NTHREADS;
            const bool two = o2 < pgc * cw;
            const int q = o / cw, cc = o - (o / cw) * cw;
            const int q2 = two ? o2 / cw : q, cc2 = two ? o2 - (o2 / cw) * cw : cc;
            S s = TS ? ldg(Ctop + (l0 + pp0 + pg0 + q) + (size_t)(cs + cc) * ldct) : S(0);
            S s2 = (TS && two) ? ldg(Ctop + (l0 + pp0 + pg0 + q2) + (size_t)(cs + cc2) * ldct) : S(0);
            for (int gg = glo; gg < ghi; ++gg) s += pbuf[(q * G + gg) * cw + cc];
            sm.w[(pp0 + pg0 + q) * cw + cc] = s;
            if (two) {
              for (int gg = glo; gg < ghi; ++gg) s2 += pbuf[(q2 * G + gg) * cw + cc2];
              sm.w[(pp0 + pg0 + q2) * cw + cc2] = s2;
            }
          }
          __syncthreads();
        }
      }
      // --- phase B: W <- T_l^T W (Q^T) or T_l W (Q); TS: Ctop rows -= W
      {
        const S* Tb = t_in_ts ? sm.ts + tsel * (TS_CAP / 2) : T + (size_t)l0 * ldt;  // (q, p) at Tb[q + p * ldtb]
        const int ldtb = t_in_ts ? ib : ldt;
        const bool tsm = t_in_ts || t_smem;
        // ib * cw <= W_CAP = 16 * NTHREADS: at most 16 outputs per thread,
        // held in registers (compile-time indices) until every read of W is done
        S wq[16];
        S cold[4];  // TS: the first four outputs' top rows, loaded before the barrier
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int o = tid + u * NTHREADS;
          S s = S(0);
          if (u < 4) cold[u] = S(0);
          if (o < ib * cw) {
            const int p = o / cw, cc = o - (o / cw) * cw;
            if (TS && u < 4) cold[u] = ldg(Ctop + (l0 + p) + (size_t)(cs + cc) * ldct);
            if (TR) {
              const S* tcol = Tb + (size_t)p * ldtb;
              for (int q = 0; q <= p; ++q) s = fma(ldx(tcol + q, tsm), sm.w[q * cw + cc], s);
            } else {
              const S* trow = Tb + p;
              for (int q = p; q < ib; ++q) s = fma(ldx(trow + (size_t)q * ldtb, tsm), sm.w[q * cw + cc], s);
            }
          }
          wq[u] = s;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int o = tid + u * NTHREADS;
          if (o < ib * cw) {
            const int p = o / cw, cc = o - (o / cw) * cw;
            sm.w[p * cw + cc] = wq[u];
            if (TS) {
              S* pt = Ctop + (l0 + p) + (size_t)(cs + cc) * ldct;
              stg(pt, (u < 4 ? cold[u < 4 ? u : 0] : ldg(pt)) - wq[u]);
            }
          }
        }
        __syncthreads();
      }
      // --- prefetch of the next block (TS, single stage in the other buffer)
      bool pre = false;
      S tpre = S(0);
      int ibn = 0, l0n = 0;
      if (can_pipe && bi + 1 < nblk && PB == ib) {
        l0n = lstart + (TR ? bi + 1 : nblk - 2 - bi) * IB;
        ibn = min(IB, lend - l0n);
        const int ocap = vcur ? VS_CAP : PART_CAP;
        if (ibn * nr <= ocap && (t_smem || ibn * ibn <= NTHREADS)) {  // one T element per thread
          pre = true;
          S* nbuf = vcur ? sm.vs : sm.part;
          const int half = nr / EPC;  // nr is a multiple of 32, so of EPC
          for (int idx = tid; idx < ibn * half; idx += NTHREADS) {
            const int p = idx / half, r = EPC * (idx - (idx / half) * half);
            const int valid = r < rows ? min(EPC, rows - r) * (int)sizeof(S) : 0;
            const S* src = V + (valid ? r + (size_t)(l0n + p) * ldv : 0);
            const unsigned dst = (unsigned)__cvta_generic_to_shared(nbuf + p * nr + r);
            const size_t gsrc = __cvta_generic_to_global(src);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(gsrc), "r"(valid) : "memory");
          }
          asm volatile("cp.async.commit_group;" ::: "memory");
          if (!t_smem && tid < ibn * ibn) {
            const int p = tid / ibn, q = tid - (tid / ibn) * ibn;
            tpre = (q <= p) ? ldg(T + q + (size_t)(l0n + p) * ldt) : S(0);
          }
        }
      }
      // --- phase C: Cstack -= Vfull W (restage V if it did not fit at once)
      for (int pp0 = 0; pp0 < ib; pp0 += PB) {
        const int pb = min(PB, ib - pp0);
        if (PB < ib) {
          __syncthreads();
          stage_refl<S, TS>(vbuf, V, ldv, nr, rlo_al, rows, l0 + pp0, pb, tri, can_pipe);
          asm volatile("cp.async.wait_all;" ::: "memory");
          __syncthreads();
        }
        if (myrows) {
          const S* vrow = vbuf + (g * RPT - rlo_al);
          for (int p = 0; p < pb; ++p) {
            const S wv = sm.w[(pp0 + p) * cw + c];
            const S* vp = vrow + (size_t)p * nr;
            if constexpr (sizeof(S) == 4) {
#pragma unroll
              for (int r4 = 0; r4 < RPT; r4 += 4) {
                const float4 v = *reinterpret_cast<const float4*>(vp + r4);
                creg[r4] = fma(-v.x, wv, creg[r4]);
                creg[r4 + 1] = fma(-v.y, wv, creg[r4 + 1]);
                creg[r4 + 2] = fma(-v.z, wv, creg[r4 + 2]);
                creg[r4 + 3] = fma(-v.w, wv, creg[r4 + 3]);
              }
            } else {
#pragma unroll
              for (int rr = 0; rr < RPT; ++rr) creg[rr] = fma(-vp[rr], wv, creg[rr]);
            }
          }
        }
      }
      if (pre) {
        // the next T goes to the other half of ts (phase C reads neither),
        // so one barrier publishes it together with the copied reflectors
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (!t_smem && tid < ibn * ibn) sm.ts[(tsel ^ 1) * (TS_CAP / 2) + tid] = tpre;
        tsel ^= 1;
        vcur ^= 1;
        staged = true;
        __syncthreads();
      } else {
        staged = false;
        __syncthreads();
      }
    }
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int r = g * RPT + rr;
      if (act && r < rows) stg(C + r + (size_t)(cs + c) * ldc, creg[rr]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Narrow update (few columns of C: the Q^T b / Q h products of a
// least-squares solve). A TSMQR/UNMQR task on a handful of columns is pure
// latency in apply_qt (a staging round trip and several barriers per inner
// block), so here the whole reflector tile, its T factors and the touched
// rows of C are staged in shared memory once per task; each inner block then
// costs three barriers. Same operations as apply_qt (blocks in order, W =
// V^T C, W <- T^T W or T W, C -= V W), different summation order.
// Usable when narrow_fits(): rows * nref <= VS_CAP, IB * nref <= PART_CAP,
// ((rows | 1) + nref) * cw <= W_CAP, IB * cw <= min(TS_CAP, NTHREADS), cw <= 16.
__host__ __device__ inline bool narrow_fits(int rows, int nref, int IB, int cw) {
  return rows * nref <= VS_CAP && IB * nref <= PART_CAP && ((rows | 1) + nref) * cw <= W_CAP && IB * cw <= TS_CAP &&
         IB * cw <= NTHREADS && cw <= 16;
}

// The reflector tile and its T factors of an apply_narrow task into shared
// memory (sm.vs, sm.part). A caller whose V and T are final before the
// task's C rows are (the Q application after the factorization) issues this
// before waiting for C and passes vt_staged = true to apply_narrow. Ends
// without a barrier; the caller's barrier (or apply_narrow's) follows.
template <typename S, bool TS>
__device__ void narrow_stage_vt(const S* __restrict__ V, int ldv, const S* __restrict__ T, int ldt, int nref, int IB,
                                int rows, const Smem<S>& sm, bool tri = false) {
  // reflectors with their masks (TS tri: zero below the diagonal; GE: zero
  // above it, unit diagonal); every element read lies inside the tile
  if (TS)
    stage_block<16>(sm.vs, rows, V, ldv, rows, nref, [tri](int r, int c) { return !(tri && r > c); }, Ident());
  else
    stage_block<16>(sm.vs, rows, V, ldv, rows, nref, [](int r, int c) { return r > c; },
                    [](int r, int c, S v) { return r == c ? S(1) : v; });
  stage_block<8>(sm.part, IB, T, ldt, IB, nref, AllRd(), Ident());
}

template <typename S, bool TS, bool TR>
__device__ void apply_narrow(const S* __restrict__ V, int ldv, const S* __restrict__ T, int ldt, int nref, int IB,
                             S* Ctop, int ldct, S* C, int ldc, int rows, int c0, int c1, const Smem<S>& sm,
                             bool tri = false, bool vt_staged = false) {
  const int tid = threadIdx.x;
  const int cw = c1 - c0;
  if (cw <= 0 || nref <= 0 || rows <= 0) return;
  S* Vs = sm.vs;            // rows x nref, column-major (ld rows)
  S* Ts = sm.part;          // IB x nref (ld IB)
  // C (GE) or the bottom tile (TS), rows x cw with an odd leading dimension
  // so that the columns read together in phase A fall in different banks
  const int ldb = rows | 1;
  S* Cb = sm.w;             // rows x cw (ld ldb)
  S* Ct = sm.w + ldb * cw;  // nref x cw (ld nref): top rows (TS)
  S* Ws = sm.ts;            // IB x cw
  S* W2 = sm.ts + NTHREADS; // IB x cw (IB * cw <= NTHREADS), T applied
  __syncthreads();
  if (!vt_staged) narrow_stage_vt<S, TS>(V, ldv, T, ldt, nref, IB, rows, sm, tri);
  // the task's rows of C -- bottom tile (rows x cw) and, TS, top rows
  // (nref x cw) -- in one batch of loads
  {
    const int nbot = rows * cw, ntot = nbot + (TS ? nref * cw : 0);
    for (int base = tid; base < ntot; base += 4 * NTHREADS) {
      S v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + u * NTHREADS;
        v[u] = S(0);
        if (idx < nbot) {
          const int c = idx / rows, r = idx - c * rows;
          v[u] = __ldcg(C + r + (size_t)(c0 + c) * ldc);
        } else if (idx < ntot) {
          const int e = idx - nbot, c = e / nref, r = e - c * nref;
          v[u] = __ldcg(Ctop + r + (size_t)(c0 + c) * ldct);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + u * NTHREADS;
        if (idx < nbot) {
          const int c = idx / rows, r = idx - c * rows;
          Cb[r + c * ldb] = v[u];
        }
        else if (idx < ntot) Ct[idx - nbot] = v[u];
      }
    }
  }
  __syncthreads();
  const int nblk = (nref + IB - 1) / IB;
  for (int bi = 0; bi < nblk; ++bi) {
    const int l0 = (TR ? bi : nblk - 1 - bi) * IB;
    const int ib = min(IB, nref - l0);
    const int nout = ib * cw;
    // threads per output (a power of two dividing 32) for the row sums
    int tpo = NTHREADS / max(nout, 1);
    tpo = tpo >= 32 ? 32 : (tpo >= 16 ? 16 : (tpo >= 8 ? 8 : (tpo >= 4 ? 4 : (tpo >= 2 ? 2 : 1))));
    const int r0 = TS ? 0 : l0;  // GE: rows above the block are untouched
    // phase A: W(p, c) = Ctop(l0+p, c) [TS] + sum_r V(r, l0+p) Cb(r, c)
    for (int base = 0; base < nout * tpo; base += NTHREADS) {
      const int gid = base + tid;
      const int o = gid / tpo, part = gid - (gid / tpo) * tpo;
      S acc = S(0);
      if (o < nout) {
        const int pp = o / cw, c = o - (o / cw) * cw;
        const S* vcol = Vs + (size_t)(l0 + pp) * rows;
        const S* ccol = Cb + (size_t)c * ldb;
        // four independent partial sums (rows r, r+tpo, r+2tpo, r+3tpo)
        S a1 = S(0), a2 = S(0), a3 = S(0);
        int r = r0 + part;
        for (; r + 3 * tpo < rows; r += 4 * tpo) {
          acc = fma(vcol[r], ccol[r], acc);
          a1 = fma(vcol[r + tpo], ccol[r + tpo], a1);
          a2 = fma(vcol[r + 2 * tpo], ccol[r + 2 * tpo], a2);
          a3 = fma(vcol[r + 3 * tpo], ccol[r + 3 * tpo], a3);
        }
        for (; r < rows; r += tpo) acc = fma(vcol[r], ccol[r], acc);
        acc = (acc + a1) + (a2 + a3);
      }
      for (int off = tpo / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (o < nout && part == 0) {
        const int pp = o / cw, c = o - (o / cw) * cw;
        if (TS) acc += Ct[(l0 + pp) + (size_t)c * nref];
        Ws[pp * cw + c] = acc;
      }
    }
    __syncthreads();
    // phase B: W <- T^T W (Q^T) or T W (Q), one output per thread
    S wv = S(0);
    int po = -1, co = 0;
    if (tid < nout) {
      po = tid / cw;
      co = tid - po * cw;
      const S* Tb = Ts + (size_t)l0 * IB;  // (q, p) at Tb[q + p * IB]
      if (TR) {
        for (int q = 0; q <= po; ++q) wv = fma(Tb[q + po * IB], Ws[q * cw + co], wv);
      } else {
        for (int q = po; q < ib; ++q) wv = fma(Tb[po + q * IB], Ws[q * cw + co], wv);
      }
    }
    if (po >= 0) W2[po * cw + co] = wv;  // a second buffer: no barrier between the reads of Ws and this write
    __syncthreads();
    // phase C: Ctop(l0+p) -= W (TS); Cb(r) -= sum_p V(r, l0+p) W(p)
    if (TS)
      for (int o = tid; o < nout; o += NTHREADS) {
        const int pp = o / cw, c = o - (o / cw) * cw;
        Ct[(l0 + pp) + (size_t)c * nref] -= W2[pp * cw + c];
      }
    // two outputs per thread interleaved (independent chains)
    const int nrr = rows - r0, nco = nrr * cw;
    for (int o = tid; o < nco; o += 2 * NTHREADS) {
      const int o2 = o + NTHREADS;
      const bool two = o2 < nco;
      const int c = o / nrr, r = r0 + (o - c * nrr);
      const int c2 = two ? o2 / nrr : c, r2 = two ? r0 + (o2 - c2 * nrr) : r;
      S acc = Cb[r + (size_t)c * ldb];
      S acc2 = Cb[r2 + (size_t)c2 * ldb];
      for (int pp = 0; pp < ib; ++pp) {
        acc = fma(-Vs[r + (size_t)(l0 + pp) * rows], W2[pp * cw + c], acc);
        acc2 = fma(-Vs[r2 + (size_t)(l0 + pp) * rows], W2[pp * cw + c2], acc2);
      }
      Cb[r + (size_t)c * ldb] = acc;
      if (two) Cb[r2 + (size_t)c2 * ldb] = acc2;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < rows * cw; idx += NTHREADS) {
    const int c = idx / rows, r = idx - (idx / rows) * rows;
    stg(C + r + (size_t)(c0 + c) * ldc, Cb[r + c * ldb]);
  }
  if (TS)
    for (int idx = tid; idx < nref * cw; idx += NTHREADS) {
      const int c = idx / nref, r = idx - (idx / nref) * nref;
      stg(Ctop + r + (size_t)(c0 + c) * ldct, Ct[idx]);
    }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// T factor of a block of ncol reflectors (LAPACK's forward, columnwise
// recurrence): T(p,p) = tau_p, T(0:p,p) = -tau_p T(0:p,0:p) (V^T v_p)(0:p).
// V(r, q) for r in [0, nr): GE: unit at r = q, zero above (rows relative to
// the block's first row); TS: full column (the stacked identity part is
// orthogonal between reflectors and drops out of V^T V).
// tri_off >= 0 (TS only): column q of V is zero below row tri_off + q
// (triangle-on-triangle reflectors).
template <typename S, bool TS>
__device__ void build_t(const S* V, int ldv, bool v_smem, int nr, int ncol, const S* tau, S* Tout,
                        int ldt, bool t_smem, int tri_off = -1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // Gram entries z(q,p), q < p, into T's strict upper triangle
  const int npairs = ncol * (ncol - 1) / 2;
  for (int pr = wid; pr < npairs; pr += NTHREADS / 32) {
    // decode pair index -> (q, p) with q < p (column-major over p)
    int p = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)pr)) * 0.5f);
    while (p * (p - 1) / 2 > pr) --p;
    while ((p + 1) * p / 2 <= pr) ++p;
    const int q = pr - p * (p - 1) / 2;
    S s = S(0);
    const int r0 = TS ? 0 : p + 1;
    const int rend = (TS && tri_off >= 0) ? min(nr, tri_off + q + 1) : nr;
    for (int r = r0 + lane; r < rend; r += 32)
      s = fma(ldx(V + r + (size_t)q * ldv, v_smem), ldx(V + r + (size_t)p * ldv, v_smem), s);
    s = warp_sum(s);
    if (lane == 0) {
      if (!TS) s += ldx(V + p + (size_t)q * ldv, v_smem);
      stx(Tout + q + (size_t)p * ldt, s, t_smem);
    }
  }
  for (int p = threadIdx.x; p < ncol; p += NTHREADS) stx(Tout + p + (size_t)p * ldt, tau[p], t_smem);
  __syncthreads();
  if (ncol <= 32) {
    // one warp, lane q owns row q of T; no CTA-wide barrier per column
    if (wid == 0) {
      for (int p = 1; p < ncol; ++p) {
        const S tp = tau[p];
        S t = S(0);
        if (lane < p && tp != S(0))
          for (int s2 = lane; s2 < p; ++s2)
            t = fma(ldx(Tout + lane + (size_t)s2 * ldt, t_smem), ldx(Tout + s2 + (size_t)p * ldt, t_smem), t);
        __syncwarp();
        if (lane < p) stx(Tout + lane + (size_t)p * ldt, -tp * t, t_smem);
        __syncwarp();
      }
    }
    __syncthreads();
    return;
  }
  for (int p = 1; p < ncol; ++p) {
    const S tp = tau[p];
    S t = S(0);
    const int q = threadIdx.x;
    if (q < p && tp != S(0)) {
      for (int s2 = q; s2 < p; ++s2)
        t = fma(ldx(Tout + q + (size_t)s2 * ldt, t_smem), ldx(Tout + s2 + (size_t)p * ldt, t_smem), t);
    }
    __syncthreads();
    if (q < p) stx(Tout + q + (size_t)p * ldt, -tp * t, t_smem);
    __syncthreads();
  }
}
// (ncol <= NTHREADS is required by the recurrence above: IB <= 256.)

// ---------------------------------------------------------------------------
// Level-2 Householder QR of a sub-panel held in shared memory.
// GE: P(nr x w), column jj has its pivot at row jj, x = P(jj+1:nr, jj).
// TS: pivot R(jj, jj) in Rs (w x w, upper), x = P(0:nr, jj), the update
//     touches Rs(jj, c) and P(:, c).
// Writes tau[0..w) and reports a non-finite norm through *bad.
//
// The norm, beta, tau and the scaling are always formed in FP64 (for the
// FP32 working precision too: the Householder vector / tau generation is the
// one place the mixed-precision path keeps FP64); the rank-1 updates run in S.
template <typename S, bool TS>
__device__ void panel_l2(S* P, int ldp, int nr, int w, S* Rs, int ldr, S* tau, S* red, int* bad,
                         int tri_off = -1) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nr_all = nr;
  for (int jj = 0; jj < w; ++jj) {
    const int x0 = TS ? 0 : jj + 1;
    // triangle-on-triangle: column jj of the bottom block has rows 0..tri_off+jj
    nr = (TS && tri_off >= 0) ? min(nr_all, tri_off + jj + 1) : nr_all;
    S* col = P + (size_t)jj * ldp;
    // warp 0 forms the reflector: norm, beta, tau, scaling of x
    if (wid == 0) {
      double s = 0.0;
      for (int r = x0 + lane; r < nr; r += 32) {
        const double v = (double)col[r];
        s = fma(v, v, s);
      }
      s = warp_sum(s);
      S* piv = TS ? (Rs + jj + (size_t)jj * ldr) : (col + jj);
      double tau_j = 0.0, scal = 0.0;
      if (lane == 0) {
        const double a = (double)*piv;
        if (!isfinite(s) || !isfinite(a)) {
          atomicOr(bad, QR_DEV_NONFINITE);
        } else if (s != 0.0) {
          const double nrm = sqrt(a * a + s);
          const double beta = (a < 0.0) ? nrm : -nrm;
          tau_j = (beta - a) / beta;
          scal = 1.0 / (a - beta);
          *piv = (S)beta;
        }
        tau[jj] = (S)tau_j;
      }
      const S sc = (S)__shfl_sync(0xffffffffu, scal, 0);
      for (int r = x0 + lane; r < nr; r += 32) col[r] *= sc;
    }
    __syncthreads();
    const S tj = tau[jj];
    if (tj != S(0)) {
      for (int cc = jj + 1 + wid; cc < w; cc += NTHREADS / 32) {
        S* pc = P + (size_t)cc * ldp;
        S d = S(0);
        for (int r = x0 + lane; r < nr; r += 32) d = fma(col[r], pc[r], d);
        d = warp_sum(d);
        S* top = TS ? (Rs + jj + (size_t)cc * ldr) : (pc + jj);
        const S wv = tj * (*top + d);
        __syncwarp();
        if (lane == 0) *top -= wv;
        for (int r = x0 + lane; r < nr; r += 32) pc[r] = fma(-wv, col[r], pc[r]);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// GEQRT: QR of the diagonal tile A (rows x cols, ld lda, rows >= cols),
// T (IB x cols, ld IB). Inner blocks of IB; each block is factored in
// sub-panels that fit shared memory (a sub-panel is applied to the rest of
// its block with its own temporary T), then T_l is formed and the block is
// applied to the tile's trailing columns.
template <typename S>
__device__ void geqrt(S* A, int lda, int rows, int cols, int IB, S* T, const Smem<S>& sm, int* bad) {
  for (int l0 = 0; l0 < cols; l0 += IB) {
    const int ib = min(IB, cols - l0);
    const int nrb = rows - l0;  // rows of the block from its first row
    int sb = PANEL_CAP / nrb;
    if (sb > ib) sb = ib;
    if (sb > 32 && sb < ib) sb = 32;
    for (int s0 = l0; s0 < l0 + ib; s0 += sb) {
      const int w = min(sb, l0 + ib - s0);
      const int nr = rows - s0;
      S* P = sm.part;  // nr x w, ld nr
      __syncthreads();
      stage_block<8>(P, nr, A + s0 + (size_t)s0 * lda, lda, nr, w, AllRd(), Ident());
      __syncthreads();
      panel_l2<S, false>(P, nr, nr, w, nullptr, 0, sm.tau + (s0 - l0), sm.red, bad);
      const bool whole = (w == ib);
      if (whole) {
        build_t<S, false>(P, nr, true, nr, w, sm.tau, T + (size_t)l0 * IB, IB, false);
      } else if (s0 + w < l0 + ib) {
        build_t<S, false>(P, nr, true, nr, w, sm.tau + (s0 - l0), sm.ts, w, true);
      }
      for (int idx = threadIdx.x; idx < nr * w; idx += NTHREADS) {
        const int cc = idx / nr, r = idx - cc * nr;
        stg(A + (s0 + r) + (size_t)(s0 + cc) * lda, P[idx]);
      }
      __syncthreads();
      if (!whole && s0 + w < l0 + ib) {
        // apply the sub-panel to the rest of the block (columns s0+w .. l0+ib)
        apply_qt<S, false>(A, lda, sm.ts - (size_t)s0 * w, w, true, s0, s0 + w, w, nullptr, 0, A, lda,
                           rows, s0 + w, l0 + ib, sm);
      }
    }
    if (sb < ib) {
      __syncthreads();
      build_t<S, false>(A + l0 + (size_t)l0 * lda, lda, false, nrb, ib, sm.tau, T + (size_t)l0 * IB, IB,
                        false);
    }
    __syncthreads();
    if (l0 + ib < cols)
      apply_qt<S, false>(A, lda, T, IB, false, l0, l0 + ib, IB, nullptr, 0, A, lda, rows, l0 + ib, cols, sm);
    __syncthreads();
  }
}

// TSQRT: QR of [R (upper triangle of the diagonal tile, ldr); B (rows x
// cols, ldb)]. B receives the reflectors' lower parts, R the new triangle,
// T (IB x cols) the block factors. Never touches R's strict lower part.
//
// tri = true is TTQRT, the triangle-on-triangle step of a reduction tree:
// B's upper triangle is another R factor (its strict lower part belongs to
// someone else and is neither read nor written); the reflectors then live in
// B's upper triangle, column c having rows 0..c.
template <typename S>
__device__ void tsqrt(S* R, int ldr, S* B, int ldb, int rows, int cols, int IB, S* T, const Smem<S>& sm,
                      int* bad, bool tri = false) {
  for (int l0 = 0; l0 < cols; l0 += IB) {
    const int ib = min(IB, cols - l0);
    int sb = PANEL_CAP / rows;
    if (sb > ib) sb = ib;
    if (sb > 32) sb = 32;  // the R sub-block lives in rs (<= 32 x 32)
    for (int s0 = l0; s0 < l0 + ib; s0 += sb) {
      const int w = min(sb, l0 + ib - s0);
      const int nr = tri ? min(rows, s0 + w) : rows;  // rows of B this sub-panel reaches
      S* P = sm.part;  // nr x w
      __syncthreads();
      stage_block<8>(P, nr, B + (size_t)s0 * ldb, ldb, nr, w, [tri, s0](int r, int c) { return !(tri && r > s0 + c); },
                     Ident());
      stage_block<4>(sm.rs, w, R + s0 + (size_t)s0 * ldr, ldr, w, w, [](int r, int c) { return r <= c; }, Ident());
      __syncthreads();
      panel_l2<S, true>(P, nr, nr, w, sm.rs, w, sm.tau + (s0 - l0), sm.red, bad, tri ? s0 : -1);
      const bool whole = (w == ib);
      if (whole) {
        build_t<S, true>(P, nr, true, nr, w, sm.tau, T + (size_t)l0 * IB, IB, false, tri ? s0 : -1);
      } else if (s0 + w < l0 + ib) {
        build_t<S, true>(P, nr, true, nr, w, sm.tau + (s0 - l0), sm.ts, w, true, tri ? s0 : -1);
      }
      for (int idx = threadIdx.x; idx < nr * w; idx += NTHREADS) {
        const int cc = idx / nr, r = idx - cc * nr;
        if (!tri || r <= s0 + cc) stg(B + r + (size_t)(s0 + cc) * ldb, P[idx]);
      }
      for (int idx = threadIdx.x; idx < w * w; idx += NTHREADS) {
        const int cc = idx / w, r = idx - cc * w;
        if (r <= cc) stg(R + (s0 + r) + (size_t)(s0 + cc) * ldr, sm.rs[idx]);
      }
      __syncthreads();
      if (!whole && s0 + w < l0 + ib) {
        apply_qt<S, true>(B, ldb, sm.ts - (size_t)s0 * w, w, true, s0, s0 + w, w, R, ldr, B, ldb, nr, s0 + w,
                          l0 + ib, sm, tri);
      }
    }
    const int nrb = tri ? min(rows, l0 + ib) : rows;  // rows the block's reflectors reach
    if (sb < ib) {
      __syncthreads();
      build_t<S, true>(B + (size_t)l0 * ldb, ldb, false, nrb, ib, sm.tau, T + (size_t)l0 * IB, IB, false,
                       tri ? l0 : -1);
    }
    __syncthreads();
    if (l0 + ib < cols)
      apply_qt<S, true>(B, ldb, T, IB, false, l0, l0 + ib, IB, R, ldr, B, ldb, nrb, l0 + ib, cols, sm, tri);
    __syncthreads();
  }
}

}  // namespace tqr

#include "tc_update.cuh"

namespace tqr {

// UNMQR: C <- Q^T C for the GEQRT factors (V in the diagonal tile, rows x
// nref reflectors, T IB x nref), columns [c0, c1) of C. tc (FP32 tiles
// only): TC_TF32 / TC_BF16X3 run the products on the tensor cores
// (apply_qt_mma), TC_NONE on the FP32/FP64 cores.
template <typename S>
__device__ void unmqr(const S* V, int ldv, const S* T, int IB, int rows, int nref, S* C, int ldc, int c0,
                      int c1, const Smem<S>& sm, int tc = TC_NONE) {
  if constexpr (sizeof(S) == 4) {
    if (tc == TC_TF32 &&
        (apply_qt_mma_staged<TC_TF32, false>(V, ldv, T, IB, nref, IB, nullptr, 0, C, ldc, rows, c0, c1, sm.vs) ||
         apply_qt_mma<TC_TF32, false>(V, ldv, T, IB, nref, IB, nullptr, 0, C, ldc, rows, c0, c1, sm.vs)))
      return;
    if (tc == TC_BF16X3 &&
        (apply_qt_mma_staged<TC_BF16X3, false>(V, ldv, T, IB, nref, IB, nullptr, 0, C, ldc, rows, c0, c1, sm.vs) ||
         apply_qt_mma<TC_BF16X3, false>(V, ldv, T, IB, nref, IB, nullptr, 0, C, ldc, rows, c0, c1, sm.vs)))
      return;
  }
  apply_qt<S, false>(V, ldv, T, IB, false, 0, nref, IB, nullptr, 0, C, ldc, rows, c0, c1, sm);
}

// TSMQR: [C1; C2] <- Q^T [C1; C2] for the TSQRT factors (V rows x nref in
// the bottom tile, T IB x nref); C1 the top tile, C2 (rows) the bottom one.
// tri = true is TTMQR: V holds triangle-on-triangle reflectors (upper
// triangular), so only the first min(rows, nref) rows of C2 change (always
// on the FP32/FP64 cores). tc as for unmqr.
template <typename S>
__device__ void tsmqr(const S* V, int ldv, const S* T, int IB, int rows, int nref, S* C1, int ldc1, S* C2,
                      int ldc2, int c0, int c1, const Smem<S>& sm, bool tri = false, int tc = TC_NONE) {
  if constexpr (sizeof(S) == 4) {
    if (!tri && tc == TC_TF32 &&
        (apply_qt_mma_staged<TC_TF32, true>(V, ldv, T, IB, nref, IB, C1, ldc1, C2, ldc2, rows, c0, c1, sm.vs) ||
         apply_qt_mma<TC_TF32, true>(V, ldv, T, IB, nref, IB, C1, ldc1, C2, ldc2, rows, c0, c1, sm.vs)))
      return;
    if (!tri && tc == TC_BF16X3 &&
        (apply_qt_mma_staged<TC_BF16X3, true>(V, ldv, T, IB, nref, IB, C1, ldc1, C2, ldc2, rows, c0, c1, sm.vs) ||
         apply_qt_mma<TC_BF16X3, true>(V, ldv, T, IB, nref, IB, C1, ldc1, C2, ldc2, rows, c0, c1, sm.vs)))
      return;
  }
  apply_qt<S, true>(V, ldv, T, IB, false, 0, nref, IB, C1, ldc1, C2, ldc2, tri ? min(rows, nref) : rows, c0, c1,
                    sm, tri);
}

}  // namespace tqr
