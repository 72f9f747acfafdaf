// Tensor-core variant of the trailing updates of an FP32 tile QR (UNMQR and
// TSMQR, the paper's DLARFB and DSSRFB, Sec. 2.1) for the mixed-precision
// least-squares solve: the two products of every inner block,
//   Y = V_l^T C (+ the top tile's rows in TS mode) and C -= V_l W,
// run as warp-level mma.sync in
//   TC_TF32:   one TF32 product (operands rounded to TF32, 10-bit fraction),
//   TC_BF16X3: three BF16 products hi*hi + hi*lo + lo*hi of the split
//              operands x = hi + lo (hi = bf16(x), lo = bf16(x - hi)),
// accumulated in FP32. W = T_l^T Y (IB x IB, triangular) stays on the FP32
// cores, and the panel kernels (Householder vectors, tau, T) are untouched.
//
// Data flow of one task (256 threads, 8 warps): the CTA takes C's columns in
// chunks of cw; each warp owns a 16-column x RW-row piece of the chunk and
// keeps it, transposed (rows of the mma tile = columns of C), in its FP32
// accumulator fragments for all inner blocks. The accumulators double as the
// A operand of Y^T = C^T V_l: for TF32 (m16n8k8) the k index of each 8-row
// step is permuted (logical k = t <-> row 2t, k = t + 4 <-> row 2t + 1), so
// an accumulator fragment (c0, c1, c2, c3) is the A fragment (a0, a2, a1,
// a3); for BF16 (m16n8k16) two neighbouring 8-row accumulator tiles are
// exactly one A fragment. The B operand of that product takes the same rows
// from the staged reflectors. Partial Y^T of the warps that share columns are
// summed through shared memory.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tile_kernels.cuh"

namespace tqr {

enum { TC_NONE = 0, TC_TF32 = 1, TC_BF16X3 = 2 };

__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// (x0, x1) -> packed bf16 pairs hi = bf16(x), lo = bf16(x - hi); x0 in the
// low half, as the mma fragments order consecutive k.
__device__ __forceinline__ void split_bf16(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Warp layout of a task: WR warps along the rows (RW rows each, RW a
// multiple of 16 and at most 64) times WM = 8 / WR along the columns (16
// each, cw = 16 WM columns per chunk). Fewest row warps that keep RW <= 64,
// then more while the column range leaves warps idle.
struct TcLayout {
  int WR, WM, RW, rowsPad, cw, IBP, ldvs, ldw;
  size_t need;  // floats of shared memory
};

__device__ __forceinline__ TcLayout tc_layout(int rows, int ncols, int IB, int kq) {
  TcLayout L;
  const int r16 = (rows + 15) / 16 * 16;
  int WR = 1;
  while (WR < 8 && (r16 + 16 * WR - 1) / (16 * WR) * 16 > 64) WR *= 2;
  const int cols16 = (ncols + 15) / 16;
  while (WR < 8 && 8 / WR > cols16 && (r16 + 32 * WR - 1) / (32 * WR) * 16 >= 16) WR *= 2;
  L.WR = WR;
  L.WM = 8 / WR;
  L.RW = (r16 + 16 * WR - 1) / (16 * WR) * 16;
  L.rowsPad = L.RW * WR;
  L.cw = 16 * L.WM;
  L.IBP = (IB + kq - 1) / kq * kq;
  L.ldvs = L.rowsPad + 8;  // staged reflector stride: conflict-free B fragments
  L.ldw = L.cw + 8;        // W stride: conflict-free A fragments of C -= V W
  L.need = (size_t)L.IBP * L.ldvs + (L.WR > 1 ? (size_t)L.WR * L.IBP * L.cw : 0) + (size_t)L.IBP * L.ldw +
           (size_t)L.IBP * L.IBP;
  return L;
}

// Q^T applied to C's columns [c0, c1) (GE mode: UNMQR with the GEQRT
// factors of V, C rows [0, rows); TS mode: TSMQR with the TSQRT factors,
// Ctop the top tile, C the bottom one), blocks of IB reflectors from l0 = 0
// to nref, T_l at T + l0 * ldt (element (q, p) at T[q + (l0 + p) ldt]).
// Returns false, having done nothing, when the task does not fit (more than
// 512 rows, IB > 32, or the shared-memory budget), and the caller then runs
// apply_qt instead. smem: the CTA's FP32 scratch of smem_elems<float>().
template <int MODE, bool TS>
__device__ bool apply_qt_mma(const float* __restrict__ V, int ldv, const float* __restrict__ T, int ldt, int nref,
                             int IB, float* Ctop, int ldct, float* C, int ldc, int rows, int c0, int c1,
                             float* smem) {
  constexpr int KQ = MODE == TC_TF32 ? 8 : 16;
  if (rows <= 0 || c1 <= c0 || nref <= 0) return true;
  if (rows > 512 || IB > 32) return false;
  const TcLayout L = tc_layout(rows, c1 - c0, IB, KQ);
  if (L.RW > 64 || L.need > smem_elems<float>()) return false;
  float* vbuf = smem;
  float* part = vbuf + (size_t)L.IBP * L.ldvs;
  float* wbuf = part + (L.WR > 1 ? (size_t)L.WR * L.IBP * L.cw : 0);
  float* tsb = wbuf + (size_t)L.IBP * L.ldw;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int wm = warp % L.WM, wr = warp / L.WM;
  const int rw0 = wr * L.RW;  // first row of this warp
  const int NJ = L.RW / 8;    // 8-row accumulator tiles per warp (2, 4, 6 or 8)
  for (int cs = c0; cs < c1; cs += L.cw) {
    const int cwn = min(L.cw, c1 - cs);
    const int colA = wm * 16 + g, colB = colA + 8;  // chunk columns of (c0, c1) and (c2, c3)
    const bool okA = colA < cwn, okB = colB < cwn;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = rw0 + 8 * j + 2 * t;
      const bool in = j < NJ;
      acc[j][0] = (in && okA && r < rows) ? ldg(C + r + (size_t)(cs + colA) * ldc) : 0.f;
      acc[j][1] = (in && okA && r + 1 < rows) ? ldg(C + r + 1 + (size_t)(cs + colA) * ldc) : 0.f;
      acc[j][2] = (in && okB && r < rows) ? ldg(C + r + (size_t)(cs + colB) * ldc) : 0.f;
      acc[j][3] = (in && okB && r + 1 < rows) ? ldg(C + r + 1 + (size_t)(cs + colB) * ldc) : 0.f;
    }
    for (int l0 = 0; l0 < nref; l0 += IB) {
      const int ib = min(IB, nref - l0);
      __syncthreads();  // the previous block's readers of vbuf, wbuf and tsb are done
      // stage V_l (zero-padded to IBP x rowsPad; GE: unit diagonal, zero above)
      for (int idx = tid; idx < L.IBP * L.rowsPad; idx += NTHREADS) {
        const int p = idx / L.rowsPad, r = idx - p * L.rowsPad;
        float v = 0.f;
        if (p < ib && r < rows) {
          if (TS) {
            v = ldg(V + r + (size_t)(l0 + p) * ldv);
          } else {
            const int d = l0 + p;
            v = r < d ? 0.f : (r == d ? 1.f : ldg(V + r + (size_t)d * ldv));
          }
        }
        vbuf[p * L.ldvs + r] = v;
      }
      for (int idx = tid; idx < ib * ib; idx += NTHREADS) {
        const int p = idx / ib, q = idx - p * ib;
        tsb[q + p * L.IBP] = q <= p ? ldg(T + q + (size_t)(l0 + p) * ldt) : 0.f;
      }
      __syncthreads();
      // --- Y^T (16 columns x IBP reflectors) over this warp's rows
      float y[4][4];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) y[nt][0] = y[nt][1] = y[nt][2] = y[nt][3] = 0.f;
      if (MODE == TC_TF32) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j < NJ) {
            const uint32_t a[4] = {tf32_of(acc[j][0]), tf32_of(acc[j][2]), tf32_of(acc[j][1]), tf32_of(acc[j][3])};
            const int rb = rw0 + 8 * j + 2 * t;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
              if (nt * 8 < L.IBP) {
                const float2 bv = *reinterpret_cast<const float2*>(vbuf + (nt * 8 + g) * L.ldvs + rb);
                const uint32_t b[2] = {tf32_of(bv.x), tf32_of(bv.y)};
                mma_tf32(y[nt], a, b);
              }
          }
        }
      } else {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          if (2 * jj < NJ) {
            uint32_t ah[4], al[4];
            split_bf16(acc[2 * jj][0], acc[2 * jj][1], ah[0], al[0]);
            split_bf16(acc[2 * jj][2], acc[2 * jj][3], ah[1], al[1]);
            split_bf16(acc[2 * jj + 1][0], acc[2 * jj + 1][1], ah[2], al[2]);
            split_bf16(acc[2 * jj + 1][2], acc[2 * jj + 1][3], ah[3], al[3]);
            const int rb = rw0 + 16 * jj + 2 * t;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
              if (nt * 8 < L.IBP) {
                const float* vp = vbuf + (nt * 8 + g) * L.ldvs + rb;
                const float2 b0 = *reinterpret_cast<const float2*>(vp);
                const float2 b1 = *reinterpret_cast<const float2*>(vp + 8);
                uint32_t bh[2], bl[2];
                split_bf16(b0.x, b0.y, bh[0], bl[0]);
                split_bf16(b1.x, b1.y, bh[1], bl[1]);
                const uint32_t ah_[4] = {ah[0], ah[1], ah[2], ah[3]}, al_[4] = {al[0], al[1], al[2], al[3]};
                const uint32_t bh_[2] = {bh[0], bh[1]}, bl_[2] = {bl[0], bl[1]};
                mma_bf16(y[nt], ah_, bh_);
                mma_bf16(y[nt], ah_, bl_);
                mma_bf16(y[nt], al_, bh_);
              }
          }
        }
      }
      // y[nt]: (0) Y(8nt + 2t, colA), (1) Y(8nt + 2t + 1, colA), (2) Y(8nt + 2t, colB), (3) Y(8nt + 2t + 1, colB)
      {
        float* dst = L.WR > 1 ? part + (size_t)wr * L.IBP * L.cw : wbuf;
        const int ld = L.WR > 1 ? L.cw : L.ldw;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
          if (nt * 8 < L.IBP) {
            const int p0 = nt * 8 + 2 * t;
            dst[p0 * ld + colA] = y[nt][0];
            dst[(p0 + 1) * ld + colA] = y[nt][1];
            dst[p0 * ld + colB] = y[nt][2];
            dst[(p0 + 1) * ld + colB] = y[nt][3];
          }
      }
      __syncthreads();
      // --- Y summed over the row warps, plus the top tile's rows (TS)
      if (L.WR > 1 || TS) {
        for (int o = tid; o < ib * L.cw; o += NTHREADS) {
          const int p = o / L.cw, col = o - p * L.cw;
          float s = 0.f;
          if (L.WR > 1) {
            for (int w2 = 0; w2 < L.WR; ++w2) s += part[((size_t)w2 * L.IBP + p) * L.cw + col];
          } else {
            s = wbuf[p * L.ldw + col];
          }
          if (TS && col < cwn) s += ldg(Ctop + (l0 + p) + (size_t)(cs + col) * ldct);
          wbuf[p * L.ldw + col] = s;
        }
        __syncthreads();
      }
      // --- W = T_l^T Y (at most 32 x 128 outputs: 16 per thread), TS: top rows -= W
      {
        float wq[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int o = tid + u * NTHREADS;
          float s = 0.f;
          if (o < ib * L.cw) {
            const int p = o / L.cw, col = o - p * L.cw;
            for (int q = 0; q <= p; ++q) s = fmaf(tsb[q + p * L.IBP], wbuf[q * L.ldw + col], s);
          }
          wq[u] = s;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int o = tid + u * NTHREADS;
          if (o < L.IBP * L.cw) {
            const int p = o / L.cw, col = o - p * L.cw;
            const float w = o < ib * L.cw ? wq[u] : 0.f;  // padding reflectors contribute nothing
            wbuf[p * L.ldw + col] = w;
            if (TS && o < ib * L.cw && col < cwn) {
              float* pt = Ctop + (l0 + p) + (size_t)(cs + col) * ldct;
              stg(pt, ldg(pt) - w);
            }
          }
        }
        __syncthreads();  // (IBP x cw <= 32 x 128: the loop above wrote every W entry)
      }
      // --- C^T -= W^T V_l^T (16 columns x RW rows per warp)
      if (MODE == TC_TF32) {
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          if (ks * 8 < L.IBP) {
            const int k0 = ks * 8;
            const uint32_t a[4] = {tf32_of(-wbuf[(k0 + t) * L.ldw + colA]), tf32_of(-wbuf[(k0 + t) * L.ldw + colB]),
                                   tf32_of(-wbuf[(k0 + t + 4) * L.ldw + colA]),
                                   tf32_of(-wbuf[(k0 + t + 4) * L.ldw + colB])};
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (j < NJ) {
                const int n0 = rw0 + 8 * j + g;
                const uint32_t b[2] = {tf32_of(vbuf[(k0 + t) * L.ldvs + n0]), tf32_of(vbuf[(k0 + t + 4) * L.ldvs + n0])};
                mma_tf32(acc[j], a, b);
              }
          }
        }
      } else {
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          if (ks * 16 < L.IBP) {
            const int k0 = ks * 16;
            uint32_t ah[4], al[4];
            const float* w0 = wbuf + (k0 + 2 * t) * L.ldw;
            split_bf16(-w0[colA], -w0[L.ldw + colA], ah[0], al[0]);
            split_bf16(-w0[colB], -w0[L.ldw + colB], ah[1], al[1]);
            split_bf16(-w0[8 * L.ldw + colA], -w0[9 * L.ldw + colA], ah[2], al[2]);
            split_bf16(-w0[8 * L.ldw + colB], -w0[9 * L.ldw + colB], ah[3], al[3]);
            const uint32_t ah_[4] = {ah[0], ah[1], ah[2], ah[3]}, al_[4] = {al[0], al[1], al[2], al[3]};
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (j < NJ) {
                const float* vp = vbuf + (k0 + 2 * t) * L.ldvs + rw0 + 8 * j + g;
                uint32_t bh[2], bl[2];
                split_bf16(vp[0], vp[L.ldvs], bh[0], bl[0]);
                split_bf16(vp[8 * L.ldvs], vp[9 * L.ldvs], bh[1], bl[1]);
                const uint32_t bh_[2] = {bh[0], bh[1]}, bl_[2] = {bl[0], bl[1]};
                mma_bf16(acc[j], ah_, bh_);
                mma_bf16(acc[j], ah_, bl_);
                mma_bf16(acc[j], al_, bh_);
              }
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = rw0 + 8 * j + 2 * t;
      if (j < NJ) {
        if (okA && r < rows) stg(C + r + (size_t)(cs + colA) * ldc, acc[j][0]);
        if (okA && r + 1 < rows) stg(C + r + 1 + (size_t)(cs + colA) * ldc, acc[j][1]);
        if (okB && r < rows) stg(C + r + (size_t)(cs + colB) * ldc, acc[j][2]);
        if (okB && r + 1 < rows) stg(C + r + 1 + (size_t)(cs + colB) * ldc, acc[j][3]);
      }
    }
    __syncthreads();
  }
  return true;
}

// Bytes of dynamic shared memory a persistent kernel gets when its tasks
// may take the staged tensor-core path: 96 KB, two CTAs per SM.
constexpr int TC_SMEM_BYTES = 96 * 1024;

__device__ __forceinline__ unsigned dyn_smem_bytes() {
  unsigned r;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

// The same update with everything the inner blocks read staged once per
// task: all nref reflectors (with the GE masks), their T factors, and per
// chunk the top tile's rows 0..nref-1 (TS), which are updated in shared
// memory and written back once. An inner block then costs two barriers:
//   product 1 (partial Y^T per warp) | W = T_l^T (sum of partials + top
//   rows), top rows -= W, one thread per column | product 2.
// Returns false when the staged buffers do not fit the dynamic shared
// memory of the launch (the caller then tries apply_qt_mma).
template <int MODE, bool TS>
__device__ bool apply_qt_mma_staged(const float* __restrict__ V, int ldv, const float* __restrict__ T, int ldt,
                                    int nref, int IB, float* Ctop, int ldct, float* C, int ldc, int rows, int c0,
                                    int c1, float* smem) {
  constexpr int KQ = MODE == TC_TF32 ? 8 : 16;
  if (rows <= 0 || c1 <= c0 || nref <= 0) return true;
  if (rows > 512 || IB > 32 || (ldv & 3) || (reinterpret_cast<uintptr_t>(V) & 15)) return false;
  const TcLayout L = tc_layout(rows, c1 - c0, IB, KQ);
  const int nrefP = (nref + IB - 1) / IB * IB + (L.IBP - IB);  // the last block reads IBP rows from l0
  const int ldcs = L.cw + 1;                                    // top rows: one column per thread
  const size_t nv = (size_t)nrefP * L.ldvs, nt = (size_t)IB * nref, nc = TS ? (size_t)nref * ldcs : 0;
  // partial Y^T always go to part, never to wbuf: a warp may start the next
  // block's product 1 while another still reads W from wbuf in product 2
  // part and ysum rows padded by 8: the tpc threads of a column read rows
  // q, q + 1, ... of one column at once, 8 banks apart
  const int ldp = L.cw + 8;
  const size_t np = (size_t)L.WR * L.IBP * ldp, nw = (size_t)L.IBP * L.ldw, ny = (size_t)L.IBP * ldp;
  if (L.RW > 64 || (nv + nt + nc + np + nw + ny) * sizeof(float) > dyn_smem_bytes()) return false;
  float* vbuf = smem;
  float* tsb = vbuf + nv;
  float* ctop = tsb + nt;
  float* part = ctop + nc;
  float* wbuf = part + np;
  float* ysum = wbuf + nw;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int wm = warp % L.WM, wr = warp / L.WM;
  const int rw0 = wr * L.RW;
  const int NJ = L.RW / 8;
  // reflectors: float4 loads down each column (rows < `rows` only; the tile
  // column holds NB >= rows rounded up to 4 elements), all of a thread's
  // loads in flight before its stores; masks applied in registers; zero
  // padding to nrefP x rowsPad. Then the T factors, 8 loads in flight.
  {
    const int q4 = L.rowsPad / 4;
    const int tot = nrefP * q4;
    for (int base = tid; base < tot; base += 4 * NTHREADS) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + u * NTHREADS;
        const int p = idx / q4, r = 4 * (idx - p * q4);
        v[u] = (idx < tot && p < nref && r < rows) ? __ldcg(reinterpret_cast<const float4*>(V + r + (size_t)p * ldv))
                                                   : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = base + u * NTHREADS;
        if (idx < tot) {
          const int p = idx / q4, r = 4 * (idx - p * q4);
          float* e = &v[u].x;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int rr = r + c;
            if (rr >= rows) e[c] = 0.f;
            else if (!TS) e[c] = rr < p ? 0.f : (rr == p ? 1.f : e[c]);
          }
          *reinterpret_cast<float2*>(vbuf + (size_t)p * L.ldvs + r) = make_float2(v[u].x, v[u].y);
          *reinterpret_cast<float2*>(vbuf + (size_t)p * L.ldvs + r + 2) = make_float2(v[u].z, v[u].w);
        }
      }
    }
    const int tt = IB * nref;
    for (int base = tid; base < tt; base += 8 * NTHREADS) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * NTHREADS;
        const int p = idx / IB, q = idx - p * IB;
        v[u] = idx < tt ? ldg(T + q + (size_t)p * ldt) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (base + u * NTHREADS < tt) tsb[base + u * NTHREADS] = v[u];
    }
  }
  // the W phase: tpc threads per column (consecutive, so within one warp)
  const int tpc = NTHREADS / L.cw;
  const int wcol = tid / tpc, wsub = tid - (tid / tpc) * tpc;
  for (int cs = c0; cs < c1; cs += L.cw) {
    const int cwn = min(L.cw, c1 - cs);
    const int colA = wm * 16 + g, colB = colA + 8;
    const bool okA = colA < cwn, okB = colB < cwn;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = rw0 + 8 * j + 2 * t;
      const bool in = j < NJ;
      acc[j][0] = (in && okA && r < rows) ? ldg(C + r + (size_t)(cs + colA) * ldc) : 0.f;
      acc[j][1] = (in && okA && r + 1 < rows) ? ldg(C + r + 1 + (size_t)(cs + colA) * ldc) : 0.f;
      acc[j][2] = (in && okB && r < rows) ? ldg(C + r + (size_t)(cs + colB) * ldc) : 0.f;
      acc[j][3] = (in && okB && r + 1 < rows) ? ldg(C + r + 1 + (size_t)(cs + colB) * ldc) : 0.f;
    }
    if (TS) {
      const int tot = nref * L.cw;
      for (int base = tid; base < tot; base += 8 * NTHREADS) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base + u * NTHREADS;
          const int p = idx / L.cw, col = idx - p * L.cw;
          v[u] = (idx < tot && col < cwn) ? ldg(Ctop + p + (size_t)(cs + col) * ldct) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int idx = base + u * NTHREADS;
          if (idx < tot) ctop[(idx / L.cw) * ldcs + (idx - (idx / L.cw) * L.cw)] = v[u];
        }
      }
    }
    __syncthreads();  // staged reflectors, T and top rows visible
    for (int l0 = 0; l0 < nref; l0 += IB) {
      const int ib = min(IB, nref - l0);
      const float* vb = vbuf + (size_t)l0 * L.ldvs;
      // --- product 1: partial Y^T of this warp's rows
      float y[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q) y[q][0] = y[q][1] = y[q][2] = y[q][3] = 0.f;
      if (MODE == TC_TF32) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j < NJ) {
            const uint32_t a[4] = {tf32_of(acc[j][0]), tf32_of(acc[j][2]), tf32_of(acc[j][1]), tf32_of(acc[j][3])};
            const int rb = rw0 + 8 * j + 2 * t;
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (q * 8 < L.IBP) {
                const float2 bv = *reinterpret_cast<const float2*>(vb + (q * 8 + g) * L.ldvs + rb);
                const uint32_t b[2] = {tf32_of(bv.x), tf32_of(bv.y)};
                mma_tf32(y[q], a, b);
              }
          }
        }
      } else {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          if (2 * jj < NJ) {
            uint32_t ah[4], al[4];
            split_bf16(acc[2 * jj][0], acc[2 * jj][1], ah[0], al[0]);
            split_bf16(acc[2 * jj][2], acc[2 * jj][3], ah[1], al[1]);
            split_bf16(acc[2 * jj + 1][0], acc[2 * jj + 1][1], ah[2], al[2]);
            split_bf16(acc[2 * jj + 1][2], acc[2 * jj + 1][3], ah[3], al[3]);
            const int rb = rw0 + 16 * jj + 2 * t;
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (q * 8 < L.IBP) {
                const float* vp = vb + (q * 8 + g) * L.ldvs + rb;
                const float2 b0 = *reinterpret_cast<const float2*>(vp);
                const float2 b1 = *reinterpret_cast<const float2*>(vp + 8);
                uint32_t bh[2], bl[2];
                split_bf16(b0.x, b0.y, bh[0], bl[0]);
                split_bf16(b1.x, b1.y, bh[1], bl[1]);
                const uint32_t ah_[4] = {ah[0], ah[1], ah[2], ah[3]}, al_[4] = {al[0], al[1], al[2], al[3]};
                const uint32_t bh_[2] = {bh[0], bh[1]}, bl_[2] = {bl[0], bl[1]};
                mma_bf16(y[q], ah_, bh_);
                mma_bf16(y[q], ah_, bl_);
                mma_bf16(y[q], al_, bh_);
              }
          }
        }
      }
      {
        float* dst = part + (size_t)wr * L.IBP * ldp;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q * 8 < L.IBP) {
            const int p0 = q * 8 + 2 * t;
            dst[p0 * ldp + colA] = y[q][0];
            dst[(p0 + 1) * ldp + colA] = y[q][1];
            dst[p0 * ldp + colB] = y[q][2];
            dst[(p0 + 1) * ldp + colB] = y[q][3];
          }
      }
      __syncthreads();
      // --- W = T_l^T (Y + top rows), top rows -= W: the tpc threads of a
      // column (one warp) sum Y(q) for q = wsub, wsub + tpc, ... (partials
      // of the row warps, plus the top rows in TS mode) into ysum, then form
      // W(p) for p = wsub, wsub + tpc, ...
      {
        const int col = wcol;
        for (int q = wsub; q < ib; q += tpc) {
          float sum = 0.f;
          for (int w2 = 0; w2 < L.WR; ++w2) sum += part[((size_t)w2 * L.IBP + q) * ldp + col];
          if (TS) sum += ctop[(l0 + q) * ldcs + col];
          ysum[q * ldp + col] = sum;
        }
        __syncwarp();  // Y complete for this column; its top rows are read
        const float* tb = tsb + (size_t)l0 * IB;  // T(q, p) of this block at tb[q + p * IB]
        for (int pp = wsub; pp < ib; pp += tpc) {
          const float* tcol = tb + (size_t)pp * IB;
          float wv = 0.f;
          for (int q = 0; q <= pp; ++q) wv = fmaf(tcol[q], ysum[q * ldp + col], wv);
          if (TS) ctop[(l0 + pp) * ldcs + col] -= wv;
          wbuf[pp * L.ldw + col] = wv;
        }
        for (int pp = ib + wsub; pp < L.IBP; pp += tpc) wbuf[pp * L.ldw + col] = 0.f;
      }
      __syncthreads();
      // --- product 2: C^T -= W^T V_l^T
      if (MODE == TC_TF32) {
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          if (ks * 8 < L.IBP) {
            const int k0 = ks * 8;
            const uint32_t a[4] = {tf32_of(-wbuf[(k0 + t) * L.ldw + colA]), tf32_of(-wbuf[(k0 + t) * L.ldw + colB]),
                                   tf32_of(-wbuf[(k0 + t + 4) * L.ldw + colA]),
                                   tf32_of(-wbuf[(k0 + t + 4) * L.ldw + colB])};
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (j < NJ) {
                const int n0 = rw0 + 8 * j + g;
                const uint32_t b[2] = {tf32_of(vb[(k0 + t) * L.ldvs + n0]), tf32_of(vb[(k0 + t + 4) * L.ldvs + n0])};
                mma_tf32(acc[j], a, b);
              }
          }
        }
      } else {
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          if (ks * 16 < L.IBP) {
            const int k0 = ks * 16;
            uint32_t ah[4], al[4];
            const float* w0 = wbuf + (k0 + 2 * t) * L.ldw;
            split_bf16(-w0[colA], -w0[L.ldw + colA], ah[0], al[0]);
            split_bf16(-w0[colB], -w0[L.ldw + colB], ah[1], al[1]);
            split_bf16(-w0[8 * L.ldw + colA], -w0[9 * L.ldw + colA], ah[2], al[2]);
            split_bf16(-w0[8 * L.ldw + colB], -w0[9 * L.ldw + colB], ah[3], al[3]);
            const uint32_t ah_[4] = {ah[0], ah[1], ah[2], ah[3]}, al_[4] = {al[0], al[1], al[2], al[3]};
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (j < NJ) {
                const float* vp = vb + (k0 + 2 * t) * L.ldvs + rw0 + 8 * j + g;
                uint32_t bh[2], bl[2];
                split_bf16(vp[0], vp[L.ldvs], bh[0], bl[0]);
                split_bf16(vp[8 * L.ldvs], vp[9 * L.ldvs], bh[1], bl[1]);
                const uint32_t bh_[2] = {bh[0], bh[1]}, bl_[2] = {bl[0], bl[1]};
                mma_bf16(acc[j], ah_, bh_);
                mma_bf16(acc[j], ah_, bl_);
                mma_bf16(acc[j], al_, bh_);
              }
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = rw0 + 8 * j + 2 * t;
      if (j < NJ) {
        if (okA && r < rows) stg(C + r + (size_t)(cs + colA) * ldc, acc[j][0]);
        if (okA && r + 1 < rows) stg(C + r + 1 + (size_t)(cs + colA) * ldc, acc[j][1]);
        if (okB && r < rows) stg(C + r + (size_t)(cs + colB) * ldc, acc[j][2]);
        if (okB && r + 1 < rows) stg(C + r + 1 + (size_t)(cs + colB) * ldc, acc[j][3]);
      }
    }
    __syncthreads();  // every product 2 has read wbuf / vb; the top rows are final
    if (TS)
      for (int idx = tid; idx < nref * L.cw; idx += NTHREADS) {
        const int p = idx / L.cw, col = idx - p * L.cw;
        if (col < cwn) stg(Ctop + p + (size_t)(cs + col) * ldct, ctop[p * ldcs + col]);
      }
  }
  __syncthreads();
  return true;
}

}  // namespace tqr
