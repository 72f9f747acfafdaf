// Least squares through the tile QR: qr_solve_ls.
//
// FP64 path: factor a copy of A in FP64 (qr_factor_p_d, p panel domains),
// Y = Q^T B, X = R^{-1} Y(0:n). Mixed path: factor an FP32 copy of A (FP64 only in the panel's
// Householder vector / tau generation), then refine on the augmented system
// [I A; A^T 0][r; x] = [b; 0] with FP64 residuals and FP64 accumulation of x
// and r; each correction is solved through the FP32 factors:
//   f = b - r - A x, g = -A^T r                      (FP64, this file)
//   R^T h = g, d = Q^T f, R dx = d(0:n) - h,
//   dr = Q [h; d(n:m)]                               (FP32 factors)
//   x += dx, r += dr                                 (FP64)
// (Bjorck's refinement of least-squares solutions; with x = r = 0 the first
// correction is the plain QR solve.) It converges while kappa(A) u_32 < 1.
//
// TF32 / BF16x3 path: the FP32 copy is factored with its UNMQR/TSMQR
// products on the tensor cores (qr_factor_mixed_s). Their unit roundoff
// (2^-11, 2^-17) makes kappa(A) u > 1 at kappa = 1e6, where the correction
// above no longer contracts, so each refinement step instead solves the
// correction equation K [dr; dx] = [f; g], K = [I A; A^T 0], by GMRES in
// FP64 preconditioned on the left by that correction M^-1 (the inverse of
// the augmented matrix of the low-precision factors): GMRES-based iterative
// refinement for least squares (Carson, Higham and Pranesh, 2020), here with
// FP64 residuals and FP64 Krylov vectors. Classical Gram-Schmidt applied
// twice orthogonalises each new Krylov vector; Givens rotations keep the
// small Hessenberg least-squares problem triangular. QR_OPT_LS_REFINE picks
// either scheme for any low precision.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "sched.cuh"
#include "tileqr_internal.h"

namespace {

constexpr int TB = 256;

template <typename Src, typename Dst>
__global__ void cvt(int64_t m, int64_t n, const Src* s, int64_t lds, Dst* d, int64_t ldd) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / m, r = e - c * m;
    d[r + c * ldd] = (Dst)s[r + c * lds];
  }
}

// Triangular solve with the n x n upper triangle of R (ld ldr), in place on
// the nk <= 8 columns of X (ld ldx). trans = 0: R x = y (backward
// substitution); trans = 1: R^T x = y (forward substitution).
//
// Wavefront over row blocks of TRSM_BS rows: the blocks are taken in solve
// order s (backward: last block first) from an atomic ticket, so the smallest
// unfinished s is always held by a running CTA and the waits end (no
// co-residency is assumed). The CTA holding s subtracts the contribution of
// every earlier-solved block s' < s as soon as flag[s'] is set (one 64 x 64
// block of R against 64 x nk solved values), then solves its diagonal block
// (one warp per right-hand side) and publishes flag[s]. Waits are bounded
// (status bit and abort flag in ctl, as in the factorization's scheduler).
constexpr int TRSM_BS = 64;
constexpr int TRSM_LD = TRSM_BS + 1;  // padded column stride of the staged block

template <typename S>
__global__ void __launch_bounds__(TB) trsm_wave(int n, const S* __restrict__ R, int64_t ldr, S* X, int64_t ldx,
                                                int nk, int trans, tqr::DevCtl* ctl, unsigned* flags,
                                                uint64_t timeout_ns) {
  __shared__ S Rb[TRSM_BS * TRSM_LD];  // Rb[c * TRSM_LD + r] = coefficient of x_c in equation r
  __shared__ S xs[TRSM_BS * 8];        // solved values of a dependency block, [c * 8 + k]
  __shared__ S ys[TRSM_BS * 8];        // right-hand side of the own block, [r * 8 + k]
  __shared__ int s_s, s_ok;
  const int nbk = (n + TRSM_BS - 1) / TRSM_BS;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int r = tid & (TRSM_BS - 1), kg = tid >> 6;  // output rows r, columns kg and kg + 4
  // stage the block of coefficients of the variables of row block bc in the
  // equations of row block br (Rb as above; zero outside the matrix)
  auto stage = [&](int br, int bc) {
    const int rr0 = br * TRSM_BS, cc0 = bc * TRSM_BS;
    const int nr = min(TRSM_BS, n - rr0), nc = min(TRSM_BS, n - cc0);
    for (int idx = tid; idx < TRSM_BS * TRSM_BS; idx += TB) {
      const int i = idx & (TRSM_BS - 1), j = idx / TRSM_BS;
      S v = S(0);
      if (trans == 0) {  // equation rr0+i, variable cc0+j: R(rr0+i, cc0+j)
        if (i < nr && j < nc) v = R[(rr0 + i) + (size_t)(cc0 + j) * ldr];
        Rb[j * TRSM_LD + i] = v;
      } else {           // equation rr0+j, variable cc0+i: R^T(rr0+j, cc0+i) = R(cc0+i, rr0+j)
        if (i < nc && j < nr) v = R[(cc0 + i) + (size_t)(rr0 + j) * ldr];
        Rb[i * TRSM_LD + j] = v;
      }
    }
  };
  for (;;) {
    if (tid == 0) {
      int sv = -1;
      if (!((volatile int*)&ctl->abort)[0]) sv = (int)atomicAdd(&ctl->ticket, 1u);
      s_s = sv;
    }
    __syncthreads();
    const int sidx = s_s;
    if (sidx < 0 || sidx >= nbk) break;
    const int b = trans ? sidx : nbk - 1 - sidx;
    const int r0 = b * TRSM_BS, nr = min(TRSM_BS, n - r0);
    S acc0 = (r < nr && kg < nk) ? X[(r0 + r) + (size_t)kg * ldx] : S(0);
    S acc1 = (r < nr && kg + 4 < nk) ? X[(r0 + r) + (size_t)(kg + 4) * ldx] : S(0);
    bool ok = true;
    for (int sp = 0; sp < sidx && ok; ++sp) {
      const int bp = trans ? sp : nbk - 1 - sp;
      const int c0 = bp * TRSM_BS, nc = min(TRSM_BS, n - c0);
      stage(b, bp);  // R does not change: staged before the wait
      if (tid == 0) s_ok = tqr::wait_ge(flags + sp, 1, 1u, ctl, timeout_ns);
      __syncthreads();
      ok = s_ok;
      if (ok) {
        for (int idx = tid; idx < TRSM_BS * 8; idx += TB) {
          const int c = idx >> 3, k = idx & 7;
          xs[idx] = (c < nc && k < nk) ? __ldcg(X + (c0 + c) + (size_t)k * ldx) : S(0);
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < TRSM_BS; ++c) {
          const S a = Rb[c * TRSM_LD + r];
          acc0 = fma(-a, xs[c * 8 + kg], acc0);
          acc1 = fma(-a, xs[c * 8 + kg + 4], acc1);
        }
      }
      __syncthreads();
    }
    if (!ok) break;
    // diagonal block: one warp per right-hand side, lane holds rows lane, lane+32
    stage(b, b);
    ys[r * 8 + kg] = acc0;
    ys[r * 8 + kg + 4] = acc1;
    __syncthreads();
    if (wid < nk) {
      const int k = wid;
      S y0 = ys[lane * 8 + k], y1 = ys[(lane + 32) * 8 + k];
      // reciprocals of the diagonal, formed off the substitution chain; the
      // chain itself is then one shuffle, one multiply and one FMA per row
      const S ri0 = lane < nr ? S(1) / Rb[lane * TRSM_LD + lane] : S(0);
      const S ri1 = lane + 32 < nr ? S(1) / Rb[(lane + 32) * TRSM_LD + lane + 32] : S(0);
      for (int t = 0; t < nr; ++t) {
        const int j = trans ? t : nr - 1 - t;
        const S v = __shfl_sync(0xffffffffu, j < 32 ? y0 : y1, j & 31);
        const S rj = __shfl_sync(0xffffffffu, j < 32 ? ri0 : ri1, j & 31);
        const S xj = v * rj;
        const S a0 = Rb[j * TRSM_LD + lane], a1 = Rb[j * TRSM_LD + lane + 32];
        if (trans) {
          if (lane > j) y0 = fma(-a0, xj, y0);
          if (lane + 32 > j) y1 = fma(-a1, xj, y1);
        } else {
          if (lane < j) y0 = fma(-a0, xj, y0);
          if (lane + 32 < j) y1 = fma(-a1, xj, y1);
        }
        if (lane == (j & 31)) {
          if (j < 32) y0 = xj;
          else y1 = xj;
        }
      }
      ys[lane * 8 + k] = y0;
      ys[(lane + 32) * 8 + k] = y1;
    }
    __syncthreads();
    if (r < nr) {
      if (kg < nk) __stcg(X + (r0 + r) + (size_t)kg * ldx, ys[r * 8 + kg]);
      if (kg + 4 < nk) __stcg(X + (r0 + r) + (size_t)(kg + 4) * ldx, ys[r * 8 + kg + 4]);
    }
    // publish: the barrier orders every thread's writes of x before
    // thread 0's fence and release (cumulative), one fence per block
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      tqr::red_release_add(flags + sidx, 1u);
    }
  }
}

// Partial products P[s][row][k] = sum_{c in split s} A(row, c) x(c, k) for
// k < nk <= 8. Grid (row blocks of TB, column splits).
__global__ void ax_partial(int64_t m, int64_t n, const double* __restrict__ A, int64_t lda, const double* __restrict__ x,
                           int64_t ldx, int nk, int64_t cols_per_split, double* P) {
  __shared__ double xs[128 * 8];
  const int64_t row = (int64_t)blockIdx.x * TB + threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.y * cols_per_split;
  const int64_t c1 = n < c0 + cols_per_split ? n : c0 + cols_per_split;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t cb = c0; cb < c1; cb += 128) {
    const int cnt = (int)(c1 - cb < 128 ? c1 - cb : 128);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * 8; e += TB) {
      const int c = e / 8, k = e % 8;
      xs[e] = k < nk ? x[(cb + c) + (size_t)k * ldx] : 0.0;
    }
    __syncthreads();
    if (row < m) {
      for (int c = 0; c < cnt; ++c) {
        const double a = A[row + (size_t)(cb + c) * lda];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = fma(a, xs[c * 8 + k], acc[k]);
      }
    }
  }
  if (row < m)
    for (int k = 0; k < nk; ++k) P[((size_t)blockIdx.y * nk + k) * m + row] = acc[k];
}

// f = b - r - sum_s P[s]  (m x nk, ld m for b, r, f taken from their own ld)
__global__ void f_combine(int64_t m, int nk, int nsplit, const double* P, const double* b, int64_t ldb,
                          const double* r, double* f) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * nk; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / m);
    const int64_t row = e - (int64_t)k * m;
    double s = b[row + (size_t)k * ldb] - r[row + (size_t)k * m];
    for (int q = 0; q < nsplit; ++q) s -= P[((size_t)q * nk + k) * m + row];
    f[row + (size_t)k * m] = s;
  }
}

// Partial Q[rb][c][k] = sum_{rows in block rb} A(row, c) r(row, k); one warp
// per column, 8 columns per CTA, r's row block staged in shared memory.
__global__ void atr_partial(int64_t m, int64_t n, const double* __restrict__ A, int64_t lda, const double* __restrict__ r,
                            int64_t ldr, int nk, int rows_per_block, double* Q) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* rs = reinterpret_cast<double*>(smraw);  // rows_per_block x 8
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
  const int cnt = (int)(m - r0 < rows_per_block ? m - r0 : rows_per_block);
  for (int e = threadIdx.x; e < cnt * 8; e += TB) {
    const int rr = e / 8, k = e % 8;
    rs[e] = k < nk ? r[(r0 + rr) + (size_t)k * ldr] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * 8 + wid;
  if (c >= n) return;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const double* a = A + (size_t)c * lda + r0;
  for (int rr = lane; rr < cnt; rr += 32) {
    const double v = a[rr];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = fma(v, rs[rr * 8 + k], acc[k]);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    acc[k] = v;
  }
  if (lane == 0)
    for (int k = 0; k < nk; ++k) Q[((size_t)blockIdx.y * n + c) * 8 + k] = acc[k];
}

// g = -sum_rb Q[rb]  (n x nk, ld n)
__global__ void g_combine(int64_t n, int nk, int nrb, const double* Q, double* g) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * nk; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / n);
    const int64_t c = e - (int64_t)k * n;
    double s = 0.0;
    for (int q = 0; q < nrb; ++q) s += Q[((size_t)q * n + c) * 8 + k];
    g[c + (size_t)k * n] = -s;
  }
}

// Per-column max |v| of an rows x nk FP64 block (ld rows) -> out[k].
__global__ void colmax(int64_t rows, int nk, const double* v, double* out) {
  __shared__ double red[TB / 32];
  const int k = blockIdx.x;
  double mx = 0.0;
  for (int64_t i = threadIdx.x; i < rows; i += TB) mx = fmax(mx, fabs(v[i + (size_t)k * rows]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < TB / 32; ++w) t = fmax(t, red[w]);
    out[k] = t;
  }
}

// Dst(rows x nk, ld ldd) = Src / scale[k] (scale 0 -> 1)
template <typename Src, typename Dst>
__global__ void scale_cvt(int64_t rows, int nk, const Src* s, int64_t lds, const double* scale, Dst* d, int64_t ldd) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * nk; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / rows);
    const int64_t i = e - (int64_t)k * rows;
    const double sc = scale[k] > 0.0 ? scale[k] : 1.0;
    d[i + (size_t)k * ldd] = (Dst)((double)s[i + (size_t)k * lds] / sc);
  }
}

// Assemble [h; d(n:m)] in place in D (m x nk, ld m): D(0:n) = H(0:n) where H
// is the n x nk block (ld n); also T(0:n) = D(0:n) - H(0:n) into T (ld n).
template <typename S>
__global__ void split_correction(int64_t m, int64_t n, int nk, S* D, const S* H, S* Tdst) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * nk; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / n);
    const int64_t i = e - (int64_t)k * n;
    const S dv = D[i + (size_t)k * m], hv = H[i + (size_t)k * n];
    Tdst[i + (size_t)k * n] = dv - hv;
    D[i + (size_t)k * m] = hv;
  }
}

// acc(rows x nk, ld ldacc) += scale[k] * (double)v (ld ldv); also per-column
// sums of squares of the increment and of the result into sq[2*k], sq[2*k+1]
// (atomic; only used for the stopping test).
template <typename S>
__global__ void accumulate(int64_t rows, int nk, const S* v, int64_t ldv, const double* scale, double* acc,
                           int64_t ldacc, double* sq) {
  const int k = blockIdx.y;
  double s_inc = 0.0, s_res = 0.0;
  const double sc = scale ? (scale[k] > 0.0 ? scale[k] : 1.0) : 1.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
    const double inc = sc * (double)v[i + (size_t)k * ldv];
    const double nv = acc[i + (size_t)k * ldacc] + inc;
    acc[i + (size_t)k * ldacc] = nv;
    s_inc += inc * inc;
    s_res += nv * nv;
  }
  if (sq) {
    for (int o = 16; o > 0; o >>= 1) {
      s_inc += __shfl_xor_sync(0xffffffffu, s_inc, o);
      s_res += __shfl_xor_sync(0xffffffffu, s_res, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&sq[2 * k], s_inc);
      atomicAdd(&sq[2 * k + 1], s_res);
    }
  }
}

// ---------------------------------------------------------------------------
// GMRES-IR building blocks (FP64). A Krylov vector of right-hand side k is
// the augmented [r (m); x (n)], len = m + n, stored at base + k * len; the
// basis vector i of a group at V + (i * nk + k) * len.

// w = K v: w_r = v_r + sum_s P[s] (P from ax_partial on v_x), written into
// the f buffer (ld m) -- the A^T v_r half goes through atr_partial/g_sum.
__global__ void aug_combine_r(int64_t m, int nk, int nsplit, const double* P, const double* v, int64_t len, double* f) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * nk; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / m);
    const int64_t row = e - (int64_t)k * m;
    double s = v[row + (size_t)k * len];
    for (int q = 0; q < nsplit; ++q) s += P[((size_t)q * nk + k) * m + row];
    f[row + (size_t)k * m] = s;
  }
}

// g = sum_rb Q[rb]  (n x nk, ld n)
__global__ void g_sum(int64_t n, int nk, int nrb, const double* Q, double* g) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * nk; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / n);
    const int64_t c = e - (int64_t)k * n;
    double s = 0.0;
    for (int q = 0; q < nrb; ++q) s += Q[((size_t)q * n + c) * 8 + k];
    g[c + (size_t)k * n] = s;
  }
}

// dst (rows x nk, ld ldd) = scale[k] * src (working precision, ld lds)
template <typename S>
__global__ void scaled_store(int64_t rows, int nk, const S* src, int64_t lds, const double* scale, double* dst,
                             int64_t ldd) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * nk; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / rows);
    const int64_t i = e - (int64_t)k * rows;
    const double sc = scale[k] > 0.0 ? scale[k] : 1.0;
    dst[i + (size_t)k * ldd] = sc * (double)src[i + (size_t)k * lds];
  }
}

constexpr int GM_BLK = 128;  // CTAs per right-hand side in the Krylov reductions

// part[(k * GM_BLK + b) * nv + i] = partial <V_i, w> of RHS k over the
// CTA's stride of elements (i < nv); w may be V_0 itself (a norm).
__global__ void __launch_bounds__(TB) gm_dots(int64_t len, int nk, int nv, const double* V, const double* w,
                                             double* part) {
  __shared__ double red[TB / 32];
  const int k = blockIdx.y, b = blockIdx.x;
  const double* wk = w + (size_t)k * len;
  for (int i = 0; i < nv; ++i) {
    const double* vi = V + ((size_t)i * nk + k) * len;
    double s = 0.0;
    for (int64_t e = (int64_t)b * TB + threadIdx.x; e < len; e += (int64_t)GM_BLK * TB) s = fma(vi[e], wk[e], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < TB / 32; ++q) t += red[q];
      part[((size_t)k * GM_BLK + b) * nv + i] = t;
    }
    __syncthreads();
  }
}

// h[k * hld + i] (+)= sum_b part (fixed order: deterministic)
__global__ void gm_reduce(int nk, int nv, const double* part, double* h, int hld, int accumulate) {
  const int k = blockIdx.x, i = threadIdx.x;
  if (i >= nv) return;
  double s = 0.0;
  for (int b = 0; b < GM_BLK; ++b) s += part[((size_t)k * GM_BLK + b) * nv + i];
  h[(size_t)k * hld + i] = accumulate ? h[(size_t)k * hld + i] + s : s;
}

// w -= sum_i coef[k * cld + i] V_i   (i < nv)
__global__ void gm_update(int64_t len, int nk, int nv, const double* V, const double* coef, int cld, double* w) {
  const int k = blockIdx.y;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    double s = w[(size_t)k * len + e];
    for (int i = 0; i < nv; ++i) s = fma(-coef[(size_t)k * cld + i], V[((size_t)i * nk + k) * len + e], s);
    w[(size_t)k * len + e] = s;
  }
}

// w *= 1 / nrm[k] (nrm = sqrt of the sum of squares in sq[k]); zero when the
// norm vanished (a lucky breakdown: that RHS's Krylov space is exhausted)
__global__ void gm_scale(int64_t len, int nk, const double* sq, int sld, double* w, double* nrm_out, int nld) {
  const int k = blockIdx.y;
  const double nr = sqrt(sq[(size_t)k * sld]);
  const double inv = nr > 0.0 ? 1.0 / nr : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && nrm_out) nrm_out[(size_t)k * nld] = nr;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
    w[(size_t)k * len + e] *= inv;
}

// State of the small least-squares problem of each RHS: Hessenberg column j
// (h[k * (KM + 1) + i], i <= j + 1, from the Gram-Schmidt coefficients and
// the new norm), the rotations cs/sn, and the rotated right-hand side gv.
// One thread per RHS applies the old rotations to column j, forms rotation
// j, and reports |gv[j + 1]|, the GMRES residual norm.
__global__ void gm_givens(int nk, int j, int KM, const double* h, double* H, double* cs, double* sn, double* gv,
                          double* resid) {
  const int k = threadIdx.x;
  if (k >= nk) return;
  double* Hk = H + (size_t)k * (KM + 1) * KM;  // column j at Hk + j * (KM + 1)
  double* col = Hk + (size_t)j * (KM + 1);
  for (int i = 0; i <= j + 1; ++i) col[i] = h[(size_t)k * (KM + 1) + i];
  double* c = cs + (size_t)k * KM;
  double* s = sn + (size_t)k * KM;
  double* g = gv + (size_t)k * (KM + 1);
  for (int i = 0; i < j; ++i) {
    const double t = c[i] * col[i] + s[i] * col[i + 1];
    col[i + 1] = -s[i] * col[i] + c[i] * col[i + 1];
    col[i] = t;
  }
  const double a = col[j], b = col[j + 1];
  const double rr = hypot(a, b);
  const double cj = rr > 0.0 ? a / rr : 1.0, sj = rr > 0.0 ? b / rr : 0.0;
  c[j] = cj;
  s[j] = sj;
  col[j] = rr;
  col[j + 1] = 0.0;
  g[j + 1] = -sj * g[j];
  g[j] = cj * g[j];
  resid[k] = fabs(g[j + 1]);
}

// y = H(0:jn, 0:jn)^-1 gv(0:jn), back substitution, one thread per RHS.
__global__ void gm_backsolve(int nk, int jn, int KM, const double* H, const double* gv, double* y) {
  const int k = threadIdx.x;
  if (k >= nk) return;
  const double* Hk = H + (size_t)k * (KM + 1) * KM;
  double* yk = y + (size_t)k * (KM + 1);
  for (int i = jn - 1; i >= 0; --i) {
    double t = gv[(size_t)k * (KM + 1) + i];
    for (int l = i + 1; l < jn; ++l) t -= Hk[(size_t)l * (KM + 1) + i] * yk[l];
    const double d = Hk[(size_t)i * (KM + 1) + i];
    yk[i] = d != 0.0 ? t / d : 0.0;
  }
}

// gv = (beta_k, 0, ...): the first rotated right-hand side of each RHS
__global__ void gm_start(int nk, int KM, const double* beta, double* gv) {
  const int k = threadIdx.x;
  if (k >= nk) return;
  for (int i = 0; i <= KM; ++i) gv[(size_t)k * (KM + 1) + i] = i == 0 ? beta[(size_t)k * (KM + 1)] : 0.0;
}

// z = sum_{i < jn} y_i V_i, then x += z_x (ld n), r += z_r (ld m), with the
// per-RHS sums of squares of dx and of the new x in sq[2k], sq[2k + 1].
__global__ void gm_apply(int64_t m, int64_t n, int nk, int jn, int KM, const double* V, const double* y, double* x,
                         double* r, double* sq) {
  const int k = blockIdx.y;
  const int64_t len = m + n;
  double s_inc = 0.0, s_res = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
    double z = 0.0;
    for (int i = 0; i < jn; ++i) z = fma(y[(size_t)k * (KM + 1) + i], V[((size_t)i * nk + k) * len + e], z);
    if (e < m) {
      r[e + (size_t)k * m] += z;
    } else {
      const double nv = x[(e - m) + (size_t)k * n] + z;
      x[(e - m) + (size_t)k * n] = nv;
      s_inc += z * z;
      s_res += nv * nv;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s_inc += __shfl_xor_sync(0xffffffffu, s_inc, o);
    s_res += __shfl_xor_sync(0xffffffffu, s_res, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sq[2 * k], s_inc);
    atomicAdd(&sq[2 * k + 1], s_res);
  }
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct SolveLayout {
  size_t a, t, scr, ap, bw, hw, tw, x, r, f, g, p, q, scale, sq, tsync;
  size_t gv, gpart, gh, gH, gcs, gsn, ggv, gres, gy;  // GMRES-IR (low precisions only)
  size_t total;
  int64_t apbytes;
  int64_t t_el, sbytes;
  int nsplit, nrb, rpb;
  int64_t cps;
};

// Panel domains for the solve's factorization when the caller passes p = 0:
// about one domain per tile column's worth of tile rows (the flat-tree panel
// chain of a tall matrix is MT tiles long), at most 32.
int auto_domains(int64_t m, int64_t n, int nb) {
  const int64_t MT = (m + nb - 1) / nb, NT = (n + nb - 1) / nb;
  return (int)std::max<int64_t>(1, std::min<int64_t>(32, (MT + NT - 1) / std::max<int64_t>(NT, 1)));
}

// Storage precision of the factorization: FP32 for every low precision.
int storage_prec(int prec) { return prec == QR_PREC_F64 ? QR_PREC_F64 : QR_PREC_F32; }

SolveLayout solve_layout(int64_t m, int64_t n, int64_t nrhs, int prec, int nb, int ib, int p) {
  SolveLayout L{};
  const size_t es = prec == QR_PREC_F64 ? 8 : 4;
  qr_workspace_p(m, n, nb, ib, p, storage_prec(prec), &L.t_el, &L.sbytes);
  const int64_t k8 = std::min<int64_t>(nrhs, 8);
  size_t off = 0;
  L.a = off; off = al(off + (size_t)m * n * es);
  L.t = off; off = al(off + (size_t)L.t_el * es);
  L.scr = off; off = al(off + (size_t)L.sbytes);
  qr_apply_workspace_p(m, n, std::min<int64_t>(nrhs, 8), nb, p, &L.apbytes);
  L.ap = off; off = al(off + (size_t)L.apbytes);
  L.bw = off; off = al(off + (size_t)m * k8 * es);
  L.hw = off; off = al(off + (size_t)n * k8 * es);
  L.tw = off; off = al(off + (size_t)n * k8 * es);
  L.x = off; off = al(off + (size_t)n * k8 * 8);
  L.r = off; off = al(off + (size_t)m * k8 * 8);
  L.f = off; off = al(off + (size_t)m * k8 * 8);
  L.g = off; off = al(off + (size_t)n * k8 * 8);
  const int64_t rblocks = (m + TB - 1) / TB;
  L.nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(16, (608 + rblocks - 1) / rblocks));
  L.cps = (n + L.nsplit - 1) / L.nsplit;
  L.p = off; off = al(off + (size_t)L.nsplit * k8 * m * 8);
  L.rpb = 512;  // 32 KB of r per CTA
  L.nrb = (int)((m + L.rpb - 1) / L.rpb);
  L.q = off; off = al(off + (size_t)L.nrb * n * 8 * 8);
  L.scale = off; off = al(off + 2 * 8 * 8);
  L.sq = off; off = al(off + 2 * 8 * 8);
  L.tsync = off; off = al(off + 64 + (size_t)((n + TRSM_BS - 1) / TRSM_BS) * 4);
  if (prec != QR_PREC_F64) {
    const size_t len = (size_t)(m + n), KM = QR_GMRES_MAX_DIM;
    L.gv = off; off = al(off + (KM + 1) * k8 * len * 8);  // Krylov basis
    L.gpart = off; off = al(off + (size_t)k8 * GM_BLK * (KM + 1) * 8);
    L.gh = off; off = al(off + 2 * (size_t)k8 * (KM + 1) * 8);  // Gram-Schmidt coefficients, two passes
    L.gH = off; off = al(off + (size_t)k8 * (KM + 1) * KM * 8);
    L.gcs = off; off = al(off + (size_t)k8 * KM * 8);
    L.gsn = off; off = al(off + (size_t)k8 * KM * 8);
    L.ggv = off; off = al(off + (size_t)k8 * (KM + 1) * 8);
    L.gres = off; off = al(off + (size_t)k8 * 8);
    L.gy = off; off = al(off + (size_t)k8 * (KM + 1) * 8);
  }
  L.total = off;
  return L;
}

int grid_for(int64_t work) { return (int)std::max<int64_t>(1, std::min<int64_t>(4096, (work + TB - 1) / TB)); }

// f = b - r - A x ; g = -A^T r  (FP64; nk <= 8 columns)
int residuals(int64_t m, int64_t n, int nk, const double* A, int64_t lda, const double* B, int64_t ldb, const SolveLayout& L,
              char* w, cudaStream_t st) {
  double* x = (double*)(w + L.x);
  double* r = (double*)(w + L.r);
  double* f = (double*)(w + L.f);
  double* g = (double*)(w + L.g);
  double* P = (double*)(w + L.p);
  double* Q = (double*)(w + L.q);
  dim3 gp((unsigned)((m + TB - 1) / TB), (unsigned)L.nsplit);
  ax_partial<<<gp, TB, 0, st>>>(m, n, A, lda, x, n, nk, L.cps, P);
  f_combine<<<grid_for(m * nk), TB, 0, st>>>(m, nk, L.nsplit, P, B, ldb, r, f);
  dim3 gq((unsigned)((n + 7) / 8), (unsigned)L.nrb);
  atr_partial<<<gq, TB, (size_t)L.rpb * 8 * 8, st>>>(m, n, A, lda, r, m, nk, L.rpb, Q);
  g_combine<<<grid_for(n * nk), TB, 0, st>>>(n, nk, L.nrb, Q, g);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

// Wavefront triangular solve (trsm_wave). sync: the solve's control block
// (tqr::DevCtl, 64 bytes) followed by one flag per row block. Ticket and
// flags are cleared here on the stream; the status and abort words persist
// over the solve and are cleared once at its start.
template <typename S>
int trsm(int64_t n, const S* R, int64_t ldr, S* X, int64_t ldx, int nk, int trans, char* sync, cudaStream_t st) {
  const int nbk = (int)((n + TRSM_BS - 1) / TRSM_BS);
  cudaError_t e = cudaMemsetAsync(sync + 8, 0, 56 + (size_t)nbk * 4, st);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, std::min(nbk, 2 * sms));
  const uint64_t timeout_ns = (uint64_t)qr_get_option(QR_OPT_WAIT_TIMEOUT_US) * 1000ull;
  trsm_wave<S><<<grid, TB, 0, st>>>((int)n, R, ldr, X, ldx, nk, trans, (tqr::DevCtl*)sync, (unsigned*)(sync + 64),
                                    timeout_ns);
  e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

// Q^T / Q through the dependency-ordered persistent application over the
// factorization's domain tree (few right-hand sides still use many SMs).
template <typename S>
int apply(int64_t m, int64_t n, int64_t nk, const S* A, int nb, int ib, int p, const S* T, S* C, int trans, void* ws,
          int64_t wsb, cudaStream_t st);
template <>
int apply<double>(int64_t m, int64_t n, int64_t nk, const double* A, int nb, int ib, int p, const double* T, double* C,
                  int trans, void* ws, int64_t wsb, cudaStream_t st) {
  return qr_apply_qt_p_d(m, n, nk, A, m, nb, ib, p, T, C, m, trans, ws, wsb, st);
}
template <>
int apply<float>(int64_t m, int64_t n, int64_t nk, const float* A, int nb, int ib, int p, const float* T, float* C,
                 int trans, void* ws, int64_t wsb, cudaStream_t st) {
  return qr_apply_qt_p_s(m, n, nk, A, m, nb, ib, p, T, C, m, trans, ws, wsb, st);
}

// colmax wrote max|f| into scale[0..nk) and max|g| into scale[8..8+nk);
// the scale used for both is their maximum.
__global__ void merge_scale(int nk, double* scale) {
  const int k = threadIdx.x;
  if (k < nk) scale[k] = fmax(scale[k], scale[8 + k]);
}

// M^-1 [f; g]: the correction through the working-precision factors.
// Reads f (m x nk) and g (n x nk), FP64; leaves dr / s in Bw (m x nk) and
// dx / s in Tw (n x nk), working precision, s = scale[k] (max |f|, |g| of
// the column, so that the working-precision values neither over- nor
// underflow).
template <typename S>
int correction(int64_t m, int64_t n, int nk, int nb, int ib, int p, const SolveLayout& L, char* w, cudaStream_t st) {
  S* Af = (S*)(w + L.a);
  S* T = (S*)(w + L.t);
  S* Bw = (S*)(w + L.bw);
  S* Hw = (S*)(w + L.hw);
  S* Tw = (S*)(w + L.tw);
  double* f = (double*)(w + L.f);
  double* g = (double*)(w + L.g);
  double* scale = (double*)(w + L.scale);
  int rc;
  colmax<<<nk, TB, 0, st>>>(m, nk, f, scale);
  colmax<<<nk, TB, 0, st>>>(n, nk, g, scale + 8);
  merge_scale<<<1, 32, 0, st>>>(nk, scale);
  // one scale per column covering both f and g
  scale_cvt<double, S><<<grid_for(m * nk), TB, 0, st>>>(m, nk, f, m, scale, Bw, m);
  scale_cvt<double, S><<<grid_for(n * nk), TB, 0, st>>>(n, nk, g, n, scale, Hw, n);
  // R^T h = g/s
  if ((rc = trsm<S>(n, Af, m, Hw, n, nk, 1, w + L.tsync, st))) return rc;
  // d = Q^T f/s
  if ((rc = apply<S>(m, n, nk, Af, nb, ib, p, T, Bw, 1, w + L.ap, L.apbytes, st))) return rc;
  // Tw = d(0:n) - h ; Bw(0:n) = h
  split_correction<S><<<grid_for(n * nk), TB, 0, st>>>(m, n, nk, Bw, Hw, Tw);
  // R dx = Tw
  if ((rc = trsm<S>(n, Af, m, Tw, n, nk, 0, w + L.tsync, st))) return rc;
  // dr = Q [h; d(n:m)]
  if ((rc = apply<S>(m, n, nk, Af, nb, ib, p, T, Bw, 0, w + L.ap, L.apbytes, st))) return rc;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : (int)e;
}

// Outer stopping test shared by both refinement schemes: every column has
// ||dx|| <= tol ||x|| (1), or, from step `from` on, no column's correction
// shrank below `ratio` times the previous one: the accuracy of FP64
// residuals is reached (2). Augmented refinement contracts linearly (from
// step 3, ratio 1/2); a GMRES-IR step solves the correction equation to a
// small relative residual, so a productive step shrinks it by orders of
// magnitude (from step 2, ratio 1/10).
int stop_test(int nk, int it, double tol, const std::vector<double>& hsq, std::vector<double>* prev, int from,
              double ratio) {
  bool met = true, stalled = it >= from;
  for (int k = 0; k < nk; ++k) {
    const double dxn = std::sqrt(hsq[2 * k]);
    if (dxn > tol * std::sqrt(hsq[2 * k + 1])) met = false;
    if (dxn <= ratio * (*prev)[k]) stalled = false;  // this column still converges
    (*prev)[k] = dxn;
  }
  return met ? 1 : (stalled ? 2 : 0);
}

// One group of <= 8 right-hand sides, Bjorck's augmented refinement.
template <typename S>
int solve_group(int64_t m, int64_t n, int nk, const double* A, int64_t lda, const double* B, int64_t ldb, double* X,
                int64_t ldx, int nb, int ib, int p, int max_iter, double tol, int* iters, int* converged,
                const SolveLayout& L, char* w, cudaStream_t st) {
  S* Bw = (S*)(w + L.bw);
  S* Tw = (S*)(w + L.tw);
  double* x = (double*)(w + L.x);
  double* r = (double*)(w + L.r);
  double* scale = (double*)(w + L.scale);
  double* sq = (double*)(w + L.sq);
  cudaError_t e;
  if ((e = cudaMemsetAsync(x, 0, (size_t)n * nk * 8, st)) != cudaSuccess) return (int)e;
  if ((e = cudaMemsetAsync(r, 0, (size_t)m * nk * 8, st)) != cudaSuccess) return (int)e;
  std::vector<double> hsq(2 * nk), prev(nk, 0.0);
  int it = 0, conv = 0;
  const int maxit = std::max(1, max_iter);
  for (; it < maxit && !conv;) {
    int rc = residuals(m, n, nk, A, lda, B, ldb, L, w, st);
    if (rc) return rc;
    if ((rc = correction<S>(m, n, nk, nb, ib, p, L, w, st))) return rc;
    if ((e = cudaMemsetAsync(sq, 0, 2 * 8 * 8, st)) != cudaSuccess) return (int)e;
    accumulate<S><<<dim3(64, nk), TB, 0, st>>>(n, nk, Tw, n, scale, x, n, sq);
    accumulate<S><<<dim3(256, nk), TB, 0, st>>>(m, nk, Bw, m, scale, r, m, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    ++it;
    if (max_iter <= 0) break;  // plain solve: one pass, no refinement test
    if ((e = cudaMemcpyAsync(hsq.data(), sq, 2 * nk * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return (int)e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return (int)e;
    conv = stop_test(nk, it, tol, hsq, &prev, 3, 0.5);
  }
  for (int k = 0; k < nk; ++k)
    if ((e = cudaMemcpyAsync(X + (size_t)k * ldx, x + (size_t)k * n, (size_t)n * 8, cudaMemcpyDeviceToDevice, st)) !=
        cudaSuccess)
      return (int)e;
  *iters = std::max(*iters, it);
  if (max_iter > 0) {
    if (!conv) *converged = 0;
    else if (conv == 2 && *converged == 1) *converged = 2;
  }
  return 0;
}

__global__ void gm_add(int nk, int nv, int hld, const double* src, double* dst) {
  const int k = blockIdx.x, i = threadIdx.x;
  if (i < nv) dst[(size_t)k * hld + i] += src[(size_t)k * hld + i];
}

// One group of <= 8 right-hand sides, GMRES-based refinement: each step
// solves K [dr; dx] = [f; g] by GMRES on M^-1 K (M^-1 = correction<S>) to a
// relative residual of 10^-QR_OPT_GMRES_TOL_EXP or QR_OPT_GMRES_MAX
// iterations, then updates x and r in FP64. *inner counts GMRES iterations.
template <typename S>
int solve_group_gmres(int64_t m, int64_t n, int nk, const double* A, int64_t lda, const double* B, int64_t ldb,
                      double* X, int64_t ldx, int nb, int ib, int p, int max_iter, double tol, int* iters,
                      int* converged, int* inner, const SolveLayout& L, char* w, cudaStream_t st) {
  constexpr int KX = QR_GMRES_MAX_DIM;  // array strides
  constexpr int HL = KX + 1;
  const int KM = (int)std::max<int64_t>(1, std::min<int64_t>(KX, qr_get_option(QR_OPT_GMRES_MAX)));
  const double tau = std::pow(10.0, -(double)qr_get_option(QR_OPT_GMRES_TOL_EXP));
  const int64_t len = m + n;
  S* Bw = (S*)(w + L.bw);
  S* Tw = (S*)(w + L.tw);
  double* x = (double*)(w + L.x);
  double* r = (double*)(w + L.r);
  double* f = (double*)(w + L.f);
  double* g = (double*)(w + L.g);
  double* P = (double*)(w + L.p);
  double* Q = (double*)(w + L.q);
  double* scale = (double*)(w + L.scale);
  double* sq = (double*)(w + L.sq);
  double* V = (double*)(w + L.gv);
  double* part = (double*)(w + L.gpart);
  double* h = (double*)(w + L.gh);
  double* h2 = h + (size_t)8 * HL;
  double* H = (double*)(w + L.gH);
  double* cs = (double*)(w + L.gcs);
  double* sn = (double*)(w + L.gsn);
  double* gv = (double*)(w + L.ggv);
  double* res = (double*)(w + L.gres);
  double* y = (double*)(w + L.gy);
  cudaError_t e;
  if ((e = cudaMemsetAsync(x, 0, (size_t)n * nk * 8, st)) != cudaSuccess) return (int)e;
  if ((e = cudaMemsetAsync(r, 0, (size_t)m * nk * 8, st)) != cudaSuccess) return (int)e;
  const dim3 gl((unsigned)std::min<int64_t>(256, (len + TB - 1) / TB), (unsigned)nk);
  auto dots = [&](const double* Vb, int nv, const double* wv, double* hout) {
    gm_dots<<<dim3(GM_BLK, nk), TB, 0, st>>>(len, nk, nv, Vb, wv, part);
    gm_reduce<<<nk, 128, 0, st>>>(nk, nv, part, hout, HL, 0);
  };
  // M^-1 [f; g] into the Krylov slot Vs (both halves, FP64)
  auto precond = [&](double* Vs) -> int {
    int rc = correction<S>(m, n, nk, nb, ib, p, L, w, st);
    if (rc) return rc;
    scaled_store<S><<<grid_for(m * nk), TB, 0, st>>>(m, nk, Bw, m, scale, Vs, len);
    scaled_store<S><<<grid_for(n * nk), TB, 0, st>>>(n, nk, Tw, n, scale, Vs + m, len);
    return 0;
  };
  std::vector<double> hsq(2 * nk), prev(nk, 0.0), hres(nk), hbeta(HL * nk);
  int it = 0, conv = 0;
  const int maxit = std::max(1, max_iter);
  for (; it < maxit && !conv;) {
    int rc = residuals(m, n, nk, A, lda, B, ldb, L, w, st);
    if (rc) return rc;
    if ((rc = precond(V))) return rc;
    dots(V, 1, V, h2);
    gm_scale<<<gl, TB, 0, st>>>(len, nk, h2, HL, V, y, HL);  // beta_k into y[k * HL]
    gm_start<<<1, 32, 0, st>>>(nk, KX, y, gv);
    if ((e = cudaMemcpyAsync(hbeta.data(), y, sizeof(double) * HL * nk, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return (int)e;
    int jn = 0;
    for (int j = 0; j < KM; ++j) {
      double* Vj = V + (size_t)j * nk * len;
      double* Wn = V + (size_t)(j + 1) * nk * len;
      // [f; g] = K V_j (FP64), then Wn = M^-1 [f; g]
      dim3 gp((unsigned)((m + TB - 1) / TB), (unsigned)L.nsplit);
      ax_partial<<<gp, TB, 0, st>>>(m, n, A, lda, Vj + m, len, nk, L.cps, P);
      aug_combine_r<<<grid_for(m * nk), TB, 0, st>>>(m, nk, L.nsplit, P, Vj, len, f);
      dim3 gq((unsigned)((n + 7) / 8), (unsigned)L.nrb);
      atr_partial<<<gq, TB, (size_t)L.rpb * 8 * 8, st>>>(m, n, A, lda, Vj, len, nk, L.rpb, Q);
      g_sum<<<grid_for(n * nk), TB, 0, st>>>(n, nk, L.nrb, Q, g);
      if ((rc = precond(Wn))) return rc;
      // classical Gram-Schmidt, twice
      dots(V, j + 1, Wn, h);
      gm_update<<<gl, TB, 0, st>>>(len, nk, j + 1, V, h, HL, Wn);
      dots(V, j + 1, Wn, h2);
      gm_update<<<gl, TB, 0, st>>>(len, nk, j + 1, V, h2, HL, Wn);
      gm_add<<<nk, 128, 0, st>>>(nk, j + 1, HL, h2, h);
      // h[j + 1] = ||Wn||, Wn /= ||Wn||
      dots(Wn, 1, Wn, h2);
      gm_scale<<<gl, TB, 0, st>>>(len, nk, h2, HL, Wn, h + (j + 1), HL);
      gm_givens<<<1, 32, 0, st>>>(nk, j, KX, h, H, cs, sn, gv, res);
      if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
      jn = j + 1;
      ++*inner;
      if ((e = cudaMemcpyAsync(hres.data(), res, sizeof(double) * nk, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return (int)e;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return (int)e;
      bool done = true;
      for (int k = 0; k < nk; ++k)
        if (hres[k] > tau * hbeta[(size_t)k * HL]) done = false;
      if (done) break;
    }
    gm_backsolve<<<1, 32, 0, st>>>(nk, jn, KX, H, gv, y);
    if ((e = cudaMemsetAsync(sq, 0, 2 * 8 * 8, st)) != cudaSuccess) return (int)e;
    gm_apply<<<gl, TB, 0, st>>>(m, n, nk, jn, KX, V, y, x, r, sq);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    ++it;
    if (max_iter <= 0) break;  // one GMRES-preconditioned solve, no refinement test
    if ((e = cudaMemcpyAsync(hsq.data(), sq, 2 * nk * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return (int)e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return (int)e;
    conv = stop_test(nk, it, tol, hsq, &prev, 2, 0.1);
  }
  for (int k = 0; k < nk; ++k)
    if ((e = cudaMemcpyAsync(X + (size_t)k * ldx, x + (size_t)k * n, (size_t)n * 8, cudaMemcpyDeviceToDevice, st)) !=
        cudaSuccess)
      return (int)e;
  *iters = std::max(*iters, it);
  if (max_iter > 0) {
    if (!conv) *converged = 0;
    else if (conv == 2 && *converged == 1) *converged = 2;
  }
  return 0;
}

}  // namespace

extern "C" {

int qr_solve_ls_workspace(int64_t m, int64_t n, int64_t nrhs, int prec, int nb, int ib, int p, int64_t* bytes) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (nrhs < 1) return -3;
  if (prec < QR_PREC_F64 || prec > QR_PREC_BF16X3) return -4;
  if (nb == 0 && qr_lookup(m, n, storage_prec(prec), &nb, &ib) != 0) return -5;
  if (!bytes) return -8;
  if (p < 0 || p > 4096) return -6;
  if (p == 0) p = auto_domains(m, n, nb);
  *bytes = (int64_t)solve_layout(m, n, nrhs, prec, nb, ib, p).total;
  return 0;
}

int qr_solve_ls(int64_t m, int64_t n, int64_t nrhs, const double* A, int64_t lda, const double* B, int64_t ldb,
                double* X, int64_t ldx, int prec, int nb, int ib, int p, int max_iter, double tol, int* info,
                void* d_work, int64_t work_bytes, void* stream) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (nrhs < 1) return -3;
  if (!A) return -4;
  if (lda < m) return -5;
  if (!B) return -6;
  if (ldb < m) return -7;
  if (!X) return -8;
  if (ldx < n) return -9;
  if (prec < QR_PREC_F64 || prec > QR_PREC_BF16X3) return -10;
  if (nb == 0 && qr_lookup(m, n, storage_prec(prec), &nb, &ib) != 0) return -11;
  if (nb < 8 || nb > 512) return -11;
  if (ib < 1 || ib > nb || ib > 256) return -12;
  if (p < 0 || p > 4096) return -13;
  if (p == 0) p = auto_domains(m, n, nb);
  if (!d_work) return -17;
  cudaStream_t st = (cudaStream_t)stream;
  const SolveLayout L = solve_layout(m, n, nrhs, prec, nb, ib, p);
  if (work_bytes < (int64_t)L.total) return -18;
  char* w = (char*)d_work;
  cudaError_t e;
  int rc;
  // factor the working-precision copy
  if (prec == QR_PREC_F64) {
    cvt<double, double><<<grid_for(m * n), TB, 0, st>>>(m, n, A, lda, (double*)(w + L.a), m);
    rc = qr_factor_p_d(m, n, (double*)(w + L.a), m, nb, ib, p, (double*)(w + L.t), w + L.scr, L.sbytes, st);
  } else {
    cvt<double, float><<<grid_for(m * n), TB, 0, st>>>(m, n, A, lda, (float*)(w + L.a), m);
    rc = qr_factor_p_tc_s(m, n, (float*)(w + L.a), m, nb, ib, p, (float*)(w + L.t), w + L.scr, L.sbytes, st,
                          tc_of_prec(prec));
  }
  if (rc) return rc;
  if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
  if ((e = cudaMemsetAsync(w + L.tsync, 0, 64, st)) != cudaSuccess) return (int)e;
  // refinement scheme: QR_OPT_LS_REFINE, automatic = augmented refinement for
  // FP32 factors, GMRES-IR for the tensor-core precisions
  const int64_t ro = qr_get_option(QR_OPT_LS_REFINE);
  const bool gmres = prec != QR_PREC_F64 && (ro == 2 || (ro == 0 && prec != QR_PREC_F32));
  int iters = 0, conv = 1, inner = 0;
  for (int64_t k0 = 0; k0 < nrhs; k0 += 8) {
    const int nk = (int)std::min<int64_t>(8, nrhs - k0);
    const double* Bk = B + (size_t)k0 * ldb;
    double* Xk = X + (size_t)k0 * ldx;
    if (prec == QR_PREC_F64)
      rc = solve_group<double>(m, n, nk, A, lda, Bk, ldb, Xk, ldx, nb, ib, p, max_iter, tol, &iters, &conv, L, w, st);
    else if (gmres)
      rc = solve_group_gmres<float>(m, n, nk, A, lda, Bk, ldb, Xk, ldx, nb, ib, p, max_iter, tol, &iters, &conv,
                                    &inner, L, w, st);
    else
      rc = solve_group<float>(m, n, nk, A, lda, Bk, ldb, Xk, ldx, nb, ib, p, max_iter, tol, &iters, &conv, L, w, st);
    if (rc) return rc;
  }
  if (info) {
    info[0] = iters;
    info[1] = conv;
    int status = 0, tstatus = 0;
    if ((rc = qr_status(w + L.scr, &status, st)) != 0) return rc;
    if ((rc = qr_status(w + L.tsync, &tstatus, st)) != 0) return rc;
    info[2] = status | tstatus;
    info[3] = inner;
  }
  return 0;
}

}  // extern "C"
