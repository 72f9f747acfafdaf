/*
 * Plain CPU oracle for Householder QR, the least-squares solve built on it,
 * and the accuracy checks used against the GPU path.
 *
 * TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and the benchmark's
 * CPU-baseline leg load this library. The GPU product path never calls it.
 *
 * Everything here is the textbook definition written out in fp64 (doubled
 * precision by compensated sums for refinement residuals; long double for the
 * brute-force Gram-Schmidt pin and the accuracy checks), column-major storage,
 * no blocking and no reordering beyond what the definition states. Built with
 * -ffp-contract=off so that x86 and Arm hosts round identically.
 *
 * The paper (Agullo, Dongarra, Nath, Tomov, "A Fully Empirical Autotuned Dense
 * QR Factorization for Multicore Architectures") tunes the tile Householder QR
 * of a matrix of order N in double precision (Sec. 2.1, Problem 2.1); tile QR
 * reaches, in exact arithmetic, the Householder QR of the whole matrix up to
 * the signs of R's rows, so the oracle is the unblocked Householder QR.
 * The reflector convention is LAPACK's (beta = -sign(alpha)*||(alpha, x)||,
 * tau = (beta - alpha)/beta, v = [1; x/(alpha - beta)]), which the paper
 * inherits from the kernels it cites in Sec. 2.1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(r, c, ld) ((size_t)(r) + (size_t)(c) * (size_t)(ld))

int oracle_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/* One Householder reflector (Sec. 2.1 kernels, LAPACK convention).
 * On entry *alpha is the pivot and x[0..len) the entries below it.
 * On exit *alpha holds beta (the new diagonal of R), x holds v[1..], and the
 * return value is tau. A zero x gives tau = 0 (H = I) and leaves alpha. */
static double make_reflector(double *alpha, double *x, int64_t len) {
  double xi2 = 0.0;
  for (int64_t r = 0; r < len; ++r) xi2 += x[r] * x[r];
  if (xi2 == 0.0) return 0.0;
  double a = *alpha;
  double norm = sqrt(a * a + xi2);
  double beta = (a < 0.0) ? norm : -norm; /* -sign(alpha)*norm, sign(0) = +1 */
  double tau = (beta - a) / beta;
  double d = a - beta;
  for (int64_t r = 0; r < len; ++r) x[r] = x[r] / d;
  *alpha = beta;
  return tau;
}

/* Unblocked Householder QR (dgeqr2-style), in place, of the m x n matrix A.
 * Computes the first kmax reflectors (kmax <= min(m, n); a smaller kmax is a
 * partial factorization whose first kmax rows of R are final).
 * On exit: R in the upper triangle of the first kmax rows, v_j below the
 * diagonal of column j (unit leading entry implicit), tau[j].
 * Trailing columns are independent given v_j, so that loop runs in parallel. */
int oracle_geqr2(int64_t m, int64_t n, int64_t kmax, double *A, int64_t lda, double *tau) {
  int64_t kk = m < n ? m : n;
  if (kmax < 0 || kmax > kk) kmax = kk;
  if (lda < m) return -5;
  for (int64_t j = 0; j < kmax; ++j) {
    double *colj = A + IDX(j, j, lda);
    double t = make_reflector(colj, colj + 1, m - j - 1);
    tau[j] = t;
    if (t == 0.0) continue;
    const double *v = colj + 1; /* v[0] = 1 implicit at row j */
    int64_t len = m - j - 1;
#pragma omp parallel for schedule(static) if ((n - j) * (m - j) > 32768)
    for (int64_t c = j + 1; c < n; ++c) {
      double *a = A + IDX(j, c, lda);
      double w = a[0];
      for (int64_t r = 0; r < len; ++r) w += v[r] * a[r + 1];
      w *= t;
      a[0] -= w;
      for (int64_t r = 0; r < len; ++r) a[r + 1] -= w * v[r];
    }
  }
  return 0;
}

/* C <- Q^T C with Q = H_0 H_1 ... H_{k-1} from oracle_geqr2 (so Q^T applies
 * H_0 first). C is m x nrhs. */
int oracle_apply_qt(int64_t m, int64_t k, const double *A, int64_t lda, const double *tau,
                    int64_t nrhs, double *C, int64_t ldc) {
  for (int64_t j = 0; j < k; ++j) {
    double t = tau[j];
    if (t == 0.0) continue;
    const double *v = A + IDX(j + 1, j, lda);
    int64_t len = m - j - 1;
#pragma omp parallel for schedule(static) if (nrhs * (m - j) > 32768)
    for (int64_t c = 0; c < nrhs; ++c) {
      double *a = C + IDX(j, c, ldc);
      double w = a[0];
      for (int64_t r = 0; r < len; ++r) w += v[r] * a[r + 1];
      w *= t;
      a[0] -= w;
      for (int64_t r = 0; r < len; ++r) a[r + 1] -= w * v[r];
    }
  }
  return 0;
}

/* C <- Q C (applies H_{k-1} first). */
int oracle_apply_q(int64_t m, int64_t k, const double *A, int64_t lda, const double *tau,
                   int64_t nrhs, double *C, int64_t ldc) {
  for (int64_t j = k - 1; j >= 0; --j) {
    double t = tau[j];
    if (t == 0.0) continue;
    const double *v = A + IDX(j + 1, j, lda);
    int64_t len = m - j - 1;
#pragma omp parallel for schedule(static) if (nrhs * (m - j) > 32768)
    for (int64_t c = 0; c < nrhs; ++c) {
      double *a = C + IDX(j, c, ldc);
      double w = a[0];
      for (int64_t r = 0; r < len; ++r) w += v[r] * a[r + 1];
      w *= t;
      a[0] -= w;
      for (int64_t r = 0; r < len; ++r) a[r + 1] -= w * v[r];
    }
  }
  return 0;
}

/* Explicit thin Q (m x n) = H_0 ... H_{n-1} [I; 0] (dorg2r-style). */
int oracle_form_q(int64_t m, int64_t n, const double *A, int64_t lda, const double *tau,
                  double *Q, int64_t ldq) {
  for (int64_t c = 0; c < n; ++c)
    for (int64_t r = 0; r < m; ++r) Q[IDX(r, c, ldq)] = (r == c) ? 1.0 : 0.0;
  return oracle_apply_q(m, n, A, lda, tau, n, Q, ldq);
}

/* Back substitution R x = y for the n x n upper triangle of R, nrhs columns. */
int oracle_trsm_upper(int64_t n, const double *R, int64_t ldr, int64_t nrhs, double *Y, int64_t ldy) {
  for (int64_t c = 0; c < nrhs; ++c) {
    double *y = Y + IDX(0, c, ldy);
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int64_t p = i + 1; p < n; ++p) s -= R[IDX(i, p, ldr)] * y[p];
      y[i] = s / R[IDX(i, i, ldr)];
    }
  }
  return 0;
}

/* Least squares min ||A x - b|| through Householder QR: factor a copy of A,
 * y = Q^T b, x = R^{-1} y[0:n]. X is n x nrhs. */
int oracle_ls_solve(int64_t m, int64_t n, const double *A, int64_t lda, int64_t nrhs,
                    const double *B, int64_t ldb, double *X, int64_t ldx) {
  if (m < n) return -1;
  double *F = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
  double *tau = (double *)malloc(sizeof(double) * (size_t)n);
  double *Y = (double *)malloc(sizeof(double) * (size_t)m * (size_t)nrhs);
  if (!F || !tau || !Y) { free(F); free(tau); free(Y); return -100; }
  for (int64_t c = 0; c < n; ++c) memcpy(F + IDX(0, c, m), A + IDX(0, c, lda), sizeof(double) * (size_t)m);
  for (int64_t c = 0; c < nrhs; ++c) memcpy(Y + IDX(0, c, m), B + IDX(0, c, ldb), sizeof(double) * (size_t)m);
  oracle_geqr2(m, n, n, F, m, tau);
  oracle_apply_qt(m, n, F, m, tau, nrhs, Y, m);
  oracle_trsm_upper(n, F, m, nrhs, Y, m);
  for (int64_t c = 0; c < nrhs; ++c) memcpy(X + IDX(0, c, ldx), Y + IDX(0, c, m), sizeof(double) * (size_t)n);
  free(F); free(tau); free(Y);
  return 0;
}

/* Error-free transformations (Knuth's TwoSum, FMA-based TwoProduct) for the
 * doubled-precision residuals of the refinement below (the compensated dot
 * product of Ogita, Rump and Oishi, "Accurate sum and dot product", 2005). */
static inline void two_sum(double a, double b, double *s, double *e) {
  double x = a + b, z = x - a;
  *s = x;
  *e = (a - (x - z)) + (b - z);
}
static inline void two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  *p = x;
  *e = fma(a, b, -x);
}

/* Reference least-squares solution: the fp64 QR solve, refined on the
 * augmented system [I A; A^T 0][r; x] = [b; 0] (Bjorck's refinement of
 * least-squares solutions) with residuals in doubled precision (compensated
 * sums) and x, r carried as unevaluated double-double pairs.
 * Corrections come from the same fp64 QR: with f = b - r - A x and
 * g = -A^T r, solve R^T h = g, d = Q^T f, dx = R^{-1}(d[0:n] - h),
 * dr = Q [h; d[n:m]]. Iterates until ||dx|| <= tol ||x|| or maxit.
 * Returns the largest iteration count over the right-hand sides. */
int oracle_ls_refine(int64_t m, int64_t n, const double *A, int64_t lda, int64_t nrhs,
                     const double *B, int64_t ldb, double *X, int64_t ldx, int maxit, double tol) {
  if (m < n) return -1;
  double *F = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
  double *tau = (double *)malloc(sizeof(double) * (size_t)n);
  double *f = (double *)malloc(sizeof(double) * (size_t)m);
  double *g = (double *)malloc(sizeof(double) * (size_t)n);
  double *d = (double *)malloc(sizeof(double) * (size_t)n);
  double *rh = (double *)malloc(sizeof(double) * (size_t)m);
  double *rlo = (double *)malloc(sizeof(double) * (size_t)m);
  double *xh = (double *)malloc(sizeof(double) * (size_t)n);
  double *xlo = (double *)malloc(sizeof(double) * (size_t)n);
  if (!F || !tau || !f || !g || !d || !rh || !rlo || !xh || !xlo) {
    free(F); free(tau); free(f); free(g); free(d); free(rh); free(rlo); free(xh); free(xlo);
    return -100;
  }
  for (int64_t c = 0; c < n; ++c) memcpy(F + IDX(0, c, m), A + IDX(0, c, lda), sizeof(double) * (size_t)m);
  oracle_geqr2(m, n, n, F, m, tau);
  int it_max = 0;
  for (int64_t c = 0; c < nrhs; ++c) {
    const double *b = B + IDX(0, c, ldb);
    double *x = X + IDX(0, c, ldx);
    /* initial solve: x = R^{-1} (Q^T b)[0:n], r = Q [0; (Q^T b)[n:m]] */
    for (int64_t i = 0; i < m; ++i) f[i] = b[i];
    oracle_apply_qt(m, n, F, m, tau, 1, f, m);
    for (int64_t i = 0; i < n; ++i) d[i] = f[i];
    oracle_trsm_upper(n, F, m, 1, d, m);
    for (int64_t i = 0; i < n; ++i) { xh[i] = d[i]; xlo[i] = 0.0; f[i] = 0.0; }
    oracle_apply_q(m, n, F, m, tau, 1, f, m);
    for (int64_t i = 0; i < m; ++i) { rh[i] = f[i]; rlo[i] = 0.0; }
    int it = 0;
    while (it < maxit) {
      ++it;
      /* f = b - r - A x, rows independent */
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < m; ++i) {
        double s, e, p, ep, comp = 0.0;
        two_sum(b[i], -rh[i], &s, &e);
        comp += e - rlo[i];
        for (int64_t q = 0; q < n; ++q) {
          double a = A[IDX(i, q, lda)];
          two_prod(a, -xh[q], &p, &ep);
          two_sum(s, p, &s, &e);
          comp += e + ep - a * xlo[q];
        }
        f[i] = s + comp;
      }
      /* g = -A^T r, columns independent */
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < n; ++q) {
        double s = 0.0, e, p, ep, comp = 0.0;
        for (int64_t i = 0; i < m; ++i) {
          double a = A[IDX(i, q, lda)];
          two_prod(a, -rh[i], &p, &ep);
          two_sum(s, p, &s, &e);
          comp += e + ep - a * rlo[i];
        }
        g[q] = s + comp;
      }
      /* R^T h = g (forward substitution), h stored in g */
      for (int64_t i = 0; i < n; ++i) {
        double s = g[i];
        for (int64_t p = 0; p < i; ++p) s -= F[IDX(p, i, m)] * g[p];
        g[i] = s / F[IDX(i, i, m)];
      }
      oracle_apply_qt(m, n, F, m, tau, 1, f, m); /* f = Q^T f = [d1; d2] */
      for (int64_t i = 0; i < n; ++i) d[i] = f[i] - g[i];
      oracle_trsm_upper(n, F, m, 1, d, m);      /* dx */
      double dxn = 0.0, xn = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        double s, e;
        two_sum(xh[i], d[i], &s, &e);
        e += xlo[i];
        two_sum(s, e, &xh[i], &xlo[i]);
        dxn += d[i] * d[i];
        xn += xh[i] * xh[i];
      }
      for (int64_t i = 0; i < n; ++i) f[i] = g[i];
      oracle_apply_q(m, n, F, m, tau, 1, f, m);  /* dr = Q [h; d2] */
      for (int64_t i = 0; i < m; ++i) {
        double s, e;
        two_sum(rh[i], f[i], &s, &e);
        e += rlo[i];
        two_sum(s, e, &rh[i], &rlo[i]);
      }
      if (sqrt(dxn) <= tol * sqrt(xn)) break;
    }
    if (it > it_max) it_max = it;
    for (int64_t i = 0; i < n; ++i) x[i] = xh[i] + xlo[i];
  }
  free(F); free(tau); free(f); free(g); free(d); free(rh); free(rlo); free(xh); free(xlo);
  return it_max;
}

/* Modified Gram-Schmidt in long double: R (n x n, upper) with positive
 * diagonal. A brute-force pin for |R| on small inputs. */
int oracle_mgs_ld(int64_t m, int64_t n, const double *A, int64_t lda, double *R, int64_t ldr) {
  long double *Q = (long double *)malloc(sizeof(long double) * (size_t)m * (size_t)n);
  if (!Q) return -100;
  for (int64_t c = 0; c < n; ++c)
    for (int64_t r = 0; r < m; ++r) Q[IDX(r, c, m)] = A[IDX(r, c, lda)];
  for (int64_t c = 0; c < n; ++c)
    for (int64_t r = 0; r < n; ++r) R[IDX(r, c, ldr)] = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    long double s = 0.0L;
    for (int64_t r = 0; r < m; ++r) s += Q[IDX(r, j, m)] * Q[IDX(r, j, m)];
    long double nrm = sqrtl(s);
    R[IDX(j, j, ldr)] = (double)nrm;
    if (nrm == 0.0L) continue;
    for (int64_t r = 0; r < m; ++r) Q[IDX(r, j, m)] /= nrm;
    for (int64_t c = j + 1; c < n; ++c) {
      long double d = 0.0L;
      for (int64_t r = 0; r < m; ++r) d += Q[IDX(r, j, m)] * Q[IDX(r, c, m)];
      R[IDX(j, c, ldr)] = (double)d;
      for (int64_t r = 0; r < m; ++r) Q[IDX(r, c, m)] -= d * Q[IDX(r, j, m)];
    }
  }
  free(Q);
  return 0;
}

/* ||A - Q R||_F / ||A||_F in long double, Q thin m x n, R the n x n upper
 * triangle of the first n rows of Rsrc (entries below its diagonal ignored). */
double oracle_fact_residual(int64_t m, int64_t n, const double *A, int64_t lda, const double *Q,
                            int64_t ldq, const double *Rsrc, int64_t ldr) {
  long double num = 0.0L, den = 0.0L;
#pragma omp parallel for reduction(+ : num, den) schedule(static)
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t r = 0; r < m; ++r) {
      long double s = A[IDX(r, c, lda)];
      den += s * s;
      for (int64_t p = 0; p <= c; ++p) s -= (long double)Q[IDX(r, p, ldq)] * Rsrc[IDX(p, c, ldr)];
      num += s * s;
    }
  }
  return (double)(sqrtl(num) / sqrtl(den));
}

/* ||I - Q^T Q||_F in long double for an m x n Q. */
double oracle_orth_residual(int64_t m, int64_t n, const double *Q, int64_t ldq) {
  long double acc = 0.0L;
#pragma omp parallel for reduction(+ : acc) schedule(dynamic, 4)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i <= j; ++i) {
      long double s = (i == j) ? 1.0L : 0.0L;
      for (int64_t r = 0; r < m; ++r) s -= (long double)Q[IDX(r, i, ldq)] * Q[IDX(r, j, ldq)];
      acc += (i == j) ? s * s : 2.0L * s * s;
    }
  }
  return (double)sqrtl(acc);
}

/* ---------------------------------------------------------------------------
 * Cholesky factorization A = L L^T (the sister factorization the paper names
 * for the same tile framework and tuner, Secs. 1 and 7), by its definition
 * column by column: L_jj = sqrt(A_jj - sum_{k<j} L_jk^2), and for i > j
 * L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj. In place on the lower triangle
 * of A (n x n, lda); the strict upper triangle is left as it was. Returns 0,
 * or j + 1 when the pivot of column j is not positive (A is not positive
 * definite; columns >= j are then unchanged). */
int oracle_potrf(int64_t n, double *A, int64_t lda) {
  for (int64_t j = 0; j < n; ++j) {
    double d = A[IDX(j, j, lda)];
    for (int64_t k = 0; k < j; ++k) d -= A[IDX(j, k, lda)] * A[IDX(j, k, lda)];
    if (!(d > 0.0)) return (int)(j + 1);
    const double ljj = sqrt(d);
    A[IDX(j, j, lda)] = ljj;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < n; ++i) {
      double s = A[IDX(i, j, lda)];
      for (int64_t k = 0; k < j; ++k) s -= A[IDX(i, k, lda)] * A[IDX(j, k, lda)];
      A[IDX(i, j, lda)] = s / ljj;
    }
  }
  return 0;
}

/* ||A - L L^T||_F / ||A||_F in long double over the full symmetric A (both
 * triangles of the n x n A are read; only the lower triangle of L). */
double oracle_chol_residual(int64_t n, const double *A, int64_t lda, const double *L, int64_t ldl) {
  long double num = 0.0L, den = 0.0L;
#pragma omp parallel for reduction(+ : num, den) schedule(dynamic, 4)
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < n; ++i) {
      long double s = A[IDX(i, j, lda)];
      den += s * s;
      const int64_t kmax = i < j ? i : j;
      for (int64_t k = 0; k <= kmax; ++k) s -= (long double)L[IDX(i, k, ldl)] * L[IDX(j, k, ldl)];
      num += s * s;
    }
  }
  return (double)(sqrtl(num) / sqrtl(den));
}
