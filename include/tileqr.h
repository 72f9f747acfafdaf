/*
 * tileqr.h -- C ABI of the GB300 tile Householder QR library.
 *
 * The method is the tile QR factorization whose two tuning parameters, the
 * tile size NB and the inner blocking IB, are tuned empirically in
 * Agullo, Dongarra, Nath, Tomov, "A Fully Empirical Autotuned Dense QR
 * Factorization for Multicore Architectures" (INRIA RR-7526):
 *   - Sec. 2.1: a matrix of order N is split into NT x NT tiles of order NB;
 *     QR is a DAG of four tile kernels (GEQRT, TSQRT, UNMQR = DLARFB,
 *     TSMQR = DSSRFB) over the tiles (flat-tree elimination).
 *   - Sec. 2.2: IB trades memory traffic for extra flops; performance is
 *     P = (4/3) N^3 / t, independent of IB (Problem 2.1 asks for the NB-IB
 *     pair maximising P).
 *
 * Conventions for every entry point:
 *   - Matrices are column-major with a leading dimension (lda >= m).
 *   - Pointers named d_* are DEVICE pointers; the caller allocates them
 *     (the library never allocates device memory) and keeps them alive until
 *     the work queued on `stream` completes. `stream` is a cudaStream_t
 *     passed as void* (NULL = legacy default stream).
 *   - Calls are asynchronous with respect to the host unless stated.
 *   - Return value (LAPACK info style): 0 = success; -i = argument i is
 *     invalid (checked on the host before anything is queued);
 *     > 0 = a CUDA runtime error code raised while queueing work.
 *   - Conditions found on the device (a dependency wait that timed out, a
 *     non-finite column norm) are recorded in a status word inside the
 *     scratch buffer and read back with qr_status(); nothing traps the GPU.
 */
#ifndef TILEQR_H
#define TILEQR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Element types of the working precision (prec arguments). */
#define QR_PREC_F64 0
#define QR_PREC_F32 1

/* Device status bits (qr_status). */
#define QR_DEV_TIMEOUT   1 /* a scheduler dependency wait ran out of time */
#define QR_DEV_NONFINITE 2 /* a column norm or pivot was Inf/NaN */

/* Options (qr_set_option). */
#define QR_OPT_WAIT_TIMEOUT_US 1 /* per-wait limit of the persistent scheduler (default 20 s) */
#define QR_OPT_CTAS_PER_SM     2 /* resident CTAs per SM of the persistent kernel (0 = max) */
#define QR_OPT_SPLIT           3 /* column chunks per update task (0 = automatic) */
#define QR_OPT_GRID_LIMIT      4 /* cap on persistent CTAs (0 = all SMs); 1 = sequential */
#define QR_OPT_DROP_TASK       5 /* test hook: omit this ticket from the task list (-1 = off) */

/*
 * qr_workspace -- sizes of the caller-owned buffers of qr_factor_*.
 * m >= n >= 0 rows/columns; nb in [8, 512] the tile order NB; ib in
 * [1, min(nb, 256)] the inner blocking IB (any such ib is accepted, a ragged
 * last inner block included; the tuner's grid uses the divisors of nb in
 * [8, nb/2]); prec QR_PREC_F64 or QR_PREC_F32. nb = 0 uses the tuned pair.
 * *t_elems: elements of the T-factor array (IB x NB per tile, Sec. 2.2).
 * *scratch_bytes: bytes of the scratch buffer (tile-layout copy of A, the
 * task list, per-tile progress counters, the status word).
 */
int qr_workspace(int64_t m, int64_t n, int nb, int ib, int prec, int64_t *t_elems,
                 int64_t *scratch_bytes);

/*
 * qr_factor_d / qr_factor_s -- tile Householder QR, A = Q R (Sec. 2.1).
 * d_A (m x n, lda): overwritten with R in its upper triangle and the tile
 *   reflectors below it (tile-QR storage: GEQRT's V below the diagonal of
 *   each diagonal tile, TSQRT's V filling each tile below it).
 * nb, ib: tile order and inner blocking; nb = 0 picks (nb, ib) from the
 *   tuning table loaded by qr_tune / qr_load_table (nearest tuned N, Sec. 5.1).
 * d_T (t_elems from qr_workspace): the IB x NB triangular block factors.
 * d_scratch (scratch_bytes): caller-owned scratch; its status word is what
 *   qr_status reads.
 * Steps queued on stream: column-major -> tile layout; one persistent kernel
 * that runs the task DAG in a precomputed topological order with per-tile
 * progress counters; tile layout -> column-major.
 */
int qr_factor_d(int64_t m, int64_t n, double *d_A, int64_t lda, int nb, int ib, double *d_T,
                void *d_scratch, int64_t scratch_bytes, void *stream);
int qr_factor_s(int64_t m, int64_t n, float *d_A, int64_t lda, int nb, int ib, float *d_T,
                void *d_scratch, int64_t scratch_bytes, void *stream);

/*
 * qr_apply_qt_d / qr_apply_qt_s -- C <- Q^T C (trans = 1) or C <- Q C
 * (trans = 0) with the orthogonal factor of qr_factor_* (Sec. 2.1: Q is the
 * product, in elimination order, of every GEQRT factor Q_kk and TSQRT factor
 * Q_ik). d_A, lda, nb, ib, d_T exactly as returned by qr_factor_* for the
 * same m x n (nb = 0 looks up the tuned pair, as qr_factor did). d_C is
 * m x nrhs (ldc >= m), updated in place. Columns of C are independent; each
 * CTA of the kernel owns a chunk of them.
 */
int qr_apply_qt_d(int64_t m, int64_t n, int64_t nrhs, const double *d_A, int64_t lda, int nb, int ib,
                  const double *d_T, double *d_C, int64_t ldc, int trans, void *stream);
int qr_apply_qt_s(int64_t m, int64_t n, int64_t nrhs, const float *d_A, int64_t lda, int nb, int ib,
                  const float *d_T, float *d_C, int64_t ldc, int trans, void *stream);

/*
 * qr_status -- synchronises `stream`, then copies the device status word of
 * the factorization that last used d_scratch into *status (QR_DEV_* bits).
 */
int qr_status(const void *d_scratch, int *status, void *stream);

/* qr_set_option / qr_get_option -- process-wide settings (QR_OPT_*). */
int qr_set_option(int opt, int64_t value);
int64_t qr_get_option(int opt);

/* qr_task_count -- number of tasks of the factorization DAG (diagnostics). */
int64_t qr_task_count(int64_t m, int64_t n, int nb, int ib);

#ifdef __cplusplus
}
#endif

#endif /* TILEQR_H */
