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

/* Element types of the working precision (prec arguments). QR_PREC_TF32 and
 * QR_PREC_BF16X3 keep FP32 storage and run the factorization's UNMQR/TSMQR
 * products on the tensor cores (qr_factor_mixed_s, qr_solve_ls). */
#define QR_PREC_F64 0
#define QR_PREC_F32 1
#define QR_PREC_TF32 2   /* one TF32 product per update, FP32 accumulation */
#define QR_PREC_BF16X3 3 /* three BF16 products of split operands (hi*hi + hi*lo + lo*hi), FP32 accumulation */

/* Device status bits (qr_status). */
#define QR_DEV_TIMEOUT   1 /* a scheduler dependency wait ran out of time */
#define QR_DEV_NONFINITE 2 /* a column norm or pivot was Inf/NaN */
#define QR_DEV_NOT_SPD   4 /* Cholesky: a pivot was not positive (chol_status gives the first such column) */
#define QR_DEV_SINGULAR  8 /* LU: a pivot was zero (lu_status gives the first such column) */

/* Options (qr_set_option). */
#define QR_OPT_WAIT_TIMEOUT_US 1 /* per-wait limit of the persistent scheduler (default 20 s) */
#define QR_OPT_CTAS_PER_SM     2 /* resident CTAs per SM of the persistent kernel (0 = max) */
#define QR_OPT_SPLIT           3 /* column chunks per update task (0 = automatic: FP64 1 up to NB 96, 2 up to 320) */
#define QR_OPT_GRID_LIMIT      4 /* cap on persistent CTAs (0 = all SMs); 1 = sequential */
#define QR_OPT_DROP_TASK       5 /* test hook: omit this ticket from the task list (-1 = off) */
#define QR_OPT_RECORD_EVENTS   6 /* 1: bracket each persistent kernel with CUDA events on its stream */
#define QR_OPT_ORDER           7 /* flat-tree ticket order: 0 earliest start time, 1 list schedule (default) */
#define QR_OPT_PANEL_WEIGHT    8 /* list schedule: GEQRT/TSQRT cost as a percentage of their flops (default 150) */
#define QR_OPT_UNMQR_WEIGHT    9 /* list schedule: UNMQR cost as a percentage of its flops (default 100) */
#define QR_OPT_LS_REFINE      10 /* qr_solve_ls refinement: 0 automatic (F32 augmented, TF32/BF16X3 GMRES-IR), 1 augmented, 2 GMRES-IR */
#define QR_OPT_GMRES_MAX      11 /* GMRES-IR: Krylov dimension per refinement step (default 50, at most QR_GMRES_MAX_DIM) */
#define QR_OPT_GMRES_TOL_EXP  12 /* GMRES-IR: inner relative residual target 10^-value (default 6) */
#define QR_GMRES_MAX_DIM      64
#define QR_OPT_SM_BUDGET      13 /* SMs the persistent factorizations may use (0 = all): the grid is capped at that many
                                    SMs' worth of CTAs and the list schedule plans for as many workers -- the GPU
                                    counterpart of the paper's core count (Sec. 6.1); qr_tune records it per entry */
#define QR_OPT_TUNE_IB_TOL    14 /* qr_tune Step 1, in 1/1000 (default 0 = Property 5.1 as stated: the best IB per NB
                                    only): each preselected NB also keeps every IB whose kernel rate is within this
                                    fraction of its best IB's, so that Step 2 decides between them */

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
 *   tuning table loaded by qr_tune / qr_load_table (nearest tuned N, Sec. 6.1).
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
 * qr_factor_mixed_s -- FP32 tile QR whose trailing-update products (UNMQR and
 * TSMQR, the paper's DLARFB and DSSRFB) run at precision prec:
 * QR_PREC_F32 (FP32 cores, the same as qr_factor_s / qr_factor_p_s),
 * QR_PREC_TF32 or QR_PREC_BF16X3 (warp-level tensor-core products, FP32
 * accumulation; tasks with more than 512 rows, IB > 32 or that do not fit
 * the shared-memory budget, and the triangle-on-triangle TTMQR updates, stay
 * on the FP32 cores). The panel kernels (norms, beta, tau in FP64; V and T)
 * are those of qr_factor_s. p >= 1 panel domains (1 = flat tree, as
 * qr_factor_s; p > 1 as qr_factor_p_s). Buffers sized by qr_workspace
 * (p = 1) or qr_workspace_p with QR_PREC_F32; output layout as qr_factor_s,
 * so qr_apply_qt_s / qr_apply_qt_p_s apply its Q. -7: bad p, -8: bad prec;
 * otherwise the return codes of qr_factor_s (p = 1) or qr_factor_p_s.
 */
int qr_factor_mixed_s(int64_t m, int64_t n, float *d_A, int64_t lda, int nb, int ib, int p, int prec, float *d_T,
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
 * qr_apply_workspace / qr_apply_qt_ws_d / qr_apply_qt_ws_s -- the same
 * product as qr_apply_qt_* (trans = 1: C <- Q^T C, 0: C <- Q C), scheduled
 * like the factorization's updates: C takes the place of a trailing tile
 * column, UNMQR on its row block k and TSMQR on its row blocks (k, i) run
 * as tasks of a persistent kernel that waits on per-row-block counters, so
 * few right-hand sides still spread over many SMs (successive elimination
 * steps proceed as a wavefront). Column chunks of at most 64 columns are
 * separate tasks. d_scratch (bytes from qr_apply_workspace for the same m, n,
 * nrhs, nb) is caller-owned; the task list is uploaded and the counters
 * cleared on every call. Arguments otherwise as qr_apply_qt_*; -12: no
 * scratch, -13: scratch too small.
 */
int qr_apply_workspace(int64_t m, int64_t n, int64_t nrhs, int nb, int64_t *bytes);
int qr_apply_qt_ws_d(int64_t m, int64_t n, int64_t nrhs, const double *d_A, int64_t lda, int nb, int ib,
                     const double *d_T, double *d_C, int64_t ldc, int trans, void *d_scratch, int64_t scratch_bytes,
                     void *stream);
int qr_apply_qt_ws_s(int64_t m, int64_t n, int64_t nrhs, const float *d_A, int64_t lda, int nb, int ib,
                     const float *d_T, float *d_C, int64_t ldc, int trans, void *d_scratch, int64_t scratch_bytes,
                     void *stream);

/*
 * Tile QR with p domains per panel (the paper's third tunable for
 * tall-skinny matrices, communication-avoiding QR, Sec. 7).
 * qr_workspace_p / qr_factor_p_d / qr_factor_p_s: as qr_workspace /
 *   qr_factor_*, with p >= 1 domains: at step k the tile rows k..MT-1 are
 *   cut into ranges of ceil(MT/p) rows starting at row k (the domains slide
 *   down with the panel), each eliminated by its own flat tree (GEQRT on its
 *   first tile, TSQRT down the range, UNMQR/TSMQR updates), and the
 *   triangles are merged by a binary tree of triangle-on-triangle steps
 *   (TTQRT, with TTMQR updates). p = 1 is the
 *   flat tree of qr_factor_* (same arithmetic). A ragged last tile row is
 *   never a domain head. Output: R in the upper triangle of d_A; below it the
 *   reflectors; a domain head's tile keeps its GEQRT reflectors below the
 *   diagonal and, once its triangle is merged away, the TTQRT reflectors in
 *   its upper triangle. d_T holds t_elems = 2 x MT x NT x IB x NB elements
 *   (GEQRT/TSQRT factors, then TTQRT factors). Scratch as qr_workspace_p
 *   reports (it includes the explicit task list). -7: p out of [1, 4096].
 * qr_apply_workspace_p / qr_apply_qt_p_d / qr_apply_qt_p_s: C <- Q^T C
 *   (trans = 1) or Q C for the factors of qr_factor_p_* with the same
 *   (m, n, nb, ib, p); a persistent kernel over C's row blocks with explicit
 *   dependencies. -8: bad p; -13: no scratch; -14: scratch too small.
 */
int qr_workspace_p(int64_t m, int64_t n, int nb, int ib, int p, int prec, int64_t *t_elems,
                   int64_t *scratch_bytes);
int qr_factor_p_d(int64_t m, int64_t n, double *d_A, int64_t lda, int nb, int ib, int p, double *d_T,
                  void *d_scratch, int64_t scratch_bytes, void *stream);
int qr_factor_p_s(int64_t m, int64_t n, float *d_A, int64_t lda, int nb, int ib, int p, float *d_T,
                  void *d_scratch, int64_t scratch_bytes, void *stream);
int qr_apply_workspace_p(int64_t m, int64_t n, int64_t nrhs, int nb, int p, int64_t *bytes);
int qr_apply_qt_p_d(int64_t m, int64_t n, int64_t nrhs, const double *d_A, int64_t lda, int nb, int ib, int p,
                    const double *d_T, double *d_C, int64_t ldc, int trans, void *d_scratch, int64_t scratch_bytes,
                    void *stream);
int qr_apply_qt_p_s(int64_t m, int64_t n, int64_t nrhs, const float *d_A, int64_t lda, int nb, int ib, int p,
                    const float *d_T, float *d_C, int64_t ldc, int trans, void *d_scratch, int64_t scratch_bytes,
                    void *stream);

/*
 * qr_factor_d_noalloc -- qr_factor_d for callers that cannot allocate device
 * memory: code running where cudaMalloc is not allowed or not wanted, such
 * as a plug-in handed pointers by a host application that owns every
 * allocation, or a real-time loop that must not allocate. It takes no
 * scratch buffer and calls no allocation routine; the paper has no
 * counterpart (it is a convenience of this library).
 * Its scratch is a fixed device array of QR_NOALLOC_SCRATCH_BYTES bytes
 * compiled into the library; every GPU that loads the library holds it until
 * the process exits. Problems whose scratch (as qr_workspace would report)
 * exceeds that size are rejected with QR_NOALLOC_TOO_LARGE before anything
 * is queued (for example 1024 x 1024 with nb = 64 fits; 4096 x 4096 does
 * not); that code lies outside the -1..-9 range of argument errors.
 * Arguments as qr_factor_d; d_A and d_T are the caller's input/output.
 * nb = 0 takes (nb, ib) from the tuning table as qr_factor_d does, but always
 * runs the flat tree: for tall-skinny shapes the table's pair was tuned
 * together with p > 1 panel domains, so it may not be the fastest here.
 * d_status (device int, may be NULL) receives the QR_DEV_* bits of this call.
 * The first call in each CUDA context (each device, and again after
 * cudaDeviceReset) looks up the array's device address
 * (cudaGetSymbolAddress) with that context current; make that first call
 * before any stream capture. All calls share the one array: calls that
 * overlap on the GPU (concurrent streams, several host threads) race and
 * corrupt each other -- serialise them. Each call clears the status word,
 * ticket and counters it needs; tasks run in the DAG's program order.
 */
#define QR_NOALLOC_SCRATCH_BYTES (16u << 20)
#define QR_NOALLOC_TOO_LARGE (-100)
int qr_factor_d_noalloc(int64_t m, int64_t n, double *d_A, int64_t lda, int nb, int ib, double *d_T,
                        int *d_status, void *stream);

/*
 * qr_status -- synchronises `stream`, then copies the device status word of
 * the factorization that last used d_scratch into *status (QR_DEV_* bits).
 */
int qr_status(const void *d_scratch, int *status, void *stream);

/*
 * qr_set_task_costs -- measured costs of the four task types (GEQRT, UNMQR,
 * TSQRT, TSMQR: any time unit, e.g. median service times from qr_set_trace)
 * for factorizations at precision prec with this (nb, ib). The host list
 * schedule that orders the persistent kernel's tickets then uses them in
 * place of its flop-count weights (QR_OPT_PANEL_WEIGHT, QR_OPT_UNMQR_WEIGHT).
 * costs = NULL removes the entry. Returns -1..-3 for a bad prec, nb, ib and
 * -4 for a cost that is not positive and finite.
 */
int qr_set_task_costs(int prec, int nb, int ib, const double *costs);

/*
 * qr_set_trace -- per-task trace of the persistent factorization and Q
 * application kernels (diagnostics; the paper's runs are timed as a whole).
 * d_buf: device array (32-byte aligned) of `capacity` records of four
 * uint64: task index in the launch's ticket order (bits 0..39), task type
 * (bits 40..47: 0 GEQRT, 1 UNMQR, 2 TSQRT, 3 TSMQR, 4 TTQRT, 5 TTMQR) and SM
 * id (bits 48..63); %globaltimer (ns) when the ticket was taken, when the
 * task's dependencies were met, and when its completion was published. Every later
 * launch of persistent_qr, persistent_qr_dag or persistent_apply_dag writes
 * record t for its task t < capacity (overwriting the previous launch's);
 * the caller owns the buffer and reads it after synchronising. NULL (or
 * capacity 0) turns tracing off. Returns -1 for a misaligned buffer, -2 for
 * a negative capacity.
 */
int qr_set_trace(void *d_buf, int64_t capacity);

/* qr_set_option / qr_get_option -- process-wide settings (QR_OPT_*). */
int qr_set_option(int opt, int64_t value);
int64_t qr_get_option(int opt);

/*
 * qr_last_kernel_ms -- with QR_OPT_RECORD_EVENTS on, waits for and returns
 * the device time (ms, CUDA events on the launching stream) of the most
 * recent persistent factorization kernel. -2 if none was recorded.
 */
int qr_last_kernel_ms(float *ms);

/*
 * qr_peak_fp64 -- measures the FP64 fused multiply-add throughput of the
 * current device with a register-resident kernel (independent FMA chains on
 * every SM, timed with CUDA events on `stream`, synchronous). *gflops gets
 * the rate in GFLOP/s (2 flops per FMA). Used as a live roofline reference.
 */
int qr_peak_fp64(double *gflops, void *stream);

/*
 * Batched QR of many small matrices of uneven sizes (one persistent launch;
 * batching is this library's extension of the paper's single-matrix QR).
 * qr_batched_plan (host only): for count matrices of sizes m[b] x n[b]
 *   (1 <= n <= m <= 65535) picks (nb, ib) per matrix from its size class
 *   (qr_batched_set_class; force_nb > 0 overrides with (force_nb, force_ib)),
 *   orders the matrices by decreasing flop count (largest first), and lays
 *   out the T factors: t_offset_out[b] elements into one T array of
 *   *t_total elements. All outputs are host arrays of count entries.
 * qr_factor_batched_d / _s: every pointer argument is a DEVICE array of
 *   count entries (d_A: device pointers to the column-major matrices, each
 *   overwritten like qr_factor's output; d_lda; d_nb, d_ib, d_order,
 *   d_t_offset as planned; d_T the T array). d_scratch: >= 256 bytes,
 *   caller-owned (work counter + status word). Queues a memset and one
 *   kernel on `stream`, so a call can be captured in a CUDA graph.
 *   Each matrix is factored by one CTA in the flat-tree tile order of
 *   Sec. 2.1 with its (nb, ib); qr_apply_qt_* with (m[b], n[b], nb=min(nb,m),
 *   ib, T + t_offset[b]) applies its Q.
 * qr_batched_set_class / qr_batched_clear_classes: the size-class table:
 *   matrices with m <= m_hi (smallest such class) use (nb, ib); the default
 *   is one tile per matrix with IB 16.
 * qr_batched_status: synchronises `stream`, reads the status word
 *   (QR_DEV_NONFINITE) of the last batched factorization using d_scratch.
 */
int qr_batched_plan(int count, const int *m, const int *n, int prec, int force_nb, int force_ib, int *nb_out,
                    int *ib_out, int *order_out, int64_t *t_offset_out, int64_t *t_total);
int qr_factor_batched_d(int count, const int *d_m, const int *d_n, double *const *d_A, const int *d_lda,
                        double *d_T, const int64_t *d_t_offset, const int *d_nb, const int *d_ib,
                        const int *d_order, void *d_scratch, void *stream);
int qr_factor_batched_s(int count, const int *d_m, const int *d_n, float *const *d_A, const int *d_lda,
                        float *d_T, const int64_t *d_t_offset, const int *d_nb, const int *d_ib,
                        const int *d_order, void *d_scratch, void *stream);
int qr_batched_set_class(int prec, int m_hi, int nb, int ib);
int qr_batched_clear_classes(int prec);
int qr_batched_status(const void *d_scratch, int *status, void *stream);

/*
 * qr_solve_ls_workspace / qr_solve_ls -- min ||A X - B||_F through the tile
 * QR (least squares is the QR's use beyond the paper, which tunes the
 * factorization only). A (m x n, m >= n, full rank), B (m x nrhs) and X
 * (n x nrhs) are FP64 device arrays; A and B are not modified.
 * prec = QR_PREC_F64: QR of an FP64 copy of A, X = R^{-1} (Q^T B)(0:n)
 *   (max_iter > 0 adds FP64 refinement as below).
 * prec = QR_PREC_F32 / QR_PREC_TF32 / QR_PREC_BF16X3: QR of an FP32 copy of
 *   A (FP64 kept in the panel's Householder vector / tau generation), its
 *   UNMQR/TSMQR products on the FP32 cores (F32) or the tensor cores (TF32,
 *   BF16X3, as qr_factor_mixed_s), then refinement of the augmented system
 *   [I A; A^T 0][r; x] = [b; 0] (Bjorck) with FP64 residuals
 *   f = b - r - A x, g = -A^T r and FP64 accumulation of x and r. The
 *   correction M^-1 [f; g] through the low-precision factors solves
 *   R^T h = g, d = Q^T f, R dx = d(0:n) - h, dr = Q [h; d(n:m)].
 *   Scheme (QR_OPT_LS_REFINE; automatic: augmented refinement for F32,
 *   GMRES-IR for TF32 and BF16X3): augmented refinement adds that
 *   correction each step; GMRES-IR (Carson, Higham and Pranesh) solves
 *   K [dr; dx] = [f; g], K the augmented matrix, each step by FP64 GMRES on
 *   M^-1 K to a relative residual of 10^-QR_OPT_GMRES_TOL_EXP or at most
 *   QR_OPT_GMRES_MAX iterations -- needed where kappa(A) u > 1 for the
 *   factorization's precision (TF32: u = 2^-11, BF16X3: about 2^-17, so
 *   kappa = 1e6 is beyond plain refinement). Stops when every column has
 *   ||dx|| <= tol ||x||, when the corrections stop shrinking (augmented:
 *   none halves any more from step 3 on; GMRES-IR: none shrinks tenfold
 *   from step 2 on), or after max_iter steps.
 * nb, ib: tile order / inner blocking of the factorization (0 = tuned table).
 * p: panel domains of the factorization (qr_factor_p_*); 0 picks
 *   ceil(MT / NT) tile-row ranges per panel, at most 32 (1 = flat tree).
 * info[4] (may be NULL): refinement steps taken (max over RHS groups); 1 if
 *   every column met ||dx|| <= tol ||x|| (1 also for a plain solve), 2 if
 *   the corrections stopped shrinking as above (the limiting accuracy of
 *   FP64 residuals is reached), 0 if max_iter ran out first; device status
 *   bits (QR_DEV_*: of the factorization, and QR_DEV_TIMEOUT from the
 *   triangular solves, whose row blocks wait on each other with the same
 *   bounded waits as the scheduler); GMRES iterations in total (0 for
 *   augmented refinement).
 * d_work (>= qr_solve_ls_workspace bytes) is caller-owned. Synchronises
 * `stream` once per refinement step (stopping test), once per GMRES
 * iteration, and at the end.
 */
int qr_solve_ls_workspace(int64_t m, int64_t n, int64_t nrhs, int prec, int nb, int ib, int p, int64_t *bytes);
int qr_solve_ls(int64_t m, int64_t n, int64_t nrhs, const double *d_A, int64_t lda, const double *d_B, int64_t ldb,
                double *d_X, int64_t ldx, int prec, int nb, int ib, int p, int max_iter, double tol, int *info,
                void *d_work, int64_t work_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Empirical NB/IB autotuner (Secs. 5–6 of the paper).
 * ------------------------------------------------------------------------ */

/*
 * qr_tune -- install-time tuning (Sec. 7: "make autotune", then an instant
 * decision at call time). Shapes (ms[i], ns[i]), nshapes >= 1.
 * mode bit 0 = 0 (PSPAYG): Step 1 = time the TSMQR kernel (the paper's
 *   DSSRFB) for every (NB, IB) of the grid NB in {64..512 step 32}, IB | NB,
 *   8 <= IB <= NB/2 (119 pairs), up to 50 launches each (Sec. 5);
 *   Property 5.1 (best IB per NB), Property 5.2 (upper convex hull) and
 *   Heuristic `heuristic` (0, 1 or 2; 2 is the paper's default) preselect at
 *   most 8 pairs (with QR_OPT_TUNE_IB_TOL > 0 each preselected NB also
 *   brings the IBs within that tolerance of its best IB's rate, a widening
 *   of Property 5.1 that this library adds); Step 2 = time qr_factor for the
 *   survivors at every shape,
 *   ascending n, `reps` runs each (median; the paper uses 6, Sec. 6.1), and
 *   prune as you go with Property 6.1 between square orders (Sec. 6.3).
 *   For tall-skinny shapes (m >= 4n, at least 4 tile rows) the chosen pair
 *   is then timed with p = 2, 4, ... panel domains (qr_factor_p_*; at most
 *   64 and 2 MT/NT), the paper's third tunable for such matrices; the
 *   table records the best p (1 = flat tree).
 * mode bit 0 = 1 (exhaustive search, ES): Step 2 over the whole grid, no
 *   pruning.
 * mode bit 1 (value 2): Step 1 as MultCallFlushLRU -- each launch works on
 *   its own copy of the operands, taken in turn from enough copies that its
 *   data was last touched two L2 capacities ago (the paper reports "No
 *   Flush", where every launch reuses the same data, and leaves the flushing
 *   variants out of scope, Sec. 5). Logged as kind 5 instead of 1.
 * use_model = k in [1, 8] (0 = off; this library's addition, the paper
 *   tunes without a model): the learned cost model (qr_mlp_*), fitted on
 *   the GPU to the Step-2 timings of the orders already done (features
 *   log m, log n, NB/512, IB/256; target log seconds), ranks the survivors
 *   of each square order from the third square order on, and only the k it
 *   ranks fastest are timed; the search goes further down the ranking while
 *   the last pair timed is the fastest so far, and times every survivor when
 *   the model's relative predictions are off (measured / predicted of a
 *   timed pair differs from that of the top-ranked pair by more than a factor
 *   e^0.25). Other shapes are timed in full. Measurements always
 *   decide; a survivor left untimed is not pruned. The final model, fitted
 *   to all Step-2 timings, is saved in the table ("model") and answers
 *   qr_model_propose. Predictions are logged as kind 4.
 * prec: QR_PREC_F64 / QR_PREC_F32. table_path (may be NULL/""): JSON decision
 * table written at the end; it also becomes the in-process table used by
 * nb = 0. log_path (may be NULL/""): JSONL of every measurement, appended;
 * measurements already in it are reused, so an interrupted run resumes.
 * d_work (work_bytes >= qr_tune_workspace): device scratch owned by the
 * caller; its first QR_MODEL_WORK_BYTES hold the model's buffers.
 * seconds_out[6] (may be NULL): total, Step-1 and Step-2 wall seconds, the
 * number of factorizations timed in this call, the seconds spent fitting
 * and evaluating the model, and the orders where the model's check fell
 * back to timing every survivor. Synchronous. Errors: -4 heuristic, -5 mode,
 * -6 use_model, -7 reps, -8 prec, -9 table not writable, -11 no d_work,
 * -12 d_work too small.
 */
#define QR_MODEL_WORK_BYTES (4ll << 20)
int qr_tune(const int64_t *ms, const int64_t *ns, int nshapes, int heuristic, int mode, int use_model, int reps,
            int prec, const char *table_path, const char *log_path, void *d_work, int64_t work_bytes,
            double *seconds_out, void *stream);

/*
 * qr_model_propose -- (nb, ib) for an untuned shape m x n from the learned
 * cost model saved by the last qr_tune with use_model > 0 (or loaded with
 * its table by qr_load_table): the pair of the model's candidate set (the
 * tuner's preselected pairs) with the least predicted time, which goes to
 * *seconds (may be NULL). d_work: device scratch of at least
 * QR_MODEL_WORK_BYTES. Synchronous. Returns 1 when no model is loaded for
 * prec (nothing written), -8 for a d_work that is too small.
 */
int qr_model_propose(int64_t m, int64_t n, int prec, int *nb, int *ib, double *seconds, void *d_work,
                     int64_t work_bytes, void *stream);

/* qr_tune_workspace -- device bytes qr_tune needs for shapes up to max_m x max_n. */
int qr_tune_workspace(int64_t max_m, int64_t max_n, int prec, int64_t *bytes);

/*
 * qr_load_table / qr_clear_tables / qr_lookup -- the decision table. A
 * request for an untuned shape uses the closest tuned one (Sec. 6.1: the
 * closest benchmarked configuration), distance |m - m_i| + |n - n_i|, ties
 * to the smaller tuned shape, among the entries of the SM budget closest to
 * QR_OPT_SM_BUDGET (see qr_lookup_sms); with no table the built-in pair
 * (128, 16).
 * prec selects the fp64 or fp32 table (fp32 falls back to fp64's).
 */
int qr_load_table(const char *path);
int qr_clear_tables(void);
int qr_lookup(int64_t m, int64_t n, int prec, int *nb, int *ib);
/* qr_lookup_p -- as qr_lookup, and *p the tuned panel domains for
 * qr_factor_p_* (1 where the table has none: the flat tree). */
int qr_lookup_p(int64_t m, int64_t n, int prec, int *nb, int *ib, int *p);
/*
 * qr_lookup_sms -- the tuned (nb, ib, p) for an m x n problem on an SM
 * budget of sms SMs (0 = the whole GPU), the GPU reading of the paper's
 * (N, ncores) table (Sec. 6.1): the closest tuned budget first (ties to the
 * smaller), then the closest tuned shape of that budget, as in the paper's
 * example where N = 1800 on 5 cores takes the point tuned for N = 2000 on 4.
 * Table entries carry the budget they were tuned under ("sms"; qr_tune
 * records QR_OPT_SM_BUDGET, 0 = whole GPU). nb = 0 in qr_factor_* looks up
 * with the current QR_OPT_SM_BUDGET. p may be NULL. TF32/BF16X3 use the fp32
 * table. With no table: (128, 16, 1).
 */
int qr_lookup_sms(int64_t m, int64_t n, int prec, int sms, int *nb, int *ib, int *p);

/*
 * Host-only decision rules of the tuner (no GPU call), exported so that they
 * can be checked on their own:
 * qr_tune_grid -- the (NB, IB) grid (NB in nb_lo..nb_hi step nb_step, IB a
 *   divisor of NB in [ib_min, NB/2]); writes up to cap pairs, returns the count.
 * qr_tune_preselect -- Property 5.1, the upper hull (Property 5.2) and
 *   Heuristic 0/1/2 over npairs Step-1 results; writes the preselected
 *   pairs (ascending NB) and returns how many (<= max_sel for H1/H2;
 *   nseg iso-segments for H2).
 * qr_tune_payg -- Property 6.1: keep[a] = 0 iff some pair with larger NB has
 *   strictly higher performance at the order just measured.
 * qr_tune_nearest -- the closest grid value (ties to the smaller), Sec. 6.1.
 */
int qr_tune_grid(int nb_lo, int nb_hi, int nb_step, int ib_min, int cap, int *nbs, int *ibs);
int qr_tune_preselect(int npairs, const int *nb, const int *ib, const double *perf, int heuristic, int max_sel,
                      int nseg, int *sel_nb, int *sel_ib);
int qr_tune_payg(int nsurv, const int *nb, const double *perf, int *keep);
int64_t qr_tune_nearest(int64_t value, const int64_t *grid, int ngrid);

/*
 * qr_step1_workspace / qr_step1_time -- the Step-1 kernel benchmark of Sec. 5
 * for one (nb, ib): `launches` back-to-back launches of a batch of
 * 2 x (SM count) independent TSMQR tile tasks, timed with CUDA events on
 * `stream`; synchronous. flush = 0: "No Flush" (same data every launch, the
 * paper's reported mode); flush = 1: MultCallFlushLRU (launch l uses
 * operand copy l mod c, with c copies covering at least two L2 capacities
 * plus one copy, at least 2: each launch reads its operands from HBM).
 * launches <= 0 picks the count from one timed launch: enough launches for
 * about 30 ms, at least 3 and at most the paper's 50. prec QR_PREC_TF32 /
 * QR_PREC_BF16X3 time the FP32 task with its products on the tensor cores
 * (the update of qr_factor_mixed_s).
 * *seconds_per_launch, and *gflops (may be NULL) = batch x 4 NB^3 / time.
 */
int qr_step1_workspace(int nb, int prec, int flush, int64_t *bytes);
int qr_step1_time(int nb, int ib, int prec, int launches, int flush, double *seconds_per_launch, double *gflops,
                  void *d_work, int64_t work_bytes, void *stream);

/*
 * qr_time_factor -- the Step-2 measurement: qr_factor at (m, n, nb, ib) on a
 * device-generated uniform[-0.5, 0.5) matrix regenerated before each run,
 * reps timed runs (CUDA events around each call; the host task order is
 * built beforehand, and problems of at most 4e6 elements get one untimed
 * warm-up run), median and minimum seconds.
 * d_work must hold A (m x n), T and the factorization scratch.
 */
int qr_time_factor(int64_t m, int64_t n, int nb, int ib, int prec, int reps, double *median_s, double *min_s,
                   void *d_work, int64_t work_bytes, void *stream);
/* qr_time_factor_p -- the same measurement of qr_factor_p_* with p domains. */
int qr_time_factor_p(int64_t m, int64_t n, int nb, int ib, int p, int prec, int reps, double *median_s,
                     double *min_s, void *d_work, int64_t work_bytes, void *stream);

/*
 * Learned cost model of the tuner (this library's addition; the paper tunes
 * without a model, Secs. 1 and 2.3). A 4 -> 64 -> 64 -> 1 perceptron with ReLU
 * hidden layers, FP32, mapping standardized (log m, log n, NB/512, IB/256)
 * to log(seconds). d_params: QR_MLP_NPARAMS floats laid out W1 (64 x 4,
 * row-major [out][in]), b1 (64), W2 (64 x 64), b2 (64), W3 (1 x 64), b3 (1).
 * d_X: nsamp x 4 row-major; d_y: nsamp targets. Device pointers, async.
 * qr_mlp_workspace: floats of scratch d_work needed by grad/train for nsamp.
 * qr_mlp_forward: d_out[s] = prediction for sample s.
 * qr_mlp_grad: d_grads (QR_MLP_NPARAMS + 1 floats) = gradient of
 *   mean((yhat - y)^2) followed by the loss itself.
 * qr_mlp_adam_step: one Adam update (beta1 0.9, beta2 0.999, eps 1e-8,
 *   bias-corrected, step t >= 1) of d_params with moments d_m, d_v.
 * qr_mlp_train: `steps` full-batch gradient + Adam steps (t = 1..steps).
 */
#define QR_MLP_NPARAMS 4545
int qr_mlp_workspace(int nsamp, int64_t *floats);
int qr_mlp_forward(int nsamp, const float *d_X, const float *d_params, float *d_out, void *stream);
int qr_mlp_grad(int nsamp, const float *d_X, const float *d_y, const float *d_params, float *d_grads, float *d_work,
                void *stream);
int qr_mlp_adam_step(const float *d_grads, float *d_params, float *d_m, float *d_v, int t, float lr, void *stream);
int qr_mlp_train(int nsamp, const float *d_X, const float *d_y, float *d_params, float *d_m, float *d_v, int steps,
                 float lr, float *d_grads, float *d_work, void *stream);

/* ------------------------------------------------------------------------
 * Tile Cholesky A = L L^T on the same persistent scheduler, with its own
 * empirical NB tuner (the paper names Cholesky and LU as the factorizations
 * its framework and tuning method carry over to, Secs. 1 and 7; it tunes QR).
 * ------------------------------------------------------------------------ */

/*
 * chol_workspace / chol_factor_d -- FP64 tile Cholesky of the symmetric
 * positive definite n x n matrix A (column-major, lda >= n; only its lower
 * triangle is read). On return the lower triangle holds L; the strict upper
 * triangle is not touched. nb: tile order, a multiple of 16 in [16, 256]
 * (0 = the Cholesky tuning table, closest tuned order; 128 without one).
 * Tasks POTRF(k), TRSM(i, k), SYRK(i, k), GEMM(i, j, k) over the tiles of
 * the lower triangle run in one persistent kernel in a list-scheduled order,
 * each waiting (bounded) on per-tile operation counters. d_scratch
 * (chol_workspace bytes: the control block, counters, task list and the tile
 * copy of A) is caller-owned. Queues: layout conversion, the persistent
 * kernel, conversion of the lower triangle back. Errors: -1 n, -2 A, -3 lda,
 * -4 nb, -5 no scratch, -6 scratch too small.
 * chol_status: synchronises `stream`; *status gets the QR_DEV_* bits of the
 * last factorization that used d_scratch (QR_DEV_NOT_SPD, QR_DEV_TIMEOUT),
 * *first_bad_col (may be NULL) the smallest column whose pivot was not
 * positive, or -1.
 * chol_task_count_n: tasks of the DAG for (n, nb).
 */
int chol_workspace(int64_t n, int nb, int64_t *bytes);
int chol_factor_d(int64_t n, double *d_A, int64_t lda, int nb, void *d_scratch, int64_t scratch_bytes, void *stream);
int chol_status(const void *d_scratch, int *status, int64_t *first_bad_col, void *stream);
int64_t chol_task_count_n(int64_t n, int nb);

/*
 * lu_workspace / lu_factor_d -- FP64 tile LU with incremental (pairwise)
 * pivoting of the n x n matrix A (column-major, lda >= n), in place: the LU
 * the paper names beside Cholesky as carrying its tile framework and tuning
 * method (Secs. 1 and 7; it defines no LU algorithm). Tasks, the flat-tree
 * DAG of the tile QR with LU kernels: GETRF(k) (partial pivoting inside the
 * diagonal tile), GESSM(k, j) (its swaps and eliminations applied to A_kj),
 * TSTRF(i, k) (pairwise-pivoted LU of [U_kk; A_ik]: a row of A_ik replaces
 * U_kk's row c when its |entry| in column c is strictly larger, first such
 * row on ties), SSSSM(i, j, k) (those swaps and eliminations applied to
 * [A_kj; A_ij]); swaps move columns c.. only. On return A holds U on and
 * above the diagonal and each task's multipliers below it (a sequence of
 * elementary transformations, not L of one row permutation).
 * d_piv (int32, lu_workspace's piv_elems, caller-owned output): tile (i, k)
 * column c at d_piv[(k * NT + i) * nb + c], NT = ceil(n / nb): GETRF the
 * tile row swapped with row c (c when none), TSTRF the row of A_ik swapped
 * with U_kk's row c (-1 when none); entries past a short last tile are not
 * written. nb in [8, 64] (0 = the LU tuning table; 64 without one). d_scratch (lu_workspace's scratch_bytes:
 * control block, counters, task list, tile copy of A) caller-owned. One
 * persistent kernel in a list-scheduled ticket order with bounded waits on
 * per-tile operation counters; layout conversions before and after. A zero
 * pivot sets QR_DEV_SINGULAR and its column is skipped (no division), as
 * LAPACK's getrf continues past one. Errors: -1 n, -2 A, -3 lda, -4 nb,
 * -5 no d_piv, -6 no scratch, -7 scratch too small.
 * lu_status: synchronises `stream`; *status gets the QR_DEV_* bits of the
 * last factorization that used d_scratch, *first_zero_col (may be NULL) the
 * smallest column whose pivot was zero, or -1.
 * lu_task_count_n: tasks of the DAG for (n, nb), -1 for bad arguments.
 */
int lu_workspace(int64_t n, int nb, int64_t *piv_elems, int64_t *scratch_bytes);
int lu_factor_d(int64_t n, double *d_A, int64_t lda, int nb, int *d_piv, void *d_scratch, int64_t scratch_bytes,
                void *stream);
int lu_status(const void *d_scratch, int *status, int64_t *first_zero_col, void *stream);
int64_t lu_task_count_n(int64_t n, int nb);

/*
 * The LU's NB tuner (Secs. 5–6 applied to its one tuning parameter, as for
 * the Cholesky).
 * lu_step1_time: Step 1 -- `launches` back-to-back launches (<= 0: enough
 *   for ~30 ms, 3 to 50) of a batch of 2 x (SM count) independent SSSSM tile
 *   tasks of order nb (the dominant task; every other column swaps), same
 *   data every launch; *seconds_per_launch, *gflops (2 nb^3 per task, may be
 *   NULL). d_work: lu_step1_workspace bytes. Errors: -1 nb (8..64), -3
 *   output, -5 no d_work, -7 d_work too small.
 * lu_time_factor: Step 2 -- reps timed lu_factor_d calls on fresh uniform
 *   [-0.5, 0.5) matrices of order n generated on the device (median and
 *   minimum seconds; the refill is not timed). d_work: lu_tune_workspace
 *   bytes for an order >= n.
 * lu_tune: Step 1 over NB in {16, 24, ..., 64}, the upper hull and Heuristic
 *   `heuristic` (qr_tune_preselect with IB fixed), Step 2 over the orders
 *   ns[] ascending with prune-as-you-go (qr_tune_payg), `reps` runs each;
 *   logs kind 21 (Step 1) and 22 (Step 2) to log_path (resumes from it),
 *   writes the table to table_path and installs it in-process.
 *   seconds_out[4]: total, Step 1, Step 2, factorizations timed.
 * lu_load_table / lu_lookup / lu_clear_table: the table lu_factor_d uses
 *   for nb = 0 (closest tuned order, ties to the smaller; 64 without one).
 */
int lu_step1_workspace(int nb, int64_t *bytes);
int lu_step1_time(int nb, int launches, double *seconds_per_launch, double *gflops, void *d_work, int64_t work_bytes,
                  void *stream);
int lu_time_factor(int64_t n, int nb, int reps, double *median_s, double *min_s, void *d_work, int64_t work_bytes,
                   void *stream);
int lu_tune_workspace(int64_t max_n, int64_t *bytes);
int lu_tune(const int64_t *ns, int nshapes, int heuristic, int reps, const char *table_path, const char *log_path,
            void *d_work, int64_t work_bytes, double *seconds_out, void *stream);
int lu_load_table(const char *path);
int lu_lookup(int64_t n, int *nb);
int lu_clear_table(void);

/*
 * The Cholesky tuner (Secs. 5–6 applied to the one tuning parameter NB).
 * chol_step1_time: Step 1 -- `launches` back-to-back launches (<= 0: enough
 *   for ~30 ms, 3 to 50) of a batch of 2 x (SM count) independent GEMM tile
 *   tasks C -= A B^T of order nb (the dominant task), same data every launch;
 *   *gflops = batch x 2 nb^3 / time. Workspace: chol_step1_workspace.
 * chol_time_factor: Step 2 measurement -- reps timed factorizations of a
 *   device-generated symmetric matrix with entries uniform[-0.5, 0.5) and n
 *   added to the diagonal (diagonally dominant, so positive definite),
 *   regenerated before each run; median and minimum seconds. d_work holds
 *   the matrix and the scratch (chol_tune_workspace for n covers it).
 * chol_tune: Step 1 over NB in {32, 64, ..., 256}; the upper hull and
 *   Heuristic `heuristic` (qr_tune_preselect); Step 2 over the orders ns[]
 *   ascending, `reps` runs each, prune as you go (Property 6.1). table_path:
 *   JSON decision table (entries n, nb, GFLOP/s credited n^3 / 3); it also
 *   becomes the in-process table of nb = 0. log_path: JSONL of every
 *   measurement (kind 11 Step 1, 12 Step 2), reused by a later run.
 *   seconds_out[4]: total, Step 1, Step 2 seconds, factorizations timed.
 * chol_load_table / chol_lookup: the decision table; closest tuned order.
 */
int chol_step1_workspace(int nb, int64_t *bytes);
int chol_step1_time(int nb, int launches, double *seconds_per_launch, double *gflops, void *d_work, int64_t work_bytes,
                    void *stream);
int chol_time_factor(int64_t n, int nb, int reps, double *median_s, double *min_s, void *d_work, int64_t work_bytes,
                     void *stream);
int chol_tune_workspace(int64_t max_n, int64_t *bytes);
int chol_tune(const int64_t *ns, int nshapes, int heuristic, int reps, const char *table_path, const char *log_path,
              void *d_work, int64_t work_bytes, double *seconds_out, void *stream);
int chol_load_table(const char *path);
int chol_lookup(int64_t n, int *nb);

/* qr_task_count -- number of tasks of the flat-tree factorization DAG at
 * precision prec (QR_PREC_*; the column split of the update tasks depends on
 * it and on QR_OPT_SPLIT). Diagnostics, and the record count of a trace. */
int64_t qr_task_count(int64_t m, int64_t n, int nb, int ib, int prec);

#ifdef __cplusplus
}
#endif

#endif /* TILEQR_H */
