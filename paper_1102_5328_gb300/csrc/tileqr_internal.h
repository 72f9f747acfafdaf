// Internal declarations shared by the library's translation units.
#pragma once
#include <array>
#include <cstdint>

#include "../../include/tileqr.h"

namespace tqr {

enum TaskType { TASK_GEQRT = 0, TASK_UNMQR = 1, TASK_TSQRT = 2, TASK_TSMQR = 3 };

// 64-bit task code: type (4 bits) | column chunk (12) | i (16) | j (16) | k (16)
__host__ __device__ inline uint64_t encode_task(int type, int s, int i, int j, int k) {
  return (uint64_t)(type & 0xF) | ((uint64_t)(s & 0xFFF) << 4) | ((uint64_t)(i & 0xFFFF) << 16) |
         ((uint64_t)(j & 0xFFFF) << 32) | ((uint64_t)(k & 0xFFFF) << 48);
}
__host__ __device__ inline void decode_task(uint64_t c, int& type, int& s, int& i, int& j, int& k) {
  type = (int)(c & 0xF);
  s = (int)((c >> 4) & 0xFFF);
  i = (int)((c >> 16) & 0xFFFF);
  j = (int)((c >> 32) & 0xFFFF);
  k = (int)((c >> 48) & 0xFFFF);
}

}  // namespace tqr

// (nb, ib) -- and the panel domains p when pd is not null -- for a shape from
// the loaded tuning table (nearest tuned shape), or the built-in default
// (128, 16, p = 1) when no table is loaded. Returns 0 on success.
int qr_table_lookup(int64_t m, int64_t n, int elem_bytes, int* nb, int* ib, int* pd = nullptr);

// Builds (and caches) the host task order for this shape so that a later
// timed qr_factor_* call does not include it. Returns 0 on success.
int qr_prepare_schedule(int64_t m, int64_t n, int nb, int ib, int prec);

// The trace buffer set by qr_set_trace (null when tracing is off) and its
// capacity in records; read at each launch of a persistent kernel.
void qr_trace_target(void** buf, int64_t* cap);

// List-schedule weights (GEQRT, UNMQR, TSQRT, TSMQR) for factorizations at
// precision prec with (nb, ib) and S column chunks: the measured costs set by
// qr_set_task_costs, else flop counts with the panel and UNMQR factors of
// QR_OPT_PANEL_WEIGHT / QR_OPT_UNMQR_WEIGHT.
std::array<double, 4> qr_task_weights(int prec, int nb, int ib, int S);

// qr_factor_p_s with the UNMQR/TSMQR products at tensor-core precision tc
// (TC_NONE, TC_TF32, TC_BF16X3 of tc_update.cuh); the same argument checks
// and return codes as qr_factor_p_s.
inline int tc_of_prec(int prec) { return prec == QR_PREC_TF32 ? 1 : (prec == QR_PREC_BF16X3 ? 2 : 0); }
int qr_factor_p_tc_s(int64_t m, int64_t n, float* A, int64_t lda, int nb, int ib, int p, float* T, void* scratch,
                     int64_t scratch_bytes, void* stream, int tc);
