// Device-side pieces shared by the persistent schedulers (factorization and
// Q application): the control block, acquire/release counter access, and the
// bounded dependency wait.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tileqr.h"

namespace tqr {

struct DevCtl {
  int status;
  int abort;
  unsigned ticket;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Per-task trace record of the persistent kernels (qr_set_trace): task
// index (bits 0..39), task type (40..47) and SM id (48..63), then the
// globaltimer when the ticket was taken, when the task's dependencies were
// met, and when it was published.
struct TraceRec {
  uint64_t task_sm, t_take, t_ready, t_done;
};
__device__ __forceinline__ unsigned sm_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void trace_put(TraceRec* tr, int64_t cap, int64_t task, int type, uint64_t t_take,
                                          uint64_t t_ready) {
  if (tr && task < cap) {
    TraceRec r;
    r.task_sm = ((uint64_t)(sm_id() & 0xFFFF) << 48) | ((uint64_t)(type & 0xFF) << 40) | (uint64_t)task;
    r.t_take = t_take;
    r.t_ready = t_ready;
    r.t_done = globaltimer();
    tr[task] = r;
  }
}

// Wait until all counters c[0..cnt) reach v. Bounded by time and by
// iterations; on expiry sets the timeout bit and the abort flag.
__device__ inline bool wait_ge(const unsigned* c, int cnt, unsigned v, DevCtl* ctl, uint64_t timeout_ns) {
  const uint64_t t0 = globaltimer();
  const uint64_t max_iter = timeout_ns / 16 + 4096;
  uint64_t iter = 0;
  for (int q = 0; q < cnt; ++q) {
    while (ld_acquire(c + q) < v) {
      if (((volatile int*)&ctl->abort)[0]) return false;
      if (++iter > max_iter || globaltimer() - t0 > timeout_ns) {
        atomicOr(&ctl->status, QR_DEV_TIMEOUT);
        atomicExch(&ctl->abort, 1);
        return false;
      }
      __nanosleep(100);
    }
  }
  return true;
}

}  // namespace tqr
