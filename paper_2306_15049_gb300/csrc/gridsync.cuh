// Grid-wide barrier for cooperatively launched kernels (all CTAs co-resident).
#pragma once

#include "internal.cuh"

namespace rk {

constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s, far beyond any phase

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier number nb (1, 2, ...) of the launch over its G co-resident CTAs: a
// monotonic arrival counter (zeroed by the host before the launch) that every
// CTA waits to reach nb * G. Returns false if this CTA gave up (timeout, or
// another CTA's error flag).
__device__ inline bool grid_sync(GridBar* bar, unsigned long long target, int* ok_s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(&bar->count, 1ull);
    if (ld_acquire_u64(&bar->count) < target) {
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (ld_acquire_u64(&bar->count) < target) {
        if ((++spins & 63u) == 0) {
          if (*((volatile int*)&bar->err)) { ok = 0; break; }
          if (global_ns() - t0 > kBarrierTimeoutNs) {
            atomicExch(&bar->err, 1);
            ok = 0;
            break;
          }
        }
      }
    }
    *ok_s = ok;
  }
  __syncthreads();
  return *ok_s != 0;
}

}  // namespace rk
