// Grid-wide barrier for cooperative launches (all blocks co-resident), with a
// wait bounded by %globaltimer: on expiry *status becomes kEtimeout and every
// block leaves.  Used by the adjoint and by the bulk-synchronous schedules.
#pragma once

#include <cstdint>

#include "eik_internal.h"

namespace eik {
namespace grid {

__device__ __forceinline__ unsigned ld_acq(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ long long now_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// count/gen: barrier words (zero before the launch); status: 0 while running.
// Returns false when the launch must stop (status set).
__device__ __forceinline__ bool barrier(unsigned *count, unsigned *gen, unsigned *status,
                                        long long timeout_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = ld_acq(gen);
    __threadfence();
    if (atomicAdd(count, 1u) + 1u == gridDim.x) {
      *count = 0u;
      __threadfence();
      st_rel(gen, g + 1u);
    } else {
      const long long t0 = now_ns();
      while (ld_acq(gen) == g) {
        if (ld_acq(status) != 0u) break;
        if (now_ns() - t0 > timeout_ns) { atomicCAS(status, 0u, kEtimeout); break; }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ld_acq(status) == 0u;
}

}  // namespace grid
}  // namespace eik
