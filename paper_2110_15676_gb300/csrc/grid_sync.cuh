// Grid-wide barrier for persistent cooperative launches, with a bounded wait.
//
// Cooperative launch guarantees that all blocks of the grid are resident, so the
// barrier cannot wait forever; the bound (a few seconds of the global timer) is a
// safety net.  On expiry a block records the error in the barrier state and every
// later barrier of the launch passes at once, so the launch still ends; the host
// reads the flag and reports AFC_E_TIMEOUT.
//
// Memory: the block's threads meet at __syncthreads, then its first thread fences
// (cumulatively for the block's writes), arrives, waits and fences again before the
// block's threads meet once more, so plain loads after the barrier see what other
// blocks wrote before it.  Arrays
// written inside a persistent launch must not be read through the read-only
// (non-coherent) path, i.e. not through const __restrict__ pointers.
#pragma once

#include "afc_internal.h"

namespace afc {

struct GridBar {
  unsigned int count;   // blocks arrived at the current barrier
  unsigned int gen;     // barrier generation
  int err;              // 1 after a wait gave up
  int pad;
};

constexpr unsigned long long kBarrierWaitNs = 4000000000ull;   // 4 s of the global timer

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void grid_barrier(GridBar* gb) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &gb->gen;
    volatile int* verr = &gb->err;
    const unsigned int g0 = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&gb->count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&gb->count, 0u);   // reset before the release
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else if (*verr == 0) {
      const unsigned long long t0 = global_ns();
      while (*vgen == g0) {
        if (*verr != 0) break;
        if (global_ns() - t0 > kBarrierWaitNs) {
          atomicExch(&gb->err, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

}  // namespace afc
