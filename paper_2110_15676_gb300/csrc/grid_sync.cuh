// Grid-wide barrier for persistent cooperative launches, with a bounded wait.
//
// Cooperative launch guarantees that all blocks of the grid are resident, so the
// barrier cannot wait forever; the bound (a few seconds of the global timer) is a
// safety net.  On expiry a block records the error in the barrier state and every
// later barrier of the launch passes at once, so the launch still ends; the host
// reads the flag and reports AFC_E_TIMEOUT.
//
// Arrival is one atomic add on a single counter: block 0 adds 2^31 - (G - 1) and
// every other block adds 1, so the grid adds exactly 2^31 per barrier.  Bit 31 of
// the counter therefore changes when, and only when, the last block arrives, and
// the low bits come back to the value they had before, so the counter needs no
// reset between barriers or launches.  A waiting block watches bit 31 against the
// value its own add returned.  On GB300 this took 1.5 us per barrier of 304
// blocks, against 2.6 us for a count that the last block resets before it bumps a
// separate generation word (two more serial atomics on the release path).
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
  unsigned int arrive;  // arrival counter; bit 31 flips once per completed barrier
  unsigned int spare;
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
    volatile unsigned int* va = &gb->arrive;
    volatile int* verr = &gb->err;
    const unsigned int add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    __threadfence();
    const unsigned int old = atomicAdd(&gb->arrive, add);
    if (*verr == 0) {
      const unsigned long long t0 = global_ns();
      while (((old ^ *va) & 0x80000000u) == 0u) {
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
