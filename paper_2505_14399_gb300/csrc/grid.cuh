// Bounded grid-wide barrier for cooperative (co-resident) launches.
//
// An arrival counter that only grows: the counter is zero at launch, every CTA adds one per
// barrier with a release atomic, and barrier number e (counted per CTA, identical in every
// CTA because all CTAs pass the same barriers) is complete once the counter reaches
// e * nblocks, which the waiting thread observes with acquire loads.  Compared with a
// generation flag flipped by the last arrival this takes one atomic round trip off the
// critical path.  Writes made by any thread of a CTA before the barrier are visible to every
// thread of every CTA after it (CTA barrier, then release/acquire at GPU scope).
//
// A wait that exceeds `limit` polls (a second or two) raises the shared error word, which
// makes every other CTA's wait return as well: the barrier returns false and the kernel
// returns instead of hanging.
#pragma once

#include "common.cuh"

namespace wmg {

struct BarrierState {
  unsigned count;
  unsigned pad0;
  int err;
  int pad1;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void add_release_gpu(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Returns false if the wait gave up or another CTA raised the error word.  `epoch` counts
// this CTA's barriers since launch (start at 0).
__device__ __forceinline__ bool grid_barrier(BarrierState* bs, unsigned nblocks, unsigned& epoch,
                                             long long limit = (1ll << 21)) {
  __shared__ int ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    add_release_gpu(&bs->count, 1u);
    const unsigned target = nblocks * epoch;
    int good = 1;
    long long spins = 0;
    while ((int)(ld_acquire_gpu(&bs->count) - target) < 0) {
      if ((++spins & 63) == 0) {
        if (*(volatile int*)&bs->err) { good = 0; break; }
        if (spins > limit) {
          atomicExch(&bs->err, 1);
          good = 0;
          break;
        }
      }
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace wmg
