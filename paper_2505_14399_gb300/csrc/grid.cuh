// Bounded grid-wide barrier for cooperative (co-resident) launches.
//
// Sense reversal through a generation counter: every CTA reads the generation, arrives on
// the counter, and the last arrival resets the counter and advances the generation; the
// others poll the generation.  A wait that exceeds `limit` polls (about a second) raises the
// shared error word, which makes every other CTA's wait return as well: the barrier returns
// false and the kernel returns instead of hanging.
#pragma once

#include "common.cuh"

namespace wmg {

struct BarrierState {
  unsigned count;
  unsigned gen;
  int err;
  int pad;
};

// Returns false if the wait gave up or another CTA raised the error word.
__device__ __forceinline__ bool grid_barrier(BarrierState* bs, unsigned nblocks,
                                             long long limit = (1ll << 22)) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &bs->gen;
    volatile int* verr = &bs->err;
    unsigned g = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(&bs->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bs->count, 0u);
      __threadfence();
      atomicAdd((unsigned*)&bs->gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g && *verr == 0) {
        if (++spins > limit) {   // 2^22 polls: about a second
          atomicExch((int*)&bs->err, 1);
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
    ok = (*verr == 0);
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace wmg
