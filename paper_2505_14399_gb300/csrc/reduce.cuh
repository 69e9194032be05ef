// Deterministic reduction helpers shared by the BLAS and Krylov kernels.
//
// A vector of length n is cut into `nblk` fixed chunks (one CTA each, an even number of
// elements so FP32 pairs can move as 16-byte accesses).  Each CTA reduces its chunk in the
// vectors' own precision with a fixed shuffle/shared-memory tree and stores one FP64
// partial; the last CTA to finish (detected with an atomic counter) sums the partials in
// index order.  The partition and the order do not depend on timing, so results are
// bitwise reproducible.
#pragma once

#include "common.cuh"

namespace wmg {

constexpr int RT = 256;  // threads per reduction CTA

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <typename R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__host__ __device__ __forceinline__ size_t reduce_chunk(size_t n, int nblk) {
  return (((n + nblk - 1) / nblk) + 1) & ~(size_t)1;
}

// Final reduction over the nblk partials of every (rhs, i), done by the last CTA.
// mode 0: complex dot -> out[rhs*ldo + i]; mode 1: norm -> dout[rhs*ldo] = sqrt(re).
// One warp per vector: lanes sum strided partials, then a shuffle tree (fixed order).
__device__ __forceinline__ void finish_partials(const double* partial, int nv, int nblk,
                                                int maxvec, int rhs, zd* out, double* dout,
                                                int ldo, int mode) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < nv; i += nw) {
    const double* p = partial + ((size_t)rhs * maxvec + i) * nblk * 2;
    double a = 0, b = 0;
    for (int k = lane; k < nblk; k += 32) {
      a += __ldcg(p + 2 * k);
      b += __ldcg(p + 2 * k + 1);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
      if (mode == 0) out[(size_t)rhs * ldo + i] = {a, b};
      else dout[(size_t)rhs * ldo] = sqrt(a);
    }
  }
}

// CTA reduction of ni complex values held per thread (R precision) into the FP64 partial
// slots partial[((rhs*maxvec + i0 + q) * nblk + blockIdx.x) * 2 + {0,1}], q < ni <= G.
template <typename R, int G>
__device__ __forceinline__ void cta_store_partials(const R* ar, const R* ai, int ni, int i0,
                                                   int rhs, int maxvec, int nblk,
                                                   double* partial, R* shg) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < G; ++q) {
    if (q < ni) {
      R dr = warp_sum_r(ar[q]);
      R di = warp_sum_r(ai[q]);
      if (lane == 0) { shg[(wid * G + q) * 2] = dr; shg[(wid * G + q) * 2 + 1] = di; }
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < 2 * ni) {
    int q = threadIdx.x >> 1, part = threadIdx.x & 1;
    R s = 0;
    for (int wv = 0; wv < RT / 32; ++wv) s += shg[(wv * G + q) * 2 + part];
    partial[(((size_t)rhs * maxvec + i0 + q) * nblk + blockIdx.x) * 2 + part] = (double)s;
    __threadfence();   // the writer publishes its partial before the CTA signals completion
  }
  __syncthreads();
}

// Arrive at the per-rhs counter; returns true in every thread of the last CTA.  Threads
// that wrote partials have fenced them already.
__device__ __forceinline__ bool last_cta(unsigned* counter, int rhs, int nblk) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter + rhs, 1u) == (unsigned)nblk - 1);
  __syncthreads();
  if (last) __threadfence();
  return last;
}

}  // namespace wmg
