// Deterministic reduction helpers shared by the BLAS and Krylov kernels.
//
// A vector of length n is cut into `nblk` fixed chunks (one CTA each, an even number of
// elements so FP32 pairs can move as 16-byte accesses).  Each CTA reduces its chunk in the
// vectors' own precision with a fixed shuffle/shared-memory tree and stores one partial in
// that precision; the last CTA to finish (detected with an atomic counter) sums the partials
// in index order.  The partition and the order do not depend on timing, so results are
// bitwise reproducible.
#pragma once

#include <type_traits>

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
// mode 0: complex dot -> out[rhs*ldo + i] = scale * sum; mode 1: norm -> dout[rhs*ldo] =
// sqrt(scale * re).  scale = 1 except for the (1/n) inner product of half-storage bases.
// One warp per vector: lanes sum strided partials, then a shuffle tree (fixed order).
// Partials are P = double for FP64 vectors and P = float for the FP32-arithmetic ones, so the
// reduction of the last CTA, which every following kernel waits for, does not run on the
// FP64 units (1/74 of the FP32 rate on this part).
template <typename P>
__device__ __forceinline__ void finish_partials(const P* partial, int nv, int nblk,
                                                int maxvec, int rhs, zd* out, double* dout,
                                                int ldo, int mode, double scale = 1.0) {
  typedef typename std::conditional<sizeof(P) == 8, double2, float2>::type P2;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < nv; i += nw) {
    const P2* p = reinterpret_cast<const P2*>(partial) + ((size_t)rhs * maxvec + i) * nblk;
    // four independent accumulators keep four loads in flight per lane
    P2 s0 = {0, 0}, s1 = {0, 0}, s2 = {0, 0}, s3 = {0, 0};
    int k = lane;
    for (; k + 96 < nblk; k += 128) {
      P2 v0 = __ldcg(p + k), v1 = __ldcg(p + k + 32);
      P2 v2 = __ldcg(p + k + 64), v3 = __ldcg(p + k + 96);
      s0.x += v0.x; s0.y += v0.y; s1.x += v1.x; s1.y += v1.y;
      s2.x += v2.x; s2.y += v2.y; s3.x += v3.x; s3.y += v3.y;
    }
    for (; k < nblk; k += 32) {
      P2 v0 = __ldcg(p + k);
      s0.x += v0.x; s0.y += v0.y;
    }
    P a = (s0.x + s1.x) + (s2.x + s3.x), b = (s0.y + s1.y) + (s2.y + s3.y);
    a = warp_sum_r(a);
    b = warp_sum_r(b);
    if (lane == 0) {
      if (mode == 0) out[(size_t)rhs * ldo + i] = {(double)a * scale, (double)b * scale};
      else dout[(size_t)rhs * ldo] = sqrt((double)a * scale);
    }
  }
}

// The partial buffer (FP64 slots) viewed as partials of type P.
template <typename P>
__device__ __forceinline__ P* partials_as(double* partial) { return reinterpret_cast<P*>(partial); }

// CTA reduction (blockDim.x <= RT threads) of ni complex values held per thread (R precision)
// into the partial slots
// partial[((rhs*maxvec + i0 + q) * nblk + blockIdx.x) * 2 + {0,1}] (type R), q < ni <= G.
template <typename R, int G>
__device__ __forceinline__ void cta_store_partials(const R* ar, const R* ai, int ni, int i0,
                                                   int rhs, int maxvec, int nblk,
                                                   R* partial, R* shg) {
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
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += shg[(wv * G + q) * 2 + part];
    partial[(((size_t)rhs * maxvec + i0 + q) * nblk + blockIdx.x) * 2 + part] = s;
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
