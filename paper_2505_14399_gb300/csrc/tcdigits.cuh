// Exact fixed-point digit products on the bf16 tensor pipe (an Ozaki-style split), shared by
// the Galerkin forward-hop kernel and the SVD basis update.
//
// A double-float value v with |v| < 2 is written as 7 base-256 digits,
//     v = sum_{i < 7} s_i 2^{-6-8i},  s_i integers, |s_i| <= 129  (remainder at most 2^-55 (1 + 2^-16)),
// each digit exact in bfloat16.  The product of two such expansions is a sum of integer digit
// products: bf16 x bf16 MMAs with FP32 accumulation are exact while the partial sums stay
// below 2^24, the digit pairs (i, j) with i + j = d share one FP32 accumulator of weight
// 2^{-12-8d}, and pairs with i + j >= 7 (weight below 2^-68) are dropped.  The exact FP32 sums
// are then scaled by their weights (exact) and added to double-float accumulators with
// error-free two-sums.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "df64.cuh"
#include "tma.cuh"

namespace wmg {

constexpr int TC_NS = 7;               // digits per value

__device__ __forceinline__ void ldm_x4t(unsigned r[4], const __nv_bfloat16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldm_x2t(unsigned r[2], const __nv_bfloat16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_addr(p)));
}

// c += a b, 16x16 (row) x 16x8 (col) bf16, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// The base-256 digits of v (|v| < 2, normalised: |v.lo| <= ulp(v.hi) / 2): v = sum_i s[i]
// 2^{-6-8i}, each digit the nearest integer to the high word of the remainder, so |s[i]| <= 128
// (+1 when a remainder rounds up).  The remainders stay exact and normalised: hi - rint(hi)
// is exact, and it is either 0 or a multiple of ulp(hi) >= 2 |lo|, so one fast two-sum
// renormalises (hi - d, lo) (the double-float sum with the zero error terms left out).
__device__ __forceinline__ void tc_digits(df v, float s[TC_NS]) {
  float hi = v.hi * 64.0f, lo = v.lo * 64.0f;
#pragma unroll
  for (int i = 0; i < TC_NS; ++i) {
    const float d = rintf(hi);
    s[i] = d;
    const float r = __fsub_rn(hi, d);
    const float h2 = __fadd_rn(r, lo);
    const float l2 = __fsub_rn(lo, __fsub_rn(h2, r));
    hi = h2 * 256.0f;
    lo = l2 * 256.0f;
  }
}

// Two digits (integers, |d| <= 129: at most 8 significant bits, so the low 16 bits of their
// FP32 words are zero and the high halves are their exact bfloat16 encodings) packed as the
// bf16 pair (d0 at the lower address, d1 at the higher).
__device__ __forceinline__ unsigned tc_pack(float d0, float d1) {
  return __byte_perm(__float_as_uint(d0), __float_as_uint(d1), 0x7632);
}

// s + e += v with an error-free two-sum (v exact)
__device__ __forceinline__ void acc_add(dfacc& a, float v) {
  float s = __fadd_rn(a.s, v);
  float bb = __fsub_rn(s, a.s);
  float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(v, bb));
  a.s = s;
  a.e = __fadd_rn(a.e, err);
}

__device__ __forceinline__ bool tc_in_range(df v) { return fabsf(v.hi) < 2.0f; }   // false for NaN

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace wmg
