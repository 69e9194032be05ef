// Double-float ("df64") arithmetic: a value is hi + lo with two FP32 numbers.
//
// GB300 runs FP32 FMA about 64x faster than FP64, so sums of products that need close
// to FP64 accuracy are formed with error-free transformations on FP32 units:
//   TwoProd(a, b):  p = a*b, e = fma(a, b, -p)             (a*b = p + e exactly)
//   TwoSum(a, b):   s = a+b, bb = s-a, e = (a-(s-bb))+(b-bb) (a+b = s + e exactly)
// (Dekker 1971; Knuth TAOCP vol. 2, Sec. 4.2.2; Ogita, Rump, Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26, 2005 -- the "Dot2" scheme).  A product of df64 numbers
// keeps hi*hi exactly plus the cross terms hi*lo + lo*hi; an accumulator is an unnormalised
// pair (s, e) whose e collects the rounding errors, so a K-term dot product carries a
// relative error of order K * 2^-48 (about 1e-13 for K ~ 10^3) instead of FP64's K * 2^-53.
#pragma once

#include "common.cuh"

namespace wmg {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_from(double x) {
  float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ df df_from(float x) { return {x, 0.0f}; }
__device__ __forceinline__ double df_to_double(float s, float e) { return (double)s + (double)e; }

// accumulator for sums of products
struct dfacc {
  float s, e;
};

// acc += a * b  (a, b df64).  The _rn intrinsics are never contracted into FMAs by the
// compiler, which the error-free transformations rely on.
__device__ __forceinline__ void df_fma(dfacc& acc, df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float pe = fmaf(a.hi, b.hi, -p);
  pe = fmaf(a.hi, b.lo, pe);
  pe = fmaf(a.lo, b.hi, pe);
  float s = __fadd_rn(acc.s, p);
  float bb = __fsub_rn(s, acc.s);
  float err = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.s = s;
  acc.e = __fadd_rn(acc.e, __fadd_rn(err, pe));
}

// complex df64 value and accumulator
struct zdf {
  df re, im;
};
struct zdfacc {
  dfacc re, im;
};

__device__ __forceinline__ zdf zdf_from(zd x) { return {df_from(x.re), df_from(x.im)}; }
__device__ __forceinline__ zdf zdf_from(zf x) { return {df_from(x.re), df_from(x.im)}; }
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// acc += conj(a) * b
__device__ __forceinline__ void zdf_fmac(zdfacc& acc, zdf a, zdf b) {
  df_fma(acc.re, a.re, b.re);
  df_fma(acc.re, a.im, b.im);
  df_fma(acc.im, a.re, b.im);
  df_fma(acc.im, df_neg(a.im), b.re);
}
// acc += a * b
__device__ __forceinline__ void zdf_fma(zdfacc& acc, zdf a, zdf b) {
  df_fma(acc.re, a.re, b.re);
  df_fma(acc.re, df_neg(a.im), b.im);
  df_fma(acc.im, a.re, b.im);
  df_fma(acc.im, a.im, b.re);
}
__device__ __forceinline__ zd zdf_result(const zdfacc& acc) {
  return {df_to_double(acc.re.s, acc.re.e), df_to_double(acc.im.s, acc.im.e)};
}

__device__ __forceinline__ double df_val(df a) { return (double)a.hi + (double)a.lo; }

// a * b + c * d as a normalised df64 value (two Dot2 steps and a Fast-TwoSum)
__device__ __forceinline__ df df_dot2(df a, df b, df c, df d) {
  dfacc t{0.0f, 0.0f};
  df_fma(t, a, b);
  df_fma(t, c, d);
  float h = __fadd_rn(t.s, t.e);
  return {h, __fsub_rn(t.e, __fsub_rn(h, t.s))};
}

// An accumulator as a normalised df64 value (Fast-TwoSum: |s| >= |e| holds for the
// accumulated sum and its collected rounding errors).
__device__ __forceinline__ df df_norm(dfacc a) {
  float h = __fadd_rn(a.s, a.e);
  return {h, __fsub_rn(a.e, __fsub_rn(h, a.s))};
}
__device__ __forceinline__ zdf zdf_norm(const zdfacc& a) { return {df_norm(a.re), df_norm(a.im)}; }

// Normalised df64 arithmetic for the few scalar steps that need it (Jacobi rotations).
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {   // |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  float s = __fadd_rn(a.hi, b.hi);
  float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s, e);
}
__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
  float p = __fmul_rn(a.hi, b);
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ float df_to_float(df a) { return __fadd_rn(a.hi, a.lo); }
// Exact comparison of normalised values.
__device__ __forceinline__ bool df_less(df a, df b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
// 1 / sqrt(x), x > 0: the FP32 estimate refined by two Newton steps y <- y + y (1 - x y^2) / 2
// in df64 (each step squares the relative error: ~1e-7 -> ~1e-14 -> rounding).
__device__ __forceinline__ df df_rsqrt(df x) {
  df y = {rsqrtf(x.hi), 0.0f};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    df r = df_add({1.0f, 0.0f}, df_neg(df_mul(x, df_mul(y, y))));
    y = df_add(y, df_mul(y, df_mul_f(r, 0.5f)));
  }
  return y;
}

// complex df64 sign and i-multiples (exact)
__device__ __forceinline__ zdf zdf_neg(zdf a) { return {df_neg(a.re), df_neg(a.im)}; }
__device__ __forceinline__ zdf zdf_ti(zdf a) { return {df_neg(a.im), a.re}; }    // i a
__device__ __forceinline__ zdf zdf_tmi(zdf a) { return {a.im, df_neg(a.re)}; }   // -i a

// 16-byte load / store of a complex df64 value stored as (re.hi, re.lo, im.hi, im.lo)
__device__ __forceinline__ zdf zdf_ld(const zdf* p) {
  float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return {{v.x, v.y}, {v.z, v.w}};
}

}  // namespace wmg
