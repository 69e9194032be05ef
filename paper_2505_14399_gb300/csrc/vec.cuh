// Storage of Krylov vectors and BLAS operands.
//
// A vector is an array of complex elements E: zd (complex double), zf (complex float),
// __half2 or __nv_bfloat162 (complex half / bfloat16, FP32 arithmetic).  VecT<E> gives
// the arithmetic type, element load/store, and -- for the FP32-arithmetic types --
// load/store of a pack of two consecutive elements as a float4 (16-byte accesses for zf,
// 8-byte for the half types).
//
// `rms`: Krylov bases in half storage are normalised to unit root-mean-square entries
// (norm sqrt(n)) instead of unit norm, so their entries stay O(1), inside FP16's normal
// range whatever the lattice volume.  GMRES only needs one inner product used
// consistently; the reductions then return (1/n) x^dag y.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace wmg {

template <typename E> struct VecT;

template <> struct VecT<zd> {
  typedef double R;
  static constexpr bool packed = false;
  static constexpr bool rms = false;
  static __device__ __forceinline__ zd ld(const zd* p, size_t i) { return p[i]; }
  static __device__ __forceinline__ void st(zd* p, size_t i, zd v) { p[i] = v; }
  static __device__ __forceinline__ float4 ld2(const zd*, size_t) { return float4{}; }
  static __device__ __forceinline__ void st2(zd*, size_t, float4) {}
  static __device__ __forceinline__ zd rnd(zd v) { return v; }
  static __device__ __forceinline__ float4 rnd2(float4 v) { return v; }
};

template <> struct VecT<zf> {
  typedef float R;
  static constexpr bool packed = true;
  static constexpr bool rms = false;
  static __device__ __forceinline__ zf ld(const zf* p, size_t i) { return p[i]; }
  static __device__ __forceinline__ void st(zf* p, size_t i, zf v) { p[i] = v; }
  static __device__ __forceinline__ float4 ld2(const zf* p, size_t k) {
    return reinterpret_cast<const float4*>(p)[k];
  }
  static __device__ __forceinline__ void st2(zf* p, size_t k, float4 v) {
    reinterpret_cast<float4*>(p)[k] = v;
  }
  static __device__ __forceinline__ zf rnd(zf v) { return v; }
  static __device__ __forceinline__ float4 rnd2(float4 v) { return v; }
};

template <typename H, typename Cvt>
struct VecHalf {
  typedef float R;
  static constexpr bool packed = true;
  static constexpr bool rms = true;
  static __device__ __forceinline__ zf ld(const H* p, size_t i) {
    float2 v = Cvt::to2(p[i]);
    return {v.x, v.y};
  }
  static __device__ __forceinline__ void st(H* p, size_t i, zf v) { p[i] = Cvt::from2(v.re, v.im); }
  static __device__ __forceinline__ float4 ld2(const H* p, size_t k) {
    uint2 u = reinterpret_cast<const uint2*>(p)[k];
    H a, b;
    memcpy(&a, &u.x, 4);
    memcpy(&b, &u.y, 4);
    float2 fa = Cvt::to2(a), fb = Cvt::to2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
  }
  static __device__ __forceinline__ void st2(H* p, size_t k, float4 v) {
    H a = Cvt::from2(v.x, v.y), b = Cvt::from2(v.z, v.w);
    uint2 u;
    memcpy(&u.x, &a, 4);
    memcpy(&u.y, &b, 4);
    reinterpret_cast<uint2*>(p)[k] = u;
  }
  // the value a store followed by a load gives back
  static __device__ __forceinline__ zf rnd(zf v) {
    float2 r = Cvt::to2(Cvt::from2(v.re, v.im));
    return {r.x, r.y};
  }
  static __device__ __forceinline__ float4 rnd2(float4 v) {
    float2 a = Cvt::to2(Cvt::from2(v.x, v.y)), b = Cvt::to2(Cvt::from2(v.z, v.w));
    return make_float4(a.x, a.y, b.x, b.y);
  }
};

struct CvtF16 {
  static __device__ __forceinline__ float2 to2(__half2 h) { return __half22float2(h); }
  static __device__ __forceinline__ __half2 from2(float a, float b) { return __floats2half2_rn(a, b); }
};
struct CvtBF16 {
  static __device__ __forceinline__ float2 to2(__nv_bfloat162 h) { return __bfloat1622float2(h); }
  static __device__ __forceinline__ __nv_bfloat162 from2(float a, float b) {
    return __floats2bfloat162_rn(a, b);
  }
};

template <> struct VecT<__half2> : VecHalf<__half2, CvtF16> {};
template <> struct VecT<__nv_bfloat162> : VecHalf<__nv_bfloat162, CvtBF16> {};

typedef __half2 zh;
typedef __nv_bfloat162 zbf;

}  // namespace wmg
