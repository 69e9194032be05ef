// Batched BLAS-1 on complex fields with deterministic reductions.
//
// Reductions use a fixed partition of each vector into `nblk` chunks (one CTA each),
// a fixed shuffle/shared-memory tree inside the CTA, and a final fixed-order tree
// over the chunk partials performed by whichever CTA finishes last (its identity
// does not change the arithmetic), so results are bitwise reproducible run to run.
//
// Every routine is templated on the vector element E (vec.cuh): complex double, complex
// float, or complex half / bfloat16 with FP32 arithmetic.  The FP32-arithmetic types move
// two complex numbers per access (float4 for complex float, 8 bytes for the half types).
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "reduce.cuh"
#include "vec.cuh"

namespace wmg {

namespace {

// pairs of complex numbers can move as one pack when both ends of the range are even
__device__ __forceinline__ bool pack_ok(size_t a, size_t b) { return ((a | b) & 1) == 0; }

template <typename E>
__global__ void __launch_bounds__(RT)
multi_dot_kernel(zd* out, int ldo, const E* __restrict__ V, size_t vstride, int nv,
                 const E* __restrict__ w, size_t n, double* partial, unsigned* counter,
                 int nblk, int maxvec, double scale) {
  dep_entry();
  typedef VecT<E> T;
  typedef typename T::R R;
  __shared__ double sh[(RT / 32) * 8 * 2];
  int rhs = blockIdx.y;
  size_t chunk = reduce_chunk(n, nblk);   // even: two-element packs
  size_t k0 = (size_t)blockIdx.x * chunk;
  size_t k1 = min(n, k0 + chunk);
  const E* wr = w + (size_t)rhs * n;
  // groups of G basis vectors share one pass over w (G independent loads per element)
  constexpr int G = 8;
  for (int i0 = 0; i0 < nv; i0 += G) {
    int ni = min(G, nv - i0);
    R ar[G], ai[G];
#pragma unroll
    for (int q = 0; q < G; ++q) { ar[q] = 0; ai[q] = 0; }
    const E* vb = V + (size_t)i0 * vstride + (size_t)rhs * n;
    bool packed = false;
    if constexpr (T::packed) packed = pack_ok(k0 | k1, vstride);
    if (packed) {
      size_t vs2 = vstride / 2;
      for (size_t k = k0 / 2 + threadIdx.x; k < k1 / 2; k += RT) {
        float4 b = T::ld2(wr, k);
#pragma unroll
        for (int q = 0; q < G; ++q) {
          if (q < ni) {
            float4 a = T::ld2(vb + (size_t)q * 2 * vs2, k);
            ar[q] = fma((R)a.x, (R)b.x, ar[q]); ar[q] = fma((R)a.y, (R)b.y, ar[q]);
            ar[q] = fma((R)a.z, (R)b.z, ar[q]); ar[q] = fma((R)a.w, (R)b.w, ar[q]);
            ai[q] = fma((R)a.x, (R)b.y, ai[q]); ai[q] = fma(-(R)a.y, (R)b.x, ai[q]);
            ai[q] = fma((R)a.z, (R)b.w, ai[q]); ai[q] = fma(-(R)a.w, (R)b.z, ai[q]);
          }
        }
      }
    } else {
      for (size_t k = k0 + threadIdx.x; k < k1; k += RT) {
        cplx<R> b = T::ld(wr, k);
#pragma unroll
        for (int q = 0; q < G; ++q) {
          if (q < ni) {
            cplx<R> a = T::ld(vb, (size_t)q * vstride + k);
            ar[q] = fma(a.re, b.re, ar[q]); ar[q] = fma(a.im, b.im, ar[q]);
            ai[q] = fma(a.re, b.im, ai[q]); ai[q] = fma(-a.im, b.re, ai[q]);
          }
        }
      }
    }
    // CTA and cross-CTA reductions in the vectors' own arithmetic (FP64 arithmetic is scarce
    // on this GPU)
    cta_store_partials<R, G>(ar, ai, ni, i0, rhs, maxvec, nblk, partials_as<R>(partial),
                             reinterpret_cast<R*>(sh));
  }
  if (!last_cta(counter, rhs, nblk)) return;
  finish_partials(partials_as<R>(partial), nv, nblk, maxvec, rhs, out, nullptr, ldo, 0, scale);
  if (threadIdx.x == 0) counter[rhs] = 0;
}

template <typename E>
__global__ void __launch_bounds__(RT)
norm_kernel(double* nrm, int ldn, const E* __restrict__ w, size_t n, double* partial,
            unsigned* counter, int nblk, int maxvec, double scale) {
  dep_entry();
  typedef VecT<E> T;
  typedef typename T::R R;
  __shared__ double sh[64];
  int rhs = blockIdx.y;
  size_t chunk = reduce_chunk(n, nblk);   // even: two-element packs
  size_t k0 = (size_t)blockIdx.x * chunk;
  size_t k1 = min(n, k0 + chunk);
  const E* wr = w + (size_t)rhs * n;
  R acc = 0;
  bool packed = false;
  if constexpr (T::packed) packed = pack_ok(k0, k1);
  if (packed) {
    for (size_t k = k0 / 2 + threadIdx.x; k < k1 / 2; k += RT) {
      float4 a = T::ld2(wr, k);
      acc = fma((R)a.x, (R)a.x, acc); acc = fma((R)a.y, (R)a.y, acc);
      acc = fma((R)a.z, (R)a.z, acc); acc = fma((R)a.w, (R)a.w, acc);
    }
  } else {
    for (size_t k = k0 + threadIdx.x; k < k1; k += RT) {
      cplx<R> a = T::ld(wr, k);
      acc = fma(a.re, a.re, acc);
      acc = fma(a.im, a.im, acc);
    }
  }
  // CTA tree and cross-CTA sum in the vectors' arithmetic
  acc = warp_sum_r(acc);
  R* shr = reinterpret_cast<R*>(sh);
  if ((threadIdx.x & 31) == 0) shr[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    R s = 0;
    for (int wv = 0; wv < RT / 32; ++wv) s += shr[wv];
    R* p = partials_as<R>(partial) + ((size_t)rhs * maxvec * nblk + blockIdx.x) * 2;
    p[0] = s;
    p[1] = 0;
    __threadfence();
  }
  if (!last_cta(counter, rhs, nblk)) return;
  finish_partials(partials_as<R>(partial), 1, nblk, maxvec, rhs, nullptr, nrm, ldn, 1, scale);
  if (threadIdx.x == 0) counter[rhs] = 0;
}

// w[rhs] += sgn * sum_i c_i V_i[rhs]
template <typename E>
__global__ void multi_axpy_kernel(E* w, const E* __restrict__ V, size_t vstride, int nv,
                                  const zd* c, int ldc, double sgn, size_t n) {
  dep_entry();
  typedef VecT<E> T;
  typedef typename T::R R;
  __shared__ cplx<R> cs[128];
  int rhs = blockIdx.y;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    zd v = c[(size_t)rhs * ldc + i];
    cs[i] = {(R)(sgn * v.re), (R)(sgn * v.im)};
  }
  __syncthreads();
  E* wr = w + (size_t)rhs * n;
  const E* vb = V + (size_t)rhs * n;
  bool packed = false;
  if constexpr (T::packed) packed = pack_ok(n, vstride);
  if (packed) {
    size_t vs2 = vstride / 2;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n / 2;
         k += (size_t)gridDim.x * blockDim.x) {
      float4 acc = T::ld2(wr, k);
      for (int i = 0; i < nv; ++i) {
        float4 v = T::ld2(vb + (size_t)i * 2 * vs2, k);
        float cr = (float)cs[i].re, ci = (float)cs[i].im;
        acc.x = fmaf(cr, v.x, acc.x); acc.x = fmaf(-ci, v.y, acc.x);
        acc.y = fmaf(cr, v.y, acc.y); acc.y = fmaf(ci, v.x, acc.y);
        acc.z = fmaf(cr, v.z, acc.z); acc.z = fmaf(-ci, v.w, acc.z);
        acc.w = fmaf(cr, v.w, acc.w); acc.w = fmaf(ci, v.z, acc.w);
      }
      T::st2(wr, k, acc);
    }
    return;
  }
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    cplx<R> acc = T::ld(wr, k);
    for (int i = 0; i < nv; ++i) cfma(acc, cs[i], T::ld(vb, (size_t)i * vstride + k));
    T::st(wr, k, acc);
  }
}

template <typename E>
__global__ void scale_inv_kernel(E* y, const E* x, const double* s, int lds, size_t n) {
  dep_entry();
  typedef VecT<E> T;
  typedef typename T::R R;
  int rhs = blockIdx.y;
  double sv = s[(size_t)rhs * lds];
  R f = sv > 0 ? (R)(1.0 / sv) : (R)0;
  const E* xr = x + (size_t)rhs * n;
  E* yr = y + (size_t)rhs * n;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    cplx<R> v = T::ld(xr, k);
    T::st(yr, k, {f * v.re, f * v.im});
  }
}

template <typename E>
__global__ void axpby_kernel(E* y, double a, const E* x, double b, size_t n) {
  dep_entry();
  typedef VecT<E> T;
  typedef typename T::R R;
  R ar = (R)a, br = (R)b;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    cplx<R> xv = T::ld(x, k), yv = T::ld(y, k);
    T::st(y, k, {fma(ar, xv.re, br * yv.re), fma(ar, xv.im, br * yv.im)});
  }
}

// y += a * x with x and y of possibly different storage (arithmetic of y)
template <typename Ey, typename Ex>
__global__ void axpy_mixed_kernel(Ey* y, double a, const Ex* x, size_t n) {
  dep_entry();
  typedef typename VecT<Ey>::R R;
  R ar = (R)a;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    auto xv = VecT<Ex>::ld(x, k);
    cplx<R> yv = VecT<Ey>::ld(y, k);
    VecT<Ey>::st(y, k, {fma(ar, (R)xv.re, yv.re), fma(ar, (R)xv.im, yv.im)});
  }
}

// y = a * x1 + b * x2 (x1, x2 in one storage, y in another; arithmetic of x)
template <typename Eo, typename Ei>
__global__ void lincomb_kernel(Eo* y, double a, const Ei* x1, double b, const Ei* x2, size_t n) {
  dep_entry();
  typedef typename VecT<Ei>::R R;
  typedef typename VecT<Eo>::R Ro;
  R ar = (R)a, br = (R)b;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    cplx<R> u = VecT<Ei>::ld(x1, k), v = VecT<Ei>::ld(x2, k);
    VecT<Eo>::st(y, k, {(Ro)fma(ar, u.re, br * v.re), (Ro)fma(ar, u.im, br * v.im)});
  }
}

template <typename Eo, typename Ei>
__global__ void convert_kernel(Eo* y, const Ei* x, const double* s, int inv, size_t n) {
  dep_entry();
  typedef typename VecT<Eo>::R Ro;
  int rhs = blockIdx.y;
  double f = 1.0;
  if (s) {
    double sv = s[rhs];
    f = inv ? (sv > 0 ? 1.0 / sv : 0.0) : sv;
  }
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    auto v = VecT<Ei>::ld(x + (size_t)rhs * n, k);
    VecT<Eo>::st(y + (size_t)rhs * n, k, {(Ro)(f * (double)v.re), (Ro)(f * (double)v.im)});
  }
}

template <typename Ei>
__global__ void accumulate_scaled_kernel(zd* y, const Ei* x, const double* s, size_t n) {
  dep_entry();
  int rhs = blockIdx.y;
  double f = s[rhs];
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    auto v = VecT<Ei>::ld(x + (size_t)rhs * n, k);
    zd& t = y[(size_t)rhs * n + k];
    t.re = fma(f, (double)v.re, t.re);
    t.im = fma(f, (double)v.im, t.im);
  }
}

template <typename E>
__global__ void gamma5_kernel(E* y, const E* x, size_t nsites) {
  typedef VecT<E> T;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < nsites * 12;
       k += (size_t)gridDim.x * blockDim.x) {
    int comp = (int)(k % 12);
    auto v = T::ld(x, k);
    if (comp >= 6) { v.re = -v.re; v.im = -v.im; }
    T::st(y, k, v);
  }
}

inline int grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  size_t cap = (size_t)num_sms() * 8;
  return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

}  // namespace

int ReduceWork::alloc(size_t n, int nrhs, int mv) {
  release();
  size_t nb = (n + 4 * RT - 1) / (4 * RT);
  size_t cap = (size_t)num_sms() * 6;
  nblk = (int)(nb < 1 ? 1 : (nb > cap ? cap : nb));
  size_t per128 = (n / 12 + 127) / 128;
  this->cap = (int)(per128 > (size_t)nblk ? per128 : (size_t)nblk);
  maxvec = mv;
  nrhs_cap = nrhs;
  WMG_TRY(dev_alloc(&partial, sizeof(double) * 2 * (size_t)this->cap * maxvec * nrhs));
  WMG_TRY(dev_alloc(&counter, sizeof(unsigned) * nrhs));
  WMG_CUDA(cudaMemset(counter, 0, sizeof(unsigned) * nrhs));
  return MG_OK;
}

void ReduceWork::release() {
  dev_free(partial);
  dev_free(counter);
  partial = nullptr;
  counter = nullptr;
}

template <typename E>
int multi_dot_v(zd* out, int ldo, const E* V, size_t vstride, int nv, const E* w, size_t n,
                int nrhs, ReduceWork& rw, cudaStream_t st, double scale) {
  if (nv > rw.maxvec || nrhs > rw.nrhs_cap) return fail(MG_EINVAL, "multi_dot: workspace too small");
  dim3 grid(rw.nblk, nrhs);
  ProfScope ps("multi_dot", (double)(nv + 1) * nrhs * n * sizeof(E), 8.0 * nv * n * nrhs, st);
  WMG_LAUNCH_DEP(multi_dot_kernel<E>, grid, RT, 0, st, out, ldo, V, vstride, nv, w, n, rw.partial, rw.counter, rw.nblk, rw.maxvec, scale);
  return MG_OK;
}

template <typename E>
int multi_axpy_v(E* w, const E* V, size_t vstride, int nv, const zd* c, int ldc, double sgn,
                 size_t n, int nrhs, cudaStream_t st) {
  if (nv > 128) return fail(MG_EINVAL, "multi_axpy: too many vectors");
  if (nv == 0) return MG_OK;
  dim3 grid(grid_for(VecT<E>::packed ? n / 2 : n), nrhs);
  ProfScope ps("multi_axpy", (double)(nv + 2) * nrhs * n * sizeof(E), 8.0 * nv * n * nrhs, st);
  WMG_LAUNCH_DEP(multi_axpy_kernel<E>, grid, 256, 0, st, w, V, vstride, nv, c, ldc, sgn, n);
  return MG_OK;
}

template <typename E>
int norm2_v(double* nrm, int ldn, const E* w, size_t n, int nrhs, ReduceWork& rw,
            cudaStream_t st, double scale) {
  if (nrhs > rw.nrhs_cap) return fail(MG_EINVAL, "norm2: workspace too small");
  dim3 grid(rw.nblk, nrhs);
  ProfScope ps("norm", (double)nrhs * n * sizeof(E), 4.0 * n * nrhs, st);
  WMG_LAUNCH_DEP(norm_kernel<E>, grid, RT, 0, st, nrm, ldn, w, n, rw.partial, rw.counter, rw.nblk, rw.maxvec, scale);
  return MG_OK;
}

template <typename E>
int scale_inv_v(E* y, const E* x, const double* s, int lds, size_t n, int nrhs, cudaStream_t st) {
  dim3 grid(grid_for(n), nrhs);
  ProfScope ps("scale", 2.0 * nrhs * n * sizeof(E), 2.0 * n * nrhs, st);
  WMG_LAUNCH_DEP(scale_inv_kernel<E>, grid, 256, 0, st, y, x, s, lds, n);
  return MG_OK;
}

template <typename E>
int axpby_v(E* y, double a, const E* x, double b, size_t n, int nrhs, cudaStream_t st) {
  size_t tot = n * nrhs;
  WMG_LAUNCH_DEP(axpby_kernel<E>, grid_for(tot), 256, 0, st, y, a, x, b, tot);
  return MG_OK;
}

template <typename Ey, typename Ex>
int axpy_mixed(Ey* y, double a, const Ex* x, size_t n, cudaStream_t st) {
  WMG_LAUNCH_DEP(axpy_mixed_kernel<Ey, Ex>, grid_for(n), 256, 0, st, y, a, x, n);
  return MG_OK;
}

template <typename Eo, typename Ei>
int lincomb_v(Eo* y, double a, const Ei* x1, double b, const Ei* x2, size_t n, cudaStream_t st) {
  WMG_LAUNCH_DEP(lincomb_kernel<Eo, Ei>, grid_for(n), 256, 0, st, y, a, x1, b, x2, n);
  return MG_OK;
}

template <typename Eo, typename Ei>
int convert_v(Eo* y, const Ei* x, const double* s, int inv, size_t n, int nrhs, cudaStream_t st) {
  dim3 grid(grid_for(n), nrhs);
  WMG_LAUNCH_DEP(convert_kernel<Eo, Ei>, grid, 256, 0, st, y, x, s, inv, n);
  return MG_OK;
}

template <typename Ei>
int accumulate_scaled_v(zd* y, const Ei* x, const double* s, size_t n, int nrhs,
                        cudaStream_t st) {
  dim3 grid(grid_for(n), nrhs);
  WMG_LAUNCH_DEP(accumulate_scaled_kernel<Ei>, grid, 256, 0, st, y, x, s, n);
  return MG_OK;
}

template <typename E>
int fill_zero_v(E* y, size_t n, cudaStream_t st) {
  WMG_CUDA(cudaMemsetAsync(y, 0, n * sizeof(E), st));
  return MG_OK;
}

template <typename E>
int apply_gamma5_v(E* y, const E* x, size_t nsites_total, cudaStream_t st) {
  gamma5_kernel<E><<<grid_for(nsites_total * 12), 256, 0, st>>>(y, x, nsites_total);
  WMG_LAUNCHED();
  return MG_OK;
}

#define INST(E)                                                                              \
  template int multi_dot_v<E>(zd*, int, const E*, size_t, int, const E*, size_t, int,        \
                              ReduceWork&, cudaStream_t, double);                            \
  template int multi_axpy_v<E>(E*, const E*, size_t, int, const zd*, int, double, size_t,    \
                               int, cudaStream_t);                                           \
  template int norm2_v<E>(double*, int, const E*, size_t, int, ReduceWork&, cudaStream_t,    \
                          double);                                                           \
  template int scale_inv_v<E>(E*, const E*, const double*, int, size_t, int, cudaStream_t); \
  template int axpby_v<E>(E*, double, const E*, double, size_t, int, cudaStream_t);          \
  template int fill_zero_v<E>(E*, size_t, cudaStream_t);                                     \
  template int apply_gamma5_v<E>(E*, const E*, size_t, cudaStream_t);                        \
  template int accumulate_scaled_v<E>(zd*, const E*, const double*, size_t, int, cudaStream_t);
INST(zd)
INST(zf)
INST(zh)
INST(zbf)
#define INSTC(A, B)                                                                          \
  template int convert_v<A, B>(A*, const B*, const double*, int, size_t, int, cudaStream_t); \
  template int axpy_mixed<A, B>(A*, double, const B*, size_t, cudaStream_t);              \
  template int lincomb_v<A, B>(A*, double, const B*, double, const B*, size_t, cudaStream_t);
INSTC(zf, zd)
INSTC(zd, zf)
INSTC(zd, zd)
INSTC(zf, zf)
INSTC(zh, zf)
INSTC(zbf, zf)
INSTC(zf, zh)
INSTC(zf, zbf)
INSTC(zh, zd)
INSTC(zbf, zd)
INSTC(zd, zh)
INSTC(zd, zbf)

}  // namespace wmg
