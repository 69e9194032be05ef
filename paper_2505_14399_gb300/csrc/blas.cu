// Batched BLAS-1 on complex fields with deterministic reductions.
//
// Reductions use a fixed partition of each vector into `nblk` chunks (one CTA each),
// a fixed shuffle/shared-memory tree inside the CTA, and a final fixed-order tree
// over the chunk partials performed by whichever CTA finishes last (its identity
// does not change the arithmetic), so results are bitwise reproducible run to run.
#include "common.cuh"
#include "internal.h"
#include "reduce.cuh"

namespace wmg {

namespace {

template <typename R>
__global__ void __launch_bounds__(RT)
multi_dot_kernel(zd* out, int ldo, const cplx<R>* __restrict__ V, size_t vstride, int nv,
                 const cplx<R>* __restrict__ w, size_t n, double* partial, unsigned* counter,
                 int nblk, int maxvec) {
  __shared__ double sh[(RT / 32) * 8 * 2];
  int rhs = blockIdx.y;
  size_t chunk = reduce_chunk(n, nblk);   // even: 16-byte FP32 pairs
  size_t k0 = (size_t)blockIdx.x * chunk;
  size_t k1 = min(n, k0 + chunk);
  const cplx<R>* wr = w + (size_t)rhs * n;
  // groups of G basis vectors share one pass over w (G independent loads per element)
  constexpr int G = 8;
  for (int i0 = 0; i0 < nv; i0 += G) {
    int ni = min(G, nv - i0);
    R ar[G], ai[G];
#pragma unroll
    for (int q = 0; q < G; ++q) { ar[q] = 0; ai[q] = 0; }
    const cplx<R>* vb = V + (size_t)i0 * vstride + (size_t)rhs * n;
    if (sizeof(R) == 4 && ((k0 | k1 | vstride) & 1) == 0) {
      // FP32: two complex numbers per 16-byte load
      const float4* w4 = reinterpret_cast<const float4*>(wr);
      const float4* v4 = reinterpret_cast<const float4*>(vb);
      size_t vs4 = vstride / 2;
      for (size_t k = k0 / 2 + threadIdx.x; k < k1 / 2; k += RT) {
        float4 b = w4[k];
#pragma unroll
        for (int q = 0; q < G; ++q) {
          if (q < ni) {
            float4 a = v4[(size_t)q * vs4 + k];
            ar[q] = fma((R)a.x, (R)b.x, ar[q]); ar[q] = fma((R)a.y, (R)b.y, ar[q]);
            ar[q] = fma((R)a.z, (R)b.z, ar[q]); ar[q] = fma((R)a.w, (R)b.w, ar[q]);
            ai[q] = fma((R)a.x, (R)b.y, ai[q]); ai[q] = fma(-(R)a.y, (R)b.x, ai[q]);
            ai[q] = fma((R)a.z, (R)b.w, ai[q]); ai[q] = fma(-(R)a.w, (R)b.z, ai[q]);
          }
        }
      }
    } else {
      for (size_t k = k0 + threadIdx.x; k < k1; k += RT) {
        cplx<R> b = wr[k];
#pragma unroll
        for (int q = 0; q < G; ++q) {
          if (q < ni) {
            cplx<R> a = vb[(size_t)q * vstride + k];
            ar[q] = fma(a.re, b.re, ar[q]); ar[q] = fma(a.im, b.im, ar[q]);
            ai[q] = fma(a.re, b.im, ai[q]); ai[q] = fma(-a.im, b.re, ai[q]);
          }
        }
      }
    }
    // CTA reduction in the vectors' own precision (FP64 arithmetic is scarce on this GPU);
    // only the CTA partial is widened to FP64 for the cross-CTA sum.
    cta_store_partials<R, G>(ar, ai, ni, i0, rhs, maxvec, nblk, partial,
                             reinterpret_cast<R*>(sh));
  }
  if (!last_cta(counter, rhs, nblk)) return;
  finish_partials(partial, nv, nblk, maxvec, rhs, out, nullptr, ldo, 0);
  if (threadIdx.x == 0) counter[rhs] = 0;
}

template <typename R>
__global__ void __launch_bounds__(RT)
norm_kernel(double* nrm, int ldn, const cplx<R>* __restrict__ w, size_t n, double* partial,
            unsigned* counter, int nblk, int maxvec) {
  __shared__ double sh[64];
  int rhs = blockIdx.y;
  size_t chunk = reduce_chunk(n, nblk);   // even: 16-byte FP32 pairs
  size_t k0 = (size_t)blockIdx.x * chunk;
  size_t k1 = min(n, k0 + chunk);
  const cplx<R>* wr = w + (size_t)rhs * n;
  R acc = 0;
  for (size_t k = k0 + threadIdx.x; k < k1; k += RT) {
    cplx<R> a = wr[k];
    acc = fma(a.re, a.re, acc);
    acc = fma(a.im, a.im, acc);
  }
  // CTA tree in the vectors' precision, FP64 only across CTAs
  acc = warp_sum_r(acc);
  R* shr = reinterpret_cast<R*>(sh);
  if ((threadIdx.x & 31) == 0) shr[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    R s = 0;
    for (int wv = 0; wv < RT / 32; ++wv) s += shr[wv];
    double* p = partial + ((size_t)rhs * maxvec * nblk + blockIdx.x) * 2;
    p[0] = (double)s;
    p[1] = 0;
    __threadfence();
  }
  if (!last_cta(counter, rhs, nblk)) return;
  finish_partials(partial, 1, nblk, maxvec, rhs, nullptr, nrm, ldn, 1);
  if (threadIdx.x == 0) counter[rhs] = 0;
}

template <typename R>
__global__ void multi_axpy_kernel(cplx<R>* w, const cplx<R>* __restrict__ V, size_t vstride,
                                  int nv, const zd* c, int ldc, double sgn, size_t n) {
  __shared__ cplx<R> cs[128];
  int rhs = blockIdx.y;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    zd v = c[(size_t)rhs * ldc + i];
    cs[i] = {(R)(sgn * v.re), (R)(sgn * v.im)};
  }
  __syncthreads();
  cplx<R>* wr = w + (size_t)rhs * n;
  if (sizeof(R) == 4 && ((n | vstride) & 1) == 0) {
    // FP32: two complex numbers per 16-byte access
    float4* w4 = reinterpret_cast<float4*>(wr);
    const float4* v4 = reinterpret_cast<const float4*>(V + (size_t)rhs * n);
    size_t vs4 = vstride / 2;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n / 2;
         k += (size_t)gridDim.x * blockDim.x) {
      float4 acc = w4[k];
      for (int i = 0; i < nv; ++i) {
        float4 v = v4[(size_t)i * vs4 + k];
        float cr = (float)cs[i].re, ci = (float)cs[i].im;
        acc.x = fmaf(cr, v.x, acc.x); acc.x = fmaf(-ci, v.y, acc.x);
        acc.y = fmaf(cr, v.y, acc.y); acc.y = fmaf(ci, v.x, acc.y);
        acc.z = fmaf(cr, v.z, acc.z); acc.z = fmaf(-ci, v.w, acc.z);
        acc.w = fmaf(cr, v.w, acc.w); acc.w = fmaf(ci, v.z, acc.w);
      }
      w4[k] = acc;
    }
    return;
  }
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    cplx<R> acc = wr[k];
    for (int i = 0; i < nv; ++i) cfma(acc, cs[i], V[(size_t)i * vstride + (size_t)rhs * n + k]);
    wr[k] = acc;
  }
}

// w[rhs] += sgn * sum_i c_i V_i[rhs] and nrm[rhs] = ||w[rhs]|| (after the update) in one pass,
// with the same fixed partition and final tree as norm_kernel.
template <typename R>
__global__ void __launch_bounds__(RT)
multi_axpy_norm_kernel(cplx<R>* w, const cplx<R>* __restrict__ V, size_t vstride, int nv,
                       const zd* c, int ldc, double sgn, size_t n, double* nrm, int ldn,
                       double* partial, unsigned* counter, int nblk, int maxvec) {
  __shared__ cplx<R> cs[128];
  __shared__ double sh[64];
  int rhs = blockIdx.y;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    zd v = c[(size_t)rhs * ldc + i];
    cs[i] = {(R)(sgn * v.re), (R)(sgn * v.im)};
  }
  __syncthreads();
  size_t chunk = reduce_chunk(n, nblk);
  size_t k0 = (size_t)blockIdx.x * chunk;
  size_t k1 = min(n, k0 + chunk);
  cplx<R>* wr = w + (size_t)rhs * n;
  const cplx<R>* vb = V + (size_t)rhs * n;
  R acc2 = 0;
  if (sizeof(R) == 4 && ((k0 | k1 | vstride) & 1) == 0) {
    float4* w4 = reinterpret_cast<float4*>(wr);
    const float4* v4 = reinterpret_cast<const float4*>(vb);
    size_t vs4 = vstride / 2;
    for (size_t k = k0 / 2 + threadIdx.x; k < k1 / 2; k += RT) {
      float4 a = w4[k];
      for (int i = 0; i < nv; ++i) {
        float4 v = v4[(size_t)i * vs4 + k];
        float cr = (float)cs[i].re, ci = (float)cs[i].im;
        a.x = fmaf(cr, v.x, a.x); a.x = fmaf(-ci, v.y, a.x);
        a.y = fmaf(cr, v.y, a.y); a.y = fmaf(ci, v.x, a.y);
        a.z = fmaf(cr, v.z, a.z); a.z = fmaf(-ci, v.w, a.z);
        a.w = fmaf(cr, v.w, a.w); a.w = fmaf(ci, v.z, a.w);
      }
      w4[k] = a;
      acc2 = fma((R)a.x, (R)a.x, acc2); acc2 = fma((R)a.y, (R)a.y, acc2);
      acc2 = fma((R)a.z, (R)a.z, acc2); acc2 = fma((R)a.w, (R)a.w, acc2);
    }
  } else {
    for (size_t k = k0 + threadIdx.x; k < k1; k += RT) {
      cplx<R> a = wr[k];
      for (int i = 0; i < nv; ++i) cfma(a, cs[i], vb[(size_t)i * vstride + k]);
      wr[k] = a;
      acc2 = fma(a.re, a.re, acc2);
      acc2 = fma(a.im, a.im, acc2);
    }
  }
  acc2 = warp_sum_r(acc2);
  R* shr = reinterpret_cast<R*>(sh);
  if ((threadIdx.x & 31) == 0) shr[threadIdx.x >> 5] = acc2;
  __syncthreads();
  if (threadIdx.x == 0) {
    R s = 0;
    for (int wv = 0; wv < RT / 32; ++wv) s += shr[wv];
    double* p = partial + ((size_t)rhs * maxvec * nblk + blockIdx.x) * 2;
    p[0] = (double)s;
    p[1] = 0;
    __threadfence();
  }
  if (!last_cta(counter, rhs, nblk)) return;
  finish_partials(partial, 1, nblk, maxvec, rhs, nullptr, nrm, ldn, 1);
  if (threadIdx.x == 0) counter[rhs] = 0;
}

template <typename R>
__global__ void scale_inv_kernel(cplx<R>* y, const cplx<R>* x, const double* s, int lds, size_t n) {
  int rhs = blockIdx.y;
  double sv = s[(size_t)rhs * lds];
  R f = sv > 0 ? (R)(1.0 / sv) : (R)0;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    cplx<R> v = x[(size_t)rhs * n + k];
    y[(size_t)rhs * n + k] = {f * v.re, f * v.im};
  }
}

template <typename R>
__global__ void axpby_kernel(cplx<R>* y, R a, const cplx<R>* x, R b, size_t n) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    cplx<R> xv = x[k], yv = y[k];
    y[k] = {fma(a, xv.re, b * yv.re), fma(a, xv.im, b * yv.im)};
  }
}

template <typename Ro, typename Ri>
__global__ void convert_kernel(cplx<Ro>* y, const cplx<Ri>* x, const double* s, int inv, size_t n) {
  int rhs = blockIdx.y;
  double f = 1.0;
  if (s) {
    double sv = s[rhs];
    f = inv ? (sv > 0 ? 1.0 / sv : 0.0) : sv;
  }
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    cplx<Ri> v = x[(size_t)rhs * n + k];
    y[(size_t)rhs * n + k] = {(Ro)(f * (double)v.re), (Ro)(f * (double)v.im)};
  }
}

template <typename Ri>
__global__ void accumulate_scaled_kernel(zd* y, const cplx<Ri>* x, const double* s, size_t n) {
  int rhs = blockIdx.y;
  double f = s[rhs];
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    cplx<Ri> v = x[(size_t)rhs * n + k];
    zd& t = y[(size_t)rhs * n + k];
    t.re = fma(f, (double)v.re, t.re);
    t.im = fma(f, (double)v.im, t.im);
  }
}

template <typename R>
__global__ void gamma5_kernel(cplx<R>* y, const cplx<R>* x, size_t nsites) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < nsites * 12;
       k += (size_t)gridDim.x * blockDim.x) {
    int comp = (int)(k % 12);
    cplx<R> v = x[k];
    y[k] = comp >= 6 ? cplx<R>{-v.re, -v.im} : v;
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
  maxvec = mv;
  nrhs_cap = nrhs;
  WMG_CUDA(cudaMalloc(&partial, sizeof(double) * 2 * (size_t)nblk * maxvec * nrhs));
  WMG_CUDA(cudaMalloc(&counter, sizeof(unsigned) * nrhs));
  WMG_CUDA(cudaMemset(counter, 0, sizeof(unsigned) * nrhs));
  return MG_OK;
}

void ReduceWork::release() {
  if (partial) cudaFree(partial);
  if (counter) cudaFree(counter);
  partial = nullptr;
  counter = nullptr;
}

template <typename R>
int multi_dot(zd* out, int ldo, const cplx<R>* V, size_t vstride, int nv, const cplx<R>* w,
              size_t n, int nrhs, ReduceWork& rw, cudaStream_t st) {
  if (nv > rw.maxvec || nrhs > rw.nrhs_cap) return fail(MG_EINVAL, "multi_dot: workspace too small");
  dim3 grid(rw.nblk, nrhs);
  ProfScope ps("multi_dot", (double)(nv + 1) * nrhs * n * sizeof(cplx<R>), 8.0 * nv * n * nrhs, st);
  multi_dot_kernel<R><<<grid, RT, 0, st>>>(out, ldo, V, vstride, nv, w, n, rw.partial,
                                           rw.counter, rw.nblk, rw.maxvec);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int multi_axpy(cplx<R>* w, const cplx<R>* V, size_t vstride, int nv, const zd* c, int ldc,
               double sgn, size_t n, int nrhs, cudaStream_t st) {
  if (nv > 128) return fail(MG_EINVAL, "multi_axpy: too many vectors");
  if (nv == 0) return MG_OK;
  dim3 grid(grid_for(n), nrhs);
  ProfScope ps("multi_axpy", (double)(nv + 2) * nrhs * n * sizeof(cplx<R>), 8.0 * nv * n * nrhs, st);
  multi_axpy_kernel<R><<<grid, 256, 0, st>>>(w, V, vstride, nv, c, ldc, sgn, n);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int norm2(double* nrm, int ldn, const cplx<R>* w, size_t n, int nrhs, ReduceWork& rw,
          cudaStream_t st) {
  if (nrhs > rw.nrhs_cap) return fail(MG_EINVAL, "norm2: workspace too small");
  dim3 grid(rw.nblk, nrhs);
  ProfScope ps("norm", (double)nrhs * n * sizeof(cplx<R>), 4.0 * n * nrhs, st);
  norm_kernel<R><<<grid, RT, 0, st>>>(nrm, ldn, w, n, rw.partial, rw.counter, rw.nblk, rw.maxvec);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int multi_axpy_norm(cplx<R>* w, const cplx<R>* V, size_t vstride, int nv, const zd* c, int ldc,
                    double sgn, size_t n, int nrhs, double* nrm, int ldn, ReduceWork& rw,
                    cudaStream_t st) {
  if (nv > 128) return fail(MG_EINVAL, "multi_axpy_norm: too many vectors");
  if (nrhs > rw.nrhs_cap) return fail(MG_EINVAL, "multi_axpy_norm: workspace too small");
  dim3 grid(rw.nblk, nrhs);
  multi_axpy_norm_kernel<R><<<grid, RT, 0, st>>>(w, V, vstride, nv, c, ldc, sgn, n, nrm, ldn,
                                                 rw.partial, rw.counter, rw.nblk, rw.maxvec);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int scale_inv(cplx<R>* y, const cplx<R>* x, const double* s, int lds, size_t n, int nrhs,
              cudaStream_t st) {
  dim3 grid(grid_for(n), nrhs);
  ProfScope ps("scale", 2.0 * nrhs * n * sizeof(cplx<R>), 2.0 * n * nrhs, st);
  scale_inv_kernel<R><<<grid, 256, 0, st>>>(y, x, s, lds, n);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int axpby(cplx<R>* y, double a, const cplx<R>* x, double b, size_t n, int nrhs, cudaStream_t st) {
  size_t tot = n * nrhs;
  axpby_kernel<R><<<grid_for(tot), 256, 0, st>>>(y, (R)a, x, (R)b, tot);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename Ro, typename Ri>
int convert(cplx<Ro>* y, const cplx<Ri>* x, const double* s, int inv, size_t n, int nrhs,
            cudaStream_t st) {
  dim3 grid(grid_for(n), nrhs);
  convert_kernel<Ro, Ri><<<grid, 256, 0, st>>>(y, x, s, inv, n);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename Ri>
int accumulate_scaled(zd* y, const cplx<Ri>* x, const double* s, size_t n, int nrhs,
                      cudaStream_t st) {
  dim3 grid(grid_for(n), nrhs);
  accumulate_scaled_kernel<Ri><<<grid, 256, 0, st>>>(y, x, s, n);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int fill_zero(cplx<R>* y, size_t n, cudaStream_t st) {
  WMG_CUDA(cudaMemsetAsync(y, 0, n * sizeof(cplx<R>), st));
  return MG_OK;
}

template <typename R>
int apply_gamma5(cplx<R>* y, const cplx<R>* x, size_t nsites_total, cudaStream_t st) {
  gamma5_kernel<R><<<grid_for(nsites_total * 12), 256, 0, st>>>(y, x, nsites_total);
  WMG_LAUNCHED();
  return MG_OK;
}

#define INST(R)                                                                            \
  template int multi_dot<R>(zd*, int, const cplx<R>*, size_t, int, const cplx<R>*, size_t, \
                            int, ReduceWork&, cudaStream_t);                              \
  template int multi_axpy<R>(cplx<R>*, const cplx<R>*, size_t, int, const zd*, int, double, \
                             size_t, int, cudaStream_t);                                   \
  template int norm2<R>(double*, int, const cplx<R>*, size_t, int, ReduceWork&, cudaStream_t); \
  template int multi_axpy_norm<R>(cplx<R>*, const cplx<R>*, size_t, int, const zd*, int,   \
                                  double, size_t, int, double*, int, ReduceWork&,          \
                                  cudaStream_t);                                           \
  template int scale_inv<R>(cplx<R>*, const cplx<R>*, const double*, int, size_t, int,     \
                            cudaStream_t);                                                 \
  template int axpby<R>(cplx<R>*, double, const cplx<R>*, double, size_t, int, cudaStream_t); \
  template int fill_zero<R>(cplx<R>*, size_t, cudaStream_t);                               \
  template int apply_gamma5<R>(cplx<R>*, const cplx<R>*, size_t, cudaStream_t);            \
  template int accumulate_scaled<R>(zd*, const cplx<R>*, const double*, size_t, int, cudaStream_t);
INST(float)
INST(double)
template int convert<float, double>(zf*, const zd*, const double*, int, size_t, int, cudaStream_t);
template int convert<double, float>(zd*, const zf*, const double*, int, size_t, int, cudaStream_t);
template int convert<double, double>(zd*, const zd*, const double*, int, size_t, int, cudaStream_t);
template int convert<float, float>(zf*, const zf*, const double*, int, size_t, int, cudaStream_t);

}  // namespace wmg
