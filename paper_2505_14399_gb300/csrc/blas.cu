// Batched BLAS-1 on complex fields with deterministic reductions.
//
// Reductions use a fixed partition of each vector into `nblk` chunks (one CTA each),
// a fixed shuffle/shared-memory tree inside the CTA, and a final fixed-order tree
// over the chunk partials performed by whichever CTA finishes last (its identity
// does not change the arithmetic), so results are bitwise reproducible run to run.
#include "common.cuh"
#include "internal.h"

namespace wmg {

namespace {

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

// CTA sum of (a, b); result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
  a = warp_sum(a);
  b = warp_sum(b);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh[2 * wid] = a; sh[2 * wid + 1] = b; }
  __syncthreads();
  if (wid == 0) {
    int nw = blockDim.x >> 5;
    a = lane < nw ? sh[2 * lane] : 0.0;
    b = lane < nw ? sh[2 * lane + 1] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
  __syncthreads();
}

// Final reduction over the nblk partials of every (rhs, i), done by the last CTA.
// mode 0: complex dot -> out[rhs*ldo + i]; mode 1: norm -> dout[rhs*ldo] = sqrt(re).
__device__ void finish_partials(double* partial, int nv, int nblk, int maxvec, int rhs,
                                zd* out, double* dout, int ldo, int mode, double* sh) {
  for (int i = 0; i < nv; ++i) {
    const double* p = partial + ((size_t)rhs * maxvec + i) * nblk * 2;
    double a = 0, b = 0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) {
      a += __ldcg(p + 2 * k);
      b += __ldcg(p + 2 * k + 1);
    }
    block_sum2(a, b, sh);
    if (threadIdx.x == 0) {
      if (mode == 0) out[(size_t)rhs * ldo + i] = {a, b};
      else dout[(size_t)rhs * ldo] = sqrt(a);
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(RT)
multi_dot_kernel(zd* out, int ldo, const cplx<R>* __restrict__ V, size_t vstride, int nv,
                 const cplx<R>* __restrict__ w, size_t n, double* partial, unsigned* counter,
                 int nblk, int maxvec) {
  __shared__ double sh[(RT / 32) * 8 * 2];
  __shared__ bool last;
  int rhs = blockIdx.y;
  size_t chunk = (n + nblk - 1) / nblk;
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
    // CTA reduction of the ni pairs in the vectors' own precision (FP64 arithmetic is
    // scarce on this GPU): warp shuffles, then one shared-memory pass; only the CTA
    // partial is widened to FP64 for the cross-CTA sum.
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    R* shg = reinterpret_cast<R*>(sh);  // [RT/32][G][2]
#pragma unroll
    for (int q = 0; q < G; ++q) {
      if (q < ni) {
        R dr = warp_sum_r(ar[q]);
        R di = warp_sum_r(ai[q]);
        if (lane == 0) { shg[(wid * G + q) * 2] = dr; shg[(wid * G + q) * 2 + 1] = di; }
      }
    }
    __syncthreads();
    if (threadIdx.x < 2 * ni) {
      int q = threadIdx.x >> 1, part = threadIdx.x & 1;
      R s = 0;
      for (int wv = 0; wv < RT / 32; ++wv) s += shg[(wv * G + q) * 2 + part];
      partial[(((size_t)rhs * maxvec + i0 + q) * nblk + blockIdx.x) * 2 + part] = (double)s;
    }
    __syncthreads();
  }
  __threadfence();
  if (threadIdx.x == 0) last = (atomicAdd(counter + rhs, 1u) == (unsigned)nblk - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  finish_partials(partial, nv, nblk, maxvec, rhs, out, nullptr, ldo, 0, sh);
  if (threadIdx.x == 0) counter[rhs] = 0;
}

template <typename R>
__global__ void __launch_bounds__(RT)
norm_kernel(double* nrm, int ldn, const cplx<R>* __restrict__ w, size_t n, double* partial,
            unsigned* counter, int nblk, int maxvec) {
  __shared__ double sh[64];
  __shared__ bool last;
  int rhs = blockIdx.y;
  size_t chunk = (n + nblk - 1) / nblk;
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
  }
  __threadfence();
  if (threadIdx.x == 0) last = (atomicAdd(counter + rhs, 1u) == (unsigned)nblk - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  finish_partials(partial, 1, nblk, maxvec, rhs, nullptr, nrm, ldn, 1, sh);
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
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    cplx<R> acc = wr[k];
    for (int i = 0; i < nv; ++i) cfma(acc, cs[i], V[(size_t)i * vstride + (size_t)rhs * n + k]);
    wr[k] = acc;
  }
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
  multi_axpy_kernel<R><<<grid, 256, 0, st>>>(w, V, vstride, nv, c, ldc, sgn, n);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int norm2(double* nrm, int ldn, const cplx<R>* w, size_t n, int nrhs, ReduceWork& rw,
          cudaStream_t st) {
  if (nrhs > rw.nrhs_cap) return fail(MG_EINVAL, "norm2: workspace too small");
  dim3 grid(rw.nblk, nrhs);
  norm_kernel<R><<<grid, RT, 0, st>>>(nrm, ldn, w, n, rw.partial, rw.counter, rw.nblk, rw.maxvec);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int scale_inv(cplx<R>* y, const cplx<R>* x, const double* s, int lds, size_t n, int nrhs,
              cudaStream_t st) {
  dim3 grid(grid_for(n), nrhs);
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
