// Batched GMRES / flexible GMRES with all Krylov scalars resident on the device.
//
// Arnoldi uses classical Gram-Schmidt applied twice (CGS2: two batched dot passes and
// two batched updates per step; single-pass for the fixed-step FP32 smoothers), the
// Hessenberg column is reduced by complex Givens rotations by one extra CTA of the step's
// normalising update, and the residual estimates |g_{j+1}| (one per step, kept on the device)
// are the only values the host reads, every `check_every` steps of a tolerance-driven solve.
// All nrhs systems advance in lockstep.
#include <cmath>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "reduce.cuh"
#include "stencil.cuh"
#include "tma.cuh"
#include "vec.cuh"

namespace wmg {

namespace {

// Per-system layout of the device scalar block (units of zd):
//   H[(m+1) x m] column-major | h2[m+1] | cs[m] (real in .re) | sn[m] | g[m+1] | y[m]
struct SmallLayout {
  int m;
  __host__ __device__ int stride() const { return (m + 1) * m + (m + 1) + m + m + (m + 1) + m; }
  __host__ __device__ int H() const { return 0; }
  __host__ __device__ int h2() const { return (m + 1) * m; }
  __host__ __device__ int cs() const { return h2() + m + 1; }
  __host__ __device__ int sn() const { return cs() + m; }
  __host__ __device__ int g() const { return sn() + m; }
  __host__ __device__ int y() const { return g() + m + 1; }
};

__global__ void init_kernel(zd* small, SmallLayout L, const double* beta, double* res, int nrhs) {
  dep_entry();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  zd* s = small + (size_t)r * L.stride();
  for (int i = 0; i < L.stride(); ++i) s[i] = {0, 0};
  s[L.g()] = {beta[r], 0};
  res[r] = beta[r];
}

// Finish column j of one system's Hessenberg matrix: H[:, j] += h2, H[j+1, j] = ||w||,
// apply the previous rotations, form the new one, update g; returns |g_{j+1}|.
// col = H[:, j] (j + 2 entries), h2 (j + 1), cs / sn (rotations 0..j; entry j is written),
// gp = {g_j, g_{j+1}}.  The arrays may live in global or shared memory.
__device__ double givens_core(zd* col, const zd* h2, zd* cs, zd* sn, zd* gp, int j,
                              double wnorm) {
  for (int i = 0; i <= j; ++i) col[i] = col[i] + h2[i];
  col[j + 1] = {wnorm, 0};
  for (int i = 0; i < j; ++i) {
    double c = cs[i].re;
    zd sv = sn[i];
    zd a = col[i], b = col[i + 1];
    zd na = c * a + sv * b;
    zd nb = c * b - cmulc(sv, a);  // -conj(s) a + c b
    col[i] = na;
    col[i + 1] = nb;
  }
  // c = |a| / rho, s = (a / |a|) conj(b) / rho with rho^2 = |a|^2 + |b|^2, from two
  // reciprocal square roots (one thread's serial FP64 chain: no hypot, sqrt or divide)
  zd a = col[j], b = col[j + 1];
  double na2 = norm2(a), rho2 = na2 + norm2(b);
  double c;
  zd sv;
  if (!(rho2 > 0.0)) {
    c = 1.0;
    sv = {0, 0};
  } else if (!(na2 > 0.0)) {
    double ir = rsqrt(rho2);
    c = 0.0;
    sv = {b.re * ir, -b.im * ir};  // s b = |b|^2/rho: choose s = conj(b)/rho
  } else {
    double ir = rsqrt(rho2), ina = rsqrt(na2);
    c = na2 * ina * ir;
    sv = (ina * ir) * (a * conj(b));
  }
  zd top = c * a + sv * b;
  col[j] = top;
  col[j + 1] = {0, 0};
  cs[j] = {c, 0};
  sn[j] = sv;
  zd gj = gp[0];
  gp[0] = c * gj;
  gp[1] = -cmulc(sv, gj);  // -conj(s) g_j
  return sqrt(norm2(gp[1]));
}

// Column j of the Hessenberg matrix and its Givens step, run by one whole CTA on shared-memory
// copies (one thread's chain of dependent updates then touches shared memory, not L2): the
// column gets the projections h2 (added to the pass-1 values, or alone when `single`) and
// H[j+1, j] = beta; the rotation updates cs, sn, g and the residual estimate res.  Called by
// the extra CTA of the normalising update, so this serial FP64 chain runs beside the
// memory-bound update instead of ending the reduction sweep.
constexpr int GV_MAX = 130;   // m <= 128
__device__ void givens_deferred(zd* sm, SmallLayout L, int j, double beta, bool single,
                                double* res) {
  __shared__ zd g_col[GV_MAX], g_h2[GV_MAX], g_cs[GV_MAX], g_sn[GV_MAX], g_g[2];
  const zd* colg = sm + L.H() + (size_t)j * (L.m + 1);
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) g_col[i] = single ? zd{0, 0} : colg[i];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) g_h2[i] = sm[L.h2() + i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    g_cs[i] = sm[L.cs() + i];
    g_sn[i] = sm[L.sn() + i];
  }
  if (threadIdx.x < 2) g_g[threadIdx.x] = sm[L.g() + j + threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) *res = givens_core(g_col, g_h2, g_cs, g_sn, g_g, j, beta);
  __syncthreads();
  zd* colw = sm + L.H() + (size_t)j * (L.m + 1);
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) colw[i] = g_col[i];
  if (threadIdx.x == 0) {
    sm[L.cs() + j] = g_cs[j];
    sm[L.sn() + j] = g_sn[j];
  }
  if (threadIdx.x < 2) sm[L.g() + j + threadIdx.x] = g_g[threadIdx.x];
}

// CGS pass 1 update fused with the pass 2 projections and the norm:
//   w -= sum_i h1_i V_i,  then  h2_i = V_i^dag w (i < nv)  and  s = ||w||^2, one sweep over w.
// The last CTA stores h2 and H[j+1, j]: with V orthonormal, the vector left after the pass 2
// update, w - V h2, has squared norm s - ||h2||^2 (Pythagoras), so the pass 2 update needs no
// reduction of its own (it also completes the Hessenberg column and the Givens step).  h2 is
// O(eps ||A v_j||) after pass 1, so the subtraction loses nothing unless the Krylov space is
// (numerically) invariant, where H[j+1, j] ~ 0 ends the solve anyway.
template <typename E>
__global__ void __launch_bounds__(RT, 3)
cgs_update_dot_kernel(E* w, const E* __restrict__ V, size_t vstride, int nv,
                      zd* small, SmallLayout L, int j, size_t n, double* wnorm, double* res,
                      double* partial, unsigned* counter, int nblk, int maxvec, double scale) {
  dep_entry();
  typedef VecT<E> T;
  typedef typename T::R R;
  constexpr int G = 8;
  __shared__ cplx<R> cs[128];
  __shared__ double sh[(RT / 32) * G * 2];
  int rhs = blockIdx.y;
  zd* sm = small + (size_t)rhs * L.stride();
  const zd* c = sm + L.H() + (size_t)j * (L.m + 1);
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    zd v = c[i];
    cs[i] = {(R)(-v.re), (R)(-v.im)};
  }
  __syncthreads();
  size_t chunk = reduce_chunk(n, nblk);
  size_t k0 = (size_t)blockIdx.x * chunk;
  size_t k1 = min(n, k0 + chunk);
  E* wr = w + (size_t)rhs * n;
  const E* vb = V + (size_t)rhs * n;
  R ss = 0;
  bool packed = false;
  if constexpr (T::packed) packed = nv <= G && ((k0 | k1 | vstride) & 1) == 0;
  if (packed) {
    // one sweep: the basis entries stay in registers between the update and the dots
    R ar[G], ai[G];
#pragma unroll
    for (int q = 0; q < G; ++q) { ar[q] = 0; ai[q] = 0; }
    size_t vs2 = vstride / 2;
    for (size_t k = k0 / 2 + threadIdx.x; k < k1 / 2; k += RT) {
      float4 a = T::ld2(wr, k);
      float4 v[G];
#pragma unroll
      for (int q = 0; q < G; ++q) {
        if (q < nv) {
          v[q] = T::ld2(vb + (size_t)q * 2 * vs2, k);
          float cr = (float)cs[q].re, ci = (float)cs[q].im;
          a.x = fmaf(cr, v[q].x, a.x); a.x = fmaf(-ci, v[q].y, a.x);
          a.y = fmaf(cr, v[q].y, a.y); a.y = fmaf(ci, v[q].x, a.y);
          a.z = fmaf(cr, v[q].z, a.z); a.z = fmaf(-ci, v[q].w, a.z);
          a.w = fmaf(cr, v[q].w, a.w); a.w = fmaf(ci, v[q].z, a.w);
        }
      }
      a = T::rnd2(a);   // continue with the values as stored
      T::st2(wr, k, a);
      ss = fma((R)a.x, (R)a.x, ss); ss = fma((R)a.y, (R)a.y, ss);
      ss = fma((R)a.z, (R)a.z, ss); ss = fma((R)a.w, (R)a.w, ss);
#pragma unroll
      for (int q = 0; q < G; ++q) {
        if (q < nv) {
          ar[q] = fma((R)v[q].x, (R)a.x, ar[q]); ar[q] = fma((R)v[q].y, (R)a.y, ar[q]);
          ar[q] = fma((R)v[q].z, (R)a.z, ar[q]); ar[q] = fma((R)v[q].w, (R)a.w, ar[q]);
          ai[q] = fma((R)v[q].x, (R)a.y, ai[q]); ai[q] = fma(-(R)v[q].y, (R)a.x, ai[q]);
          ai[q] = fma((R)v[q].z, (R)a.w, ai[q]); ai[q] = fma(-(R)v[q].w, (R)a.z, ai[q]);
        }
      }
    }
    cta_store_partials<R, G>(ar, ai, nv, 0, rhs, maxvec, nblk, partials_as<R>(partial),
                             reinterpret_cast<R*>(sh));
  } else {
    // general case: update sweep (with the norm), then projection sweeps over groups of G
    for (size_t k = k0 + threadIdx.x; k < k1; k += RT) {
      cplx<R> a = T::ld(wr, k);
      for (int i = 0; i < nv; ++i) cfma(a, cs[i], T::ld(vb, (size_t)i * vstride + k));
      a = T::rnd(a);
      T::st(wr, k, a);
      ss = fma(a.re, a.re, ss);
      ss = fma(a.im, a.im, ss);
    }
    // projections on the updated w (each thread rereads its own elements: L1/L2 hits)
    for (int i0 = 0; i0 < nv; i0 += G) {
      int ni = min(G, nv - i0);
      R ar[G], ai[G];
#pragma unroll
      for (int q = 0; q < G; ++q) { ar[q] = 0; ai[q] = 0; }
      for (size_t k = k0 + threadIdx.x; k < k1; k += RT) {
        cplx<R> b = T::ld(wr, k);
#pragma unroll
        for (int q = 0; q < G; ++q) {
          if (q < ni) {
            cplx<R> a = T::ld(vb, (size_t)(i0 + q) * vstride + k);
            ar[q] = fma(a.re, b.re, ar[q]); ar[q] = fma(a.im, b.im, ar[q]);
            ai[q] = fma(a.re, b.im, ai[q]); ai[q] = fma(-a.im, b.re, ai[q]);
          }
        }
      }
      cta_store_partials<R, G>(ar, ai, ni, i0, rhs, maxvec, nblk, partials_as<R>(partial),
                               reinterpret_cast<R*>(sh));
    }
  }
  // ||w||^2 goes to slot nv (< maxvec: nv <= m)
  R zero = 0;
  cta_store_partials<R, 1>(&ss, &zero, 1, nv, rhs, maxvec, nblk, partials_as<R>(partial),
                           reinterpret_cast<R*>(sh));
  if (!last_cta(counter, rhs, nblk)) return;
  finish_partials(partials_as<R>(partial), nv + 1, nblk, maxvec, rhs, small + L.h2(), nullptr,
                  L.stride(), 0,
                  scale);
  __syncthreads();
  if (threadIdx.x == 0) {
    counter[rhs] = 0;
    const zd* h2 = sm + L.h2();
    double hh = 0;
    for (int i = 0; i < nv; ++i) hh += norm2(h2[i]);
    double b2 = h2[nv].re - hh;
    wnorm[rhs] = b2 > 0 ? sqrt(b2) : 0.0;   // the Givens step follows in the update
  }
}

// CGS pass 2 update written straight into the next basis column:
//   v_{j+1} = (w - sum_i h2_i V_i) / H[j+1, j]   (0 if H[j+1, j] = 0).
// The last CTA of every rhs row does not update: it completes Hessenberg column j = nv - 1
// and its Givens step (givens_deferred) while the others stream the vectors.
template <typename E>
__global__ void __launch_bounds__(256)
cgs_update_scale_kernel(E* vout, const E* __restrict__ w, const E* __restrict__ V,
                        size_t vstride, int nv, zd* small, SmallLayout L,
                        const double* wnorm, size_t n, double* res, int single) {
  dep_entry();
  typedef VecT<E> T;
  typedef typename T::R R;
  __shared__ cplx<R> cs[128];
  int rhs = blockIdx.y;
  if (blockIdx.x == gridDim.x - 1) {
    givens_deferred(small + (size_t)rhs * L.stride(), L, nv - 1, wnorm[rhs], single != 0,
                    res + (size_t)(nv - 1) * gridDim.y + rhs);
    return;
  }
  const size_t nthreads = (size_t)(gridDim.x - 1) * blockDim.x;
  const zd* h2 = small + (size_t)rhs * L.stride() + L.h2();
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cs[i] = {(R)(-h2[i].re), (R)(-h2[i].im)};
  __syncthreads();
  double beta = wnorm[rhs];
  R f = beta > 0 ? (R)(1.0 / beta) : (R)0;
  const E* wr = w + (size_t)rhs * n;
  const E* vb = V + (size_t)rhs * n;
  E* outr = vout + (size_t)rhs * n;
  bool packed = false;
  if constexpr (T::packed) packed = ((n | vstride) & 1) == 0;
  if (packed) {
    size_t vs2 = vstride / 2;
    float ff = (float)f;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n / 2; k += nthreads) {
      float4 a = T::ld2(wr, k);
      for (int i = 0; i < nv; ++i) {
        float4 v = T::ld2(vb + (size_t)i * 2 * vs2, k);
        float cr = (float)cs[i].re, ci = (float)cs[i].im;
        a.x = fmaf(cr, v.x, a.x); a.x = fmaf(-ci, v.y, a.x);
        a.y = fmaf(cr, v.y, a.y); a.y = fmaf(ci, v.x, a.y);
        a.z = fmaf(cr, v.z, a.z); a.z = fmaf(-ci, v.w, a.z);
        a.w = fmaf(cr, v.w, a.w); a.w = fmaf(ci, v.z, a.w);
      }
      T::st2(outr, k, make_float4(ff * a.x, ff * a.y, ff * a.z, ff * a.w));
    }
    return;
  }
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += nthreads) {
    cplx<R> a = T::ld(wr, k);
    for (int i = 0; i < nv; ++i) cfma(a, cs[i], T::ld(vb, (size_t)i * vstride + k));
    T::st(outr, k, {f * a.re, f * a.im});
  }
}

// ---------------------------------------------------------------- bulk-copy fed CGS sweeps
// Complex-float bases of at most ST_NV columns.  Each CTA owns one contiguous chunk of every
// vector (the fixed partition of the reductions) and streams it through shared memory in
// tiles (1024 or 512 elements): thread 0 issues one bulk copy per vector and tile into a ring of
// `stages` buffers, completion arrives as transaction bytes on the stage's mbarrier, and
// the CTA computes from shared memory while the following tiles are in flight.  The bytes
// in flight per SM no longer depend on registers (the register-fed sweeps above reached a
// third of the HBM bandwidth at their occupancy).
//   MODE 0: h_i = V_i^dag w                      (CGS pass 1 projections)
//   MODE 1: w -= V c; h2_i = V_i^dag w; ||w||^2; H[j+1, j] as in cgs_update_dot_kernel
//   MODE 2: h_i = V_i^dag w and ||w||^2; H[j+1, j]^2 = ||w||^2 - ||h||^2 (single-pass
//           classical Gram-Schmidt; see GmresV::fixed)
// In modes 1 and 2 the Hessenberg column and its Givens step are completed by the
// normalising update that follows (givens_deferred).
// A bounded wait that gives up sets *err, waits (bounded) for the CTA's copies in flight
// and returns; the caller reports MG_ETIMEOUT.
constexpr int ST_NV = 16;      // columns handled (NVM = 8 or 16 accumulator sets)
constexpr int ST_MAXS = 6;
constexpr int ST_WAIT = 1 << 20;

// Tile length (complex elements per vector, a multiple of 2 RT) and ring depth: about
// 100 KB of copies in flight per CTA, two CTAs per SM.
__host__ __device__ inline int st_te(int nv) { return nv <= 3 ? 4 * RT : 2 * RT; }
__host__ __device__ inline int st_stages(int nv) {
  return nv <= 1 ? 6 : nv <= 3 ? 3 : nv <= 5 ? 4 : nv <= 8 ? 3 : 2;
}
__host__ __device__ inline size_t st_smem(int nv) {
  return (size_t)st_stages(nv) * (nv + 1) * st_te(nv) * sizeof(zf);
}

template <int MODE, int NVM>
__global__ void __launch_bounds__(RT)
stream_cgs_kernel(zf* w, const zf* __restrict__ V, size_t vstride, int nv, size_t n, zd* out,
                  int ldo, zd* small, SmallLayout L, int j, double* wnorm, double* res,
                  double* partial, unsigned* counter, int nblk, int maxvec, double scale,
                  int* err) {
  extern __shared__ __align__(16) unsigned char st_raw[];
  __shared__ uint64_t bars[ST_MAXS];
  __shared__ float sh[(RT / 32) * NVM * 2];
  __shared__ zf cs[NVM];
  float4* buf = reinterpret_cast<float4*>(st_raw);
  const int stages = st_stages(nv);
  const int te = st_te(nv);
  const int tp = te / 2;   // float4 packs per vector and tile
  const int nvec = nv + 1;
  int rhs = blockIdx.y;
  zd* sm = small ? small + (size_t)rhs * L.stride() : nullptr;
  size_t chunk = reduce_chunk(n, nblk);
  size_t k0 = (size_t)blockIdx.x * chunk;
  size_t k1 = min(n, k0 + chunk);
  size_t len = k1 > k0 ? k1 - k0 : 0;
  int ntiles = (int)((len + te - 1) / te);
  zf* wr = w + (size_t)rhs * n;
  const zf* vb = V + (size_t)rhs * n;
  if (threadIdx.x == 0) {
    for (int st = 0; st < stages; ++st) mbar_init(&bars[st], 1);
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int it) {   // thread 0: tile `it` of every vector into stage it % stages
    int st = it % stages;
    size_t e0 = k0 + (size_t)it * te;
    uint32_t cnt = (uint32_t)min((size_t)te, k1 - e0);
    uint32_t bytes = cnt * (uint32_t)sizeof(zf);
    mbar_arrive_expect_tx(&bars[st], bytes * nvec);
    bulk_g2s(buf + (size_t)(st * nvec) * tp, wr + e0, bytes, &bars[st]);
    for (int q = 0; q < nv; ++q)
      bulk_g2s(buf + (size_t)(st * nvec + 1 + q) * tp, vb + (size_t)q * vstride + e0, bytes,
               &bars[st]);
  };
  // dependent launch: w comes from the previous kernel in projection mode; in update mode w
  // and V are unchanged by it (only the coefficients are new), so the first tiles are in
  // flight before the wait
  if (MODE != 1) dep_wait();
  if (threadIdx.x == 0)
    for (int it = 0; it < stages && it < ntiles; ++it) issue(it);
  if (MODE == 1) dep_wait();
  dep_trigger();
  if (MODE == 1 && threadIdx.x < nv) {
    zd c = sm[L.H() + (size_t)j * (L.m + 1) + threadIdx.x];
    cs[threadIdx.x] = {(float)(-c.re), (float)(-c.im)};
  }
  __syncthreads();
  float ar[NVM], ai[NVM];
#pragma unroll
  for (int q = 0; q < NVM; ++q) { ar[q] = 0.f; ai[q] = 0.f; }
  float ss = 0.f;
  int failed_at = -1;
  for (int it = 0; it < ntiles; ++it) {
    int st = it % stages;
    bool ok = mbar_wait(&bars[st], (uint32_t)((it / stages) & 1), ST_WAIT);
    if (ok) {
      size_t e0 = (size_t)it * te;
      int cnt = (int)min((size_t)te, len - e0);
      const float4* sb = buf + (size_t)(st * nvec) * tp;
      for (int p = threadIdx.x; 2 * p < cnt; p += RT) {
        float4 a = sb[p];
        if (MODE == 1) {
#pragma unroll
          for (int q = 0; q < NVM; ++q) {
            if (q < nv) {
              float4 v = sb[(size_t)(1 + q) * tp + p];
              float cr = cs[q].re, ci = cs[q].im;
              a.x = fmaf(cr, v.x, a.x); a.x = fmaf(-ci, v.y, a.x);
              a.y = fmaf(cr, v.y, a.y); a.y = fmaf(ci, v.x, a.y);
              a.z = fmaf(cr, v.z, a.z); a.z = fmaf(-ci, v.w, a.z);
              a.w = fmaf(cr, v.w, a.w); a.w = fmaf(ci, v.z, a.w);
            }
          }
          reinterpret_cast<float4*>(wr + k0 + e0)[p] = a;
        }
        if (MODE != 0) {
          ss = fmaf(a.x, a.x, ss); ss = fmaf(a.y, a.y, ss);
          ss = fmaf(a.z, a.z, ss); ss = fmaf(a.w, a.w, ss);
        }
#pragma unroll
        for (int q = 0; q < NVM; ++q) {
          if (q < nv) {
            float4 v = sb[(size_t)(1 + q) * tp + p];
            ar[q] = fmaf(v.x, a.x, ar[q]); ar[q] = fmaf(v.y, a.y, ar[q]);
            ar[q] = fmaf(v.z, a.z, ar[q]); ar[q] = fmaf(v.w, a.w, ar[q]);
            ai[q] = fmaf(v.x, a.y, ai[q]); ai[q] = fmaf(-v.y, a.x, ai[q]);
            ai[q] = fmaf(v.z, a.w, ai[q]); ai[q] = fmaf(-v.w, a.z, ai[q]);
          }
        }
      }
    }
    // every thread is done with stage st (and agrees whether its copies arrived)
    if (!__syncthreads_and(ok)) {
      failed_at = it;
      break;
    }
    if (threadIdx.x == 0 && it + stages < ntiles) {
      fence_proxy_async();
      issue(it + stages);
    }
  }
  if (failed_at >= 0) {
    if (threadIdx.x == 0) {
      *(volatile int*)err = 1;
      // let the copies still in flight land before the CTA's shared memory is released
      for (int it = failed_at; it < ntiles && it < failed_at + stages; ++it)
        mbar_wait(&bars[it % stages], (uint32_t)((it / stages) & 1), ST_WAIT);
    }
    return;
  }
  cta_store_partials<float, NVM>(ar, ai, nv, 0, rhs, maxvec, nblk, partials_as<float>(partial),
                                 sh);
  if (MODE != 0) {
    float zero = 0.f;
    cta_store_partials<float, 1>(&ss, &zero, 1, nv, rhs, maxvec, nblk,
                                 partials_as<float>(partial), sh);
  }
  if (!last_cta(counter, rhs, nblk)) return;
  if (MODE == 0) {
    finish_partials(partials_as<float>(partial), nv, nblk, maxvec, rhs, out, nullptr, ldo, 0,
                    scale);
    if (threadIdx.x == 0) counter[rhs] = 0;
    return;
  }
  // projections and H[j+1, j]; the Givens step follows in the normalising update
  __shared__ zd g_h2[NVM + 1];
  finish_partials(partials_as<float>(partial), nv + 1, nblk, maxvec, rhs, g_h2, nullptr, 0, 0,
                  scale);
  __syncthreads();
  for (int i = threadIdx.x; i <= nv; i += RT) sm[L.h2() + i] = g_h2[i];
  if (threadIdx.x == 0) {
    counter[rhs] = 0;
    double hh = 0;
    for (int i = 0; i < nv; ++i) hh += norm2(g_h2[i]);
    double b2 = g_h2[nv].re - hh;
    wnorm[rhs] = b2 > 0 ? sqrt(b2) : 0.0;
  }
}

// One fixed-step GMRES step's operator and projections in one kernel (single-pass classical
// Gram-Schmidt, complex-float basis):  w = D v_j  (the FP32 Wilson-Dirac stencil, Eq. 1,
// lane-contiguous links), h_i = V_i^dag w for i < nv = j + 1, ||w||^2, and in the last CTA
// H[j+1, j]^2 = ||w||^2 - ||h||^2 as in stream_cgs_kernel<2>.  The basis reads at each
// thread's own site do not depend on the stencil, so they overlap its latency-bound hops,
// and w is not read back.  One thread per site and rhs row (blockIdx.y); BT and the register
// budget (MINB resident CTAs) are launch shapes the autotuner picks per (columns, link
// layout, volume, rhs).
template <int NVM, bool FIRST, int LL, int BT, int MINB>
__global__ void __launch_bounds__(BT, MINB)
dslash_proj_kernel(zf* w, zf* V, size_t vstride, int nv, size_t n,
                   const float2* __restrict__ links, stencil::KGeom g, zd* small, SmallLayout L,
                   double* wnorm, double* partial, unsigned* counter, int maxvec,
                   const zf* __restrict__ b0, const double* beta0, const zf* __restrict__ sin,
                   int par) {
  using namespace stencil;
  dep_entry();
  __shared__ float sh[(BT / 32) * NVM * 2];
  const int rhs = blockIdx.y;
  // par: the even-odd Schur operator's second hop, w = x - (-kappa H_eo) t_o on even
  // half-lattice fields, with t_o = -kappa H_oe x (the odd field sin) computed by the caller
  const int nsites = par ? g.V / 2 : g.V;
  float2* vb = reinterpret_cast<float2*>(V) + (size_t)rhs * n;
  // FIRST (step 0): the stencil reads b and everything is scaled by 1 / ||b|| (linear),
  // v_0 = b / ||b|| is written here (no separate scaling pass); otherwise the input is v_j
  const float2* vin = FIRST ? reinterpret_cast<const float2*>(b0) + (size_t)rhs * n
                            : vb + (size_t)(nv - 1) * vstride;
  float sc = 1.0f;
  if (FIRST) {
    double bb = beta0[rhs];
    sc = bb > 0 ? (float)(1.0 / bb) : 0.0f;
  }
  float2* wr = reinterpret_cast<float2*>(w) + (size_t)rhs * n;
  const float2* vst = par ? reinterpret_cast<const float2*>(sin) + (size_t)rhs * n : vin;
  float ar[NVM], ai[NVM];
#pragma unroll
  for (int q = 0; q < NVM; ++q) { ar[q] = 0.f; ai[q] = 0.f; }
  float ss = 0.f;
  // one site per thread (the launcher sizes the grid to cover every site): with no loop the
  // projection accumulators are not live across the stencil's hops, which need the registers
  const int site = blockIdx.x * BT + threadIdx.x;
  if (site < nsites) {
    int c[4];
    // site: the output index (lexicographic, or the checkerboard index with par); ls: the
    // lattice site the hops start from
    const int ls = stencil_site(g, par ? 0 : -1, site, c);
    zf acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {0.f, 0.f};
    hop_pair<0, 0, StC64, LL>(g, ls, c, vst, 0, par != 0, links, acc);
    hop_pair<1, 0, StC64, LL>(g, ls, c, vst, 0, par != 0, links, acc);
    hop_pair<2, 0, StC64, LL>(g, ls, c, vst, 0, par != 0, links, acc);
    hop_pair<3, 0, StC64, LL>(g, ls, c, vst, 0, par != 0, links, acc);
    zf p[12], x0[12];
    SiteIO<StC64>::load(vin, (size_t)site, x0);
    const float mk = par ? (float)g.kappa : (float)(-g.kappa);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      p[k].re = sc * fmaf(mk, acc[k].re, x0[k].re);
      p[k].im = sc * fmaf(mk, acc[k].im, x0[k].im);
      ss = fmaf(p[k].re, p[k].re, ss);
      ss = fmaf(p[k].im, p[k].im, ss);
      x0[k].re *= sc;
      x0[k].im *= sc;
    }
    SiteIO<StC64>::store(wr, (size_t)site, p);
    if (FIRST) SiteIO<StC64>::store(vb, (size_t)site, x0);   // v_0
#pragma unroll
    for (int q = 0; q < NVM; ++q) {
      if (q < nv) {
        zf v[12];
        if (FIRST) {   // nv = 1: v_0 is in registers (just written, not read back)
#pragma unroll
          for (int k = 0; k < 12; ++k) v[k] = x0[k];
        } else {
          SiteIO<StC64>::load(vb + (size_t)q * vstride, (size_t)site, v);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          ar[q] = fmaf(v[k].re, p[k].re, ar[q]);
          ar[q] = fmaf(v[k].im, p[k].im, ar[q]);
          ai[q] = fmaf(v[k].re, p[k].im, ai[q]);
          ai[q] = fmaf(-v[k].im, p[k].re, ai[q]);
        }
      }
    }
  }
  const int nblk = gridDim.x;
  cta_store_partials<float, NVM>(ar, ai, nv, 0, rhs, maxvec, nblk, partials_as<float>(partial),
                                 sh);
  float zero = 0.f;
  cta_store_partials<float, 1>(&ss, &zero, 1, nv, rhs, maxvec, nblk, partials_as<float>(partial),
                               sh);
  if (!last_cta(counter, rhs, nblk)) return;
  // projections and H[j+1, j]; the Givens step follows in the normalising update
  __shared__ zd g_h2[NVM + 1];
  finish_partials(partials_as<float>(partial), nv + 1, nblk, maxvec, rhs, g_h2, nullptr, 0, 0);
  __syncthreads();
  zd* sm = small + (size_t)rhs * L.stride();
  for (int i = threadIdx.x; i <= nv; i += BT) sm[L.h2() + i] = g_h2[i];
  if (threadIdx.x == 0) {
    counter[rhs] = 0;
    double hh = 0;
    for (int i = 0; i < nv; ++i) hh += norm2(g_h2[i]);
    double b2 = g_h2[nv].re - hh;
    wnorm[rhs] = b2 > 0 ? sqrt(b2) : 0.0;
  }
}

// launch shapes of the fused kernel: threads per CTA and resident CTAs per SM asked of the
// register allocator (register cap 64K / (BT MINB), allocated in steps of 8): 256 x 2 and
// 128 x 4 (128 registers), 128 x 5 (96), 128 x 6 (80; spills 12-64 bytes per thread).
constexpr int kProjShapes = 4;

template <int NVM, bool FIRST, int LL, int BT, int MINB>
void launch_proj_shape(int nv, int V, int nblk, int nrhs, cudaStream_t st, zf* w, zf* V_,
                       size_t fs, size_t n, const float2* L32, const stencil::KGeom& kg, zd* small,
                       SmallLayout L, double* dnorm, ReduceWork& rw, const zf* b0,
                       const double* beta0, const zf* sin, int par, cudaError_t* err) {
  const int ns = par ? V / 2 : V;
  const int nb = (ns + BT - 1) / BT;   // one site per thread; launch_proj checked nb <= nblk
  *err = launch_dep(dslash_proj_kernel<NVM, FIRST, LL, BT, MINB>, dim3(nb, nrhs), BT, 0, st, w,
                    V_, fs, nv, n, L32, kg, small, L, dnorm, rw.partial, rw.counter, rw.maxvec,
                    b0, beta0, sin, par);
}

template <int NVM, bool FIRST, int LL>
void launch_proj_v(int v, int nv, int nrhs, cudaStream_t st, zf* w, zf* V_, size_t fs, size_t n,
                   const float2* L32, const stencil::KGeom& kg, zd* small, SmallLayout L,
                   double* dnorm, ReduceWork& rw, const zf* b0, const double* beta0,
                   const zf* sin, int par, cudaError_t* err) {
  switch (v) {
    case 1: launch_proj_shape<NVM, FIRST, LL, 128, 4>(nv, kg.V, rw.cap, nrhs, st, w, V_, fs, n, L32, kg, small, L, dnorm, rw, b0, beta0, sin, par, err); break;
    case 2: launch_proj_shape<NVM, FIRST, LL, 128, 5>(nv, kg.V, rw.cap, nrhs, st, w, V_, fs, n, L32, kg, small, L, dnorm, rw, b0, beta0, sin, par, err); break;
    case 3: launch_proj_shape<NVM, FIRST, LL, 128, 6>(nv, kg.V, rw.cap, nrhs, st, w, V_, fs, n, L32, kg, small, L, dnorm, rw, b0, beta0, sin, par, err); break;
    default: launch_proj_shape<NVM, FIRST, LL, 256, 2>(nv, kg.V, rw.cap, nrhs, st, w, V_, fs, n, L32, kg, small, L, dnorm, rw, b0, beta0, sin, par, err); break;
  }
}

template <int LL>
int launch_proj(int nv, bool first, int nrhs, cudaStream_t st, zf* w, zf* V, size_t fs,
                size_t n, const float2* L32, const stencil::KGeom& kg, zd* small, SmallLayout L,
                double* dnorm, ReduceWork& rw, const zf* b0, const double* beta0, const zf* sin,
                int par) {
  const int nvm = first ? 0 : nv <= 4 ? 4 : nv <= 8 ? 8 : 16;
  // every shape takes one site per thread, so its grid (at least 128 threads per CTA) must
  // fit the partial slots of the reduction workspace
  const int ns = par ? kg.V / 2 : kg.V;
  if ((ns + 127) / 128 > rw.cap)
    return fail(MG_EINVAL, "dslash_proj: reduction workspace holds too few CTA partials");
  cudaError_t err = cudaSuccess;
  auto run = [&](int v) {
    if (first) launch_proj_v<4, true, LL>(v, nv, nrhs, st, w, V, fs, n, L32, kg, small, L, dnorm, rw, b0, beta0, sin, par, &err);
    else if (nvm == 4) launch_proj_v<4, false, LL>(v, nv, nrhs, st, w, V, fs, n, L32, kg, small, L, dnorm, rw, b0, beta0, sin, par, &err);
    else if (nvm == 8) launch_proj_v<8, false, LL>(v, nv, nrhs, st, w, V, fs, n, L32, kg, small, L, dnorm, rw, b0, beta0, sin, par, &err);
    else launch_proj_v<16, false, LL>(v, nv, nrhs, st, w, V, fs, n, L32, kg, small, L, dnorm, rw, b0, beta0, sin, par, &err);
  };
  // tuning key: a dtype code of its own per (columns class, link layout), parity -2; the
  // kernel is idempotent (it rewrites w, its partials and its Hessenberg column from inputs
  // it does not modify), so the tuner may run it several times
  int v = tuned_variant(1000 + 100 * par + 10 * nvm + LL, -2, 0, kg.V, nrhs, st, kProjShapes, run);
  if (v < 0) return fail(MG_ECUDA, "fused stencil autotune failed");
  run(v);
  count_launch();
  if (err != cudaSuccess)
    return fail(MG_ECUDA, std::string("dslash_proj launch: ") + cudaGetErrorString(err));
  return MG_OK;
}

int dslash_proj_launch(zf* w, zf* V, size_t fs, size_t n, int nrhs, zd* small,
                       SmallLayout L, int j, double* dnorm, ReduceWork& rw,
                       const FusedStencil& fz, cudaStream_t st, const zf* b0 = nullptr,
                       const double* beta0 = nullptr) {
  stencil::KGeom kg = stencil::to_kgeom(fz.g);
  int nv = j + 1;
  const float2* L32 = static_cast<const float2*>(fz.links);
  const zf* sin = nullptr;
  const int par = fz.schur ? 1 : 0;
  if (par) {
    // first hop of the Schur operator, t_o = -kappa H_oe x, x = b (first step) or v_j
    sin = static_cast<const zf*>(fz.odd);
    const zf* x = b0 ? b0 : V + (size_t)j * fs;
    WMG_TRY(dslash_launch(MG_C64, fz.odd, x, fz.links, fz.g, 1, 0, nrhs, st, n, n, fz.layout));
  }
  // algorithmic bytes: per right-hand side the nv basis columns read (v_j, the stencil input,
  // is one of them) and w written -- the first step reads b and writes v_0 and w instead --
  // and the 36 complex link entries of a site once per launch; the Schur form's second hop
  // reads t_o besides and all 8 links of each even output site
  const double fields = (b0 ? 3.0 : (double)(nv + 1)) + par;
  const double nout = par ? kg.V / 2 : kg.V;
  double byts = nout * 8.0 * (12.0 * fields * nrhs + (par ? 72.0 : 36.0));
  ProfScope ps(par ? "schur_proj" : "dslash_proj", byts,
               (1320.0 + 48.0 * (nv + 1)) * nout * nrhs, st);
  if (fz.layout == 2) return launch_proj<2>(nv, b0 != nullptr, nrhs, st, w, V, fs, n, L32, kg, small, L, dnorm, rw, b0, beta0, sin, par);
  return launch_proj<1>(nv, b0 != nullptr, nrhs, st, w, V, fs, n, L32, kg, small, L, dnorm, rw, b0, beta0, sin, par);
}

template <int NVM>
int stream_cgs_launch(zf* w, const zf* V, size_t fs, size_t n, int nrhs, zd* small,
                      SmallLayout L, int j, double* dnorm, double* reshist, ReduceWork& rw,
                      double scale, int* err, bool cgs1, cudaStream_t st) {
  {
    size_t mx = st_smem(NVM);
    WMG_TRY(smem_attr(stream_cgs_kernel<0, NVM>, mx));
    WMG_TRY(smem_attr(stream_cgs_kernel<1, NVM>, mx));
    WMG_TRY(smem_attr(stream_cgs_kernel<2, NVM>, mx));
  }
  int nv = j + 1;
  int per_sm = NVM <= 8 ? 2 : 1;
  int nb = rw.nblk < per_sm * num_sms() ? rw.nblk : per_sm * num_sms();
  size_t sh = st_smem(nv);
  double fb = (double)nrhs * n * sizeof(zf);
  zd* Hcol = small + L.H() + (size_t)j * (L.m + 1);
  if (cgs1) {
    ProfScope ps("cgs1_dot_norm", (nv + 1) * fb, (8.0 * nv + 4.0) * n * nrhs, st);
    WMG_LAUNCH_DEP(stream_cgs_kernel<2, NVM>, dim3(nb, nrhs), RT, sh, st, w, V, fs, nv, n, nullptr, 0, small, L, j, dnorm, reshist, rw.partial, rw.counter, nb, rw.maxvec, scale, err);
    return MG_OK;
  }
  {
    ProfScope ps("multi_dot", (nv + 1) * fb, 8.0 * nv * n * nrhs, st);
    WMG_LAUNCH_DEP(stream_cgs_kernel<0, NVM>, dim3(nb, nrhs), RT, sh, st, w, V, fs, nv, n, Hcol, L.stride(), small, L, j, dnorm, reshist, rw.partial, rw.counter, nb, rw.maxvec, scale, err);
  }
  {
    ProfScope ps("cgs_update_dot", (nv + 2) * fb, (16.0 * nv + 4.0) * n * nrhs, st);
    WMG_LAUNCH_DEP(stream_cgs_kernel<1, NVM>, dim3(nb, nrhs), RT, sh, st, w, V, fs, nv, n, nullptr, 0, small, L, j, dnorm, reshist, rw.partial, rw.counter, nb, rw.maxvec, scale, err);
  }
  return MG_OK;
}

// Both CGS reduction sweeps of Arnoldi step j through the bulk-copy kernels (complex float,
// j + 1 <= ST_NV basis columns).
int stream_cgs(zf* w, const zf* V, size_t fs, size_t n, int nrhs, zd* small, SmallLayout L,
               int j, double* dnorm, double* reshist, ReduceWork& rw, double scale, bool cgs1,
               cudaStream_t st) {
  int* err = device_error_word();
  if (!err) return fail(MG_ECUDA, "stream_cgs: no error word");
  if (j + 1 <= 8)
    return stream_cgs_launch<8>(w, V, fs, n, nrhs, small, L, j, dnorm, reshist, rw, scale, err,
                                cgs1, st);
  return stream_cgs_launch<16>(w, V, fs, n, nrhs, small, L, j, dnorm, reshist, rw, scale, err,
                               cgs1, st);
}

// CTAs per (rhs) row of a reduction launch: one wave of `kernel` at its occupancy, capped by
// the partial buffer's chunk count.
template <typename K>
int reduction_blocks(K kernel, int cap) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, RT, 0) != cudaSuccess || occ < 1)
    occ = 1;
  int b = occ * num_sms();
  return b < cap ? b : cap;
}

// Back substitution R y = g over the first `steps` columns.
__global__ void solve_kernel(zd* small, SmallLayout L, int steps, int nrhs) {
  dep_entry();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  zd* s = small + (size_t)r * L.stride();
  const zd* H = s + L.H();
  const zd* g = s + L.g();
  zd* y = s + L.y();
  for (int i = steps - 1; i >= 0; --i) {
    zd acc = g[i];
    for (int k = i + 1; k < steps; ++k) acc = acc - H[(size_t)k * (L.m + 1) + i] * y[k];
    zd d = H[(size_t)i * (L.m + 1) + i];
    double dd = norm2(d);
    y[i] = dd > 0 ? (1.0 / dd) * cmulc(d, acc) : zd{0, 0};
  }
}

}  // namespace

template <typename E>
int GmresV<E>::alloc(size_t n_, int nrhs_, int m_, bool flexible_) {
  if (n == n_ && nrhs >= nrhs_ && m >= m_ && (flexible || !flexible_)) return MG_OK;
  release();
  n = n_;
  nrhs = nrhs_;
  m = m_;
  flexible = flexible_;
  size_t fb = sizeof(E) * n * nrhs;
  WMG_TRY(dev_alloc(&V, fb * (m + 1)));
  if (flexible) WMG_TRY(dev_alloc(&Z, fb * m));
  WMG_TRY(dev_alloc(&w, fb));
  SmallLayout L{m};
  WMG_TRY(dev_alloc(&small, sizeof(zd) * L.stride() * nrhs));
  WMG_TRY(dev_alloc(&dnorm, sizeof(double) * nrhs * 4));
  WMG_TRY(dev_alloc(&reshist, sizeof(double) * nrhs * m));
  WMG_TRY(host_alloc(&host_res, sizeof(double) * nrhs * (m + 2)));
  WMG_TRY(rw.alloc(n, nrhs, m + 1));
  return MG_OK;
}

template <typename E>
void GmresV<E>::release() {
  dev_free(V);
  dev_free(Z);
  dev_free(w);
  dev_free(small);
  dev_free(dnorm);
  dev_free(reshist);
  host_free(host_res);
  V = Z = w = nullptr;
  small = nullptr;
  dnorm = nullptr;
  reshist = nullptr;
  host_res = nullptr;
  rw.release();
  n = 0;
  nrhs = 0;
  m = 0;
}

// dnorm layout: [0..nrhs) current ||w||, [nrhs..2nrhs) beta, [2nrhs..3nrhs) residual estimate
template <typename E>
int GmresV<E>::arnoldi_step(const OpV<E>& A, const OpV<E>* M, int j, cudaStream_t st,
                            bool single_pass, const FusedStencil* fused, const E* b0,
                            bool next) {
  SmallLayout L{m};
  size_t fs = n * nrhs;
  E* vj = V + (size_t)j * fs;
  bool fuse = false;
  if constexpr (std::is_same<E, zf>::value)
    fuse = fused && single_pass && !M && j + 1 <= ST_NV &&
           n == (size_t)(fused->schur ? fused->g.V / 2 : fused->g.V) * 12;
  if (fuse) {
    // the stencil and the single-pass projections in one kernel
    if constexpr (std::is_same<E, zf>::value)
      WMG_TRY(dslash_proj_launch(w, V, fs, n, nrhs, small, L, j, dnorm, rw, *fused, st, b0,
                                 b0 ? dnorm + nrhs : nullptr));
  } else if (M) {
    E* zj = Z + (size_t)j * fs;
    WMG_TRY((*M)(zj, vj, st));
    WMG_TRY(A(w, zj, st));
  } else {
    WMG_TRY(A(w, vj, st));
  }
  zd* Hcol = small + L.H() + (size_t)j * (m + 1);
  // CGS2 in three sweeps: projections; update + re-projections + norm; update +
  // normalisation into column j + 1, with the Givens step beside it
  double fb = (double)nrhs * n * sizeof(E);
  bool streamed = fuse;
  if constexpr (std::is_same<E, zf>::value) {
    if (!fuse && j + 1 <= ST_NV && (n & 1) == 0) {
      WMG_TRY(stream_cgs(w, V, fs, n, nrhs, small, L, j, dnorm, reshist, rw, ip_scale(),
                         single_pass, st));
      streamed = true;
    }
  }
  if (!streamed) {
    WMG_TRY(multi_dot_v<E>(Hcol, L.stride(), V, fs, j + 1, w, n, nrhs, rw, st, ip_scale()));
    static const int ud_blocks = reduction_blocks(cgs_update_dot_kernel<E>, 1 << 30);
    int nb = ud_blocks < rw.nblk ? ud_blocks : rw.nblk;
    ProfScope ps("cgs_update_dot", (j + 3) * fb, (16.0 * (j + 1) + 4.0) * n * nrhs, st);
    WMG_LAUNCH_DEP(cgs_update_dot_kernel<E>, dim3(nb, nrhs), RT, 0, st, w, V, fs, j + 1, small, L, j, n, dnorm, reshist, rw.partial, rw.counter, nb, rw.maxvec, ip_scale());
  }
  if (!next) {
    // the Givens step of column j alone (the last CTA of the update kernel)
    ProfScope ps("cgs_givens", 0.0, 0.0, st);
    WMG_LAUNCH_DEP(cgs_update_scale_kernel<E>, dim3(1, nrhs), 256, 0, st,
                   V + (size_t)(j + 1) * fs, w, V, fs, j + 1, small, L, dnorm, n, reshist,
                   single_pass && streamed ? 1 : 0);
    return MG_OK;
  }
  {
  ProfScope ps("cgs_update_scale", (j + 3) * fb, (8.0 * (j + 1) + 2.0) * n * nrhs, st);
  size_t g = (n / 2 + 255) / 256;
  size_t cap = (size_t)num_sms() * 8;
  // + 1 CTA per rhs row for the deferred Givens step
  dim3 grid((unsigned)(g < cap ? (g < 1 ? 1 : g) : cap) + 1, nrhs);
  WMG_LAUNCH_DEP(cgs_update_scale_kernel<E>, grid, 256, 0, st, V + (size_t)(j + 1) * fs, w, V, fs, j + 1, small, L, dnorm, n, reshist, single_pass && streamed ? 1 : 0);
  }
  return MG_OK;
}

template <typename E>
int GmresV<E>::fixed(const OpV<E>& A, E* x, const E* b, int steps, cudaStream_t st,
                     bool accumulate, const FusedStencil* fused, double xsign) {
  if (steps > m) return fail(MG_EINVAL, "gmres: more steps than allocated");
  SmallLayout L{m};
  size_t fs = n * nrhs;
  if (!accumulate) WMG_TRY(fill_zero_v<E>(x, fs, st));
  if (steps == 0) return MG_OK;
  WMG_TRY(norm2_v<E>(dnorm + nrhs, 1, b, n, nrhs, rw, st, ip_scale()));
  WMG_LAUNCH_DEP(init_kernel, (nrhs + 31) / 32, 32, 0, st, small, L, dnorm + nrhs, dnorm + 2 * nrhs, nrhs);
  // the fused first step scales b itself and writes v_0 (see dslash_proj_kernel)
  bool fuse0 = false;
  if constexpr (std::is_same<E, zf>::value)
    fuse0 = fused && n == (size_t)(fused->schur ? fused->g.V / 2 : fused->g.V) * 12;
  if (!fuse0) WMG_TRY(scale_inv_v<E>(V, b, dnorm + nrhs, 1, n, nrhs, st));
  // A fixed number of steps from zero (the smoothers): complex-float bases of up to 16
  // columns orthogonalise with a single classical Gram-Schmidt pass, H[j+1, j] from
  // Pythagoras.  Over these few steps the basis stays orthogonal to ~eps_32 times the
  // conditioning of the small Krylov basis, which leaves the smoother's approximate
  // minimisation unchanged to FP32 rounding; the tolerance-driven solves keep CGS2.
  // the last step needs its Hessenberg column and Givens step, not the next basis column
  for (int j = 0; j < steps; ++j)
    WMG_TRY(arnoldi_step(A, nullptr, j, st, true, fused, fuse0 && j == 0 ? b : nullptr,
                         j + 1 < steps));
  WMG_LAUNCH_DEP(solve_kernel, (nrhs + 31) / 32, 32, 0, st, small, L, steps, nrhs);
  WMG_TRY(multi_axpy_v<E>(x, V, fs, steps, small + L.y(), L.stride(), xsign, n, nrhs, st));
  return MG_OK;
}

template <typename E>
int GmresV<E>::solve(const OpV<E>& A, const OpV<E>* M, E* x, const E* b, double rtol,
                     int restart, int maxiter, int* its_out, cudaStream_t st, int check_every) {
  if (restart > m) return fail(MG_EINVAL, "gmres: restart longer than allocated");
  if (M && !flexible) return fail(MG_EINVAL, "gmres: flexible space not allocated");
  SmallLayout L{m};
  size_t fs = n * nrhs;
  WMG_TRY(fill_zero_v<E>(x, fs, st));
  // bnorm on host
  std::vector<double> bn(nrhs), res(nrhs);
  WMG_TRY(norm2_v<E>(dnorm + nrhs, 1, b, n, nrhs, rw, st, ip_scale()));
  WMG_CUDA(cudaMemcpyAsync(host_res, dnorm + nrhs, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  WMG_CUDA(cudaStreamSynchronize(st));
  for (int r = 0; r < nrhs; ++r) bn[r] = host_res[r];
  // r = b (x0 = 0); the residual lives in w between cycles
  E* rvec = w;
  WMG_CUDA(cudaMemcpyAsync(rvec, b, sizeof(E) * fs, cudaMemcpyDeviceToDevice, st));
  int its = 0;
  bool converged = false;
  for (int r = 0; r < nrhs; ++r) res[r] = bn[r];
  auto all_done = [&](const double* rr) {
    for (int r = 0; r < nrhs; ++r)
      if (!(rr[r] <= rtol * bn[r])) return false;
    return true;
  };
  if (all_done(res.data())) converged = true;
  bool first = true;
  while (!converged && its < maxiter) {
    // the first cycle's residual is b itself, whose norms are already in dnorm + nrhs
    if (!first) WMG_TRY(norm2_v<E>(dnorm + nrhs, 1, rvec, n, nrhs, rw, st, ip_scale()));
    first = false;
    WMG_LAUNCH_DEP(init_kernel, (nrhs + 31) / 32, 32, 0, st, small, L, dnorm + nrhs, dnorm + 2 * nrhs, nrhs);
    WMG_TRY(scale_inv_v<E>(V, rvec, dnorm + nrhs, 1, n, nrhs, st));
    int steps = 0, checked = 0;
    if (check_every < 1) check_every = 1;
    for (int j = 0; j < restart && its < maxiter; ++j) {
      WMG_TRY(arnoldi_step(A, M, j, st));
      ++steps;
      ++its;
      bool check = ((j + 1 - checked) >= check_every) || j + 1 == restart || its >= maxiter;
      if (!check) continue;
      WMG_CUDA(cudaMemcpyAsync(host_res, reshist + (size_t)checked * nrhs,
                               sizeof(double) * nrhs * (j + 1 - checked), cudaMemcpyDeviceToHost,
                               st));
      WMG_CUDA(cudaStreamSynchronize(st));
      if (take_device_error()) return fail(MG_ETIMEOUT, "gmres: a bounded wait gave up");
      bool stop = false;
      for (int jj = checked; jj <= j && !stop; ++jj) {
        const double* rr = host_res + (size_t)(jj - checked) * nrhs;
        for (int r = 0; r < nrhs; ++r)
          if (!std::isfinite(rr[r])) return fail(MG_ENAN, "gmres: non-finite residual");
        if (all_done(rr)) {
          its -= j - jj;     // steps past convergence are discarded
          steps = jj + 1;
          stop = true;
        }
      }
      checked = j + 1;
      if (stop) break;
    }
    WMG_LAUNCH_DEP(solve_kernel, (nrhs + 31) / 32, 32, 0, st, small, L, steps, nrhs);
    WMG_TRY(multi_axpy_v<E>(x, M ? Z : V, fs, steps, small + L.y(), L.stride(), 1.0, n, nrhs, st));
    // true residual r = b - A x
    WMG_TRY(A(rvec, x, st));
    WMG_TRY(axpby_v<E>(rvec, 1.0, b, -1.0, fs, 1, st));
    WMG_TRY(norm2_v<E>(dnorm + 3 * nrhs, 1, rvec, n, nrhs, rw, st, ip_scale()));
    WMG_CUDA(cudaMemcpyAsync(host_res + nrhs, dnorm + 3 * nrhs, sizeof(double) * nrhs,
                             cudaMemcpyDeviceToHost, st));
    WMG_CUDA(cudaStreamSynchronize(st));
    if (take_device_error()) return fail(MG_ETIMEOUT, "gmres: a bounded wait gave up");
    if (all_done(host_res + nrhs)) converged = true;
  }
  if (its_out) *its_out = its;
  if (!converged) return fail(MG_ENOCONV, "gmres: no convergence within maxiter");
  return MG_OK;
}

template class GmresV<zf>;
template class GmresV<zd>;
template class GmresV<zh>;
template class GmresV<zbf>;

}  // namespace wmg
