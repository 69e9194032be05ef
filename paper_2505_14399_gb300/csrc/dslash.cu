// Wilson-Dirac stencil (the operator D of Eq. 1), full and single-parity, any storage.
//
// One thread per output site and right-hand side.  Each of the 8 hops loads the
// neighbour spinor, projects it to a 2-spin half spinor with (1 -/+ gamma_mu) in the
// chiral basis, multiplies by U_mu(x) or U_mu(x-mu)^dag, and reconstructs the lower
// spin pair from the upper one.  Spinor loads are 16-byte vector loads of the
// [site][spin][colour] layout; links are read through the read-only path.
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "stencil.cuh"
#include "vec.cuh"

namespace wmg {
namespace {

using namespace stencil;

// parity < 0: out = in - kappa H in (full lattice).  parity p >= 0: out_p = -kappa H in_{1-p}
// on half-lattice (checkerboard-indexed) fields.
template <typename S, int DAG, int TPB, int MINB, int LL>
__global__ void __launch_bounds__(TPB, MINB)
dslash_kernel(typename S::elem* __restrict__ out, const typename S::elem* __restrict__ in,
              const typename S::elem* __restrict__ links, KGeom g, int parity, int nsites,
              size_t in_stride, size_t out_stride) {
  dep_entry();
  typedef typename S::real R;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsites) return;
  size_t rhs = blockIdx.y;
  int site;
  if (parity < 0) {
    site = i;
  } else {
    int s0 = 2 * i;
    int x0 = s0 % g.L[0];
    int rest = s0 / g.L[0];
    int y = rest % g.L[1];
    int z = (rest / g.L[1]) % g.L[2];
    int t = rest / (g.L[1] * g.L[2]);
    site = s0 + (((x0 + y + z + t) & 1) != parity ? 1 : 0);
  }
  int c[4];
  c[0] = site % g.L[0];
  int rest = site / g.L[0];
  c[1] = rest % g.L[1];
  rest /= g.L[1];
  c[2] = rest % g.L[2];
  c[3] = rest / g.L[2];
  cplx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {0, 0};
  bool half_in = parity >= 0;
  size_t in_off = rhs * in_stride;
  hop_pair<0, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
  hop_pair<1, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
  hop_pair<2, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
  hop_pair<3, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
  R mk = (R)(-g.kappa);
  cplx<R> res[12];
  if (parity < 0) {
    cplx<R> p[12];
    SiteIO<S>::load(in + in_off, (size_t)site, p);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      res[k].re = fma(mk, acc[k].re, p[k].re);
      res[k].im = fma(mk, acc[k].im, p[k].im);
    }
    SiteIO<S>::store(out + rhs * out_stride, (size_t)site, res);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) res[k] = mk * acc[k];
    apply_sub<S>(g, rhs * out_stride, i, res);
    SiteIO<S>::store(out + rhs * out_stride, (size_t)i, res);
  }
}

// Two threads per site, warp-uniform: the first 64 threads of a CTA take the forward hops
// of 64 sites, the other 64 the backward hops of the same sites; the halves meet in shared
// memory.  Twice the threads with half the dependent work each, for lattices too small to
// fill the GPU with one thread per site.
template <typename S, int DAG, int LL>
__global__ void __launch_bounds__(128)
dslash_split_kernel(typename S::elem* __restrict__ out, const typename S::elem* __restrict__ in,
                    const typename S::elem* __restrict__ links, KGeom g, int parity, int nsites,
                    size_t in_stride, size_t out_stride) {
  dep_entry();
  typedef typename S::real R;
  __shared__ cplx<R> sacc[12][64];
  const int half = threadIdx.x >> 6, ls = threadIdx.x & 63;
  const int i = blockIdx.x * 64 + ls;
  const bool active = i < nsites;
  const size_t rhs = blockIdx.y;
  const bool half_in = parity >= 0;
  const size_t in_off = rhs * in_stride;
  cplx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {0, 0};
  int site = 0;
  int c[4] = {0, 0, 0, 0};
  if (active) {
    site = stencil_site(g, parity, i, c);
    if (half == 0) {
      hop_fwd<0, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
      hop_fwd<1, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
      hop_fwd<2, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
      hop_fwd<3, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
    } else {
      hop_bwd<0, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
      hop_bwd<1, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
      hop_bwd<2, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
      hop_bwd<3, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
    }
  }
  if (half == 1) {
#pragma unroll
    for (int k = 0; k < 12; ++k) sacc[k][ls] = acc[k];
  }
  __syncthreads();
  if (half != 0 || !active) return;
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] += sacc[k][ls];
  R mk = (R)(-g.kappa);
  cplx<R> res[12];
  if (parity < 0) {
    cplx<R> p[12];
    SiteIO<S>::load(in + in_off, (size_t)site, p);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      res[k].re = fma(mk, acc[k].re, p[k].re);
      res[k].im = fma(mk, acc[k].im, p[k].im);
    }
    SiteIO<S>::store(out + rhs * out_stride, (size_t)site, res);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) res[k] = mk * acc[k];
    apply_sub<S>(g, rhs * out_stride, i, res);
    SiteIO<S>::store(out + rhs * out_stride, (size_t)i, res);
  }
}

// Launch shapes: threads per CTA and the minimum resident CTAs per SM requested from
// the register allocator (register cap = 64K / (TPB * MINB)).  The autotuner below
// picks one per (dtype, parity, dagger, volume, nrhs).
struct Shape {
  int tpb, minb;
};
constexpr Shape kShapes[] = {{128, 1}, {128, 6}, {128, 8}, {256, 4}, {64, 16}, {128, 0},
                             {128, 0}, {128, 0}};
// entry 5 is the two-threads-per-site kernel (dslash_split_kernel); entries 6 and 7 take
// 2 and 4 right-hand sides per thread (dslash_mrhs_kernel), candidates only when nrhs > 1
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);
constexpr int kNumSingle = 6;

template <typename S, int DAG, int TPB, int MINB, int LL>
void launch_shape(void* out, const void* in, const void* links, const KGeom& k, int parity,
                  int nsites, int nrhs, cudaStream_t st, size_t in_stride, size_t out_stride) {
  typedef typename S::elem E;
  dim3 grid((nsites + TPB - 1) / TPB, nrhs);
  launch_dep(dslash_kernel<S, DAG, TPB, MINB, LL>, grid, TPB, 0, st, (E*)out, (const E*)in, (const E*)links, k, parity, nsites, in_stride, out_stride);
}

template <typename S, int DAG, int LL>
void launch_variant(int v, void* out, const void* in, const void* links, const KGeom& k,
                    int parity, int nsites, int nrhs, cudaStream_t st, size_t is, size_t os) {
  switch (v) {
    case 1: launch_shape<S, DAG, 128, 6, LL>(out, in, links, k, parity, nsites, nrhs, st, is, os); break;
    case 2: launch_shape<S, DAG, 128, 8, LL>(out, in, links, k, parity, nsites, nrhs, st, is, os); break;
    case 3: launch_shape<S, DAG, 256, 4, LL>(out, in, links, k, parity, nsites, nrhs, st, is, os); break;
    case 4: launch_shape<S, DAG, 64, 16, LL>(out, in, links, k, parity, nsites, nrhs, st, is, os); break;
    case 5: {
      typedef typename S::elem E;
      dim3 grid((nsites + 63) / 64, nrhs);
      launch_dep(dslash_split_kernel<S, DAG, LL>, grid, 128, 0, st, (E*)out, (const E*)in,
                 (const E*)links, k, parity, nsites, is, os);
      break;
    }
    case 6: launch_dslash_mrhs<S>(2, DAG, LL, out, in, links, k, parity, nsites, nrhs, st, is, os); break;
    case 7: launch_dslash_mrhs<S>(4, DAG, LL, out, in, links, k, parity, nsites, nrhs, st, is, os); break;
    default: launch_shape<S, DAG, 128, 1, LL>(out, in, links, k, parity, nsites, nrhs, st, is, os); break;
  }
}

template <typename S>
int launch_typed(void* out, const void* in, const void* links, const Geom& g, int parity,
                 int dagger, int nrhs, cudaStream_t st, size_t in_stride, size_t out_stride,
                 int dtype, int layout, const void* subf) {
  KGeom k = to_kgeom(g);
  k.sub = parity >= 0 ? subf : nullptr;
  int nsites = parity < 0 ? g.V : g.V / 2;
  auto run = [&](int v) {
    if (layout == 0) {
      if (dagger) launch_variant<S, 1, 0>(v, out, in, links, k, parity, nsites, nrhs, st, in_stride, out_stride);
      else launch_variant<S, 0, 0>(v, out, in, links, k, parity, nsites, nrhs, st, in_stride, out_stride);
    } else if (layout == 1) {
      if (dagger) launch_variant<S, 1, 1>(v, out, in, links, k, parity, nsites, nrhs, st, in_stride, out_stride);
      else launch_variant<S, 0, 1>(v, out, in, links, k, parity, nsites, nrhs, st, in_stride, out_stride);
    } else if constexpr (!std::is_same<S, StC128>::value) {
      // two stored rows (FP32 and half storage only: the FP64 stencil is bound by its FMA
      // rate, where rebuilding the third row would cost more than the bytes it saves)
      if (dagger) launch_variant<S, 1, 2>(v, out, in, links, k, parity, nsites, nrhs, st, in_stride, out_stride);
      else launch_variant<S, 0, 2>(v, out, in, links, k, parity, nsites, nrhs, st, in_stride, out_stride);
    }
  };
  if (layout == 2 && std::is_same<S, StC128>::value)
    return fail(MG_EINVAL, "dslash: two-row links are not used with complex double fields");
  int v = tuned_variant(dtype + 16 * layout, parity, dagger, g.V, nrhs, st,
                        nrhs > 1 ? kNumShapes : kNumSingle, run);
  if (v < 0) return fail(MG_ECUDA, "dslash autotune failed");
  // algorithmic bytes: in + out spinors per rhs and each link once (parity: all 4V links),
  // 18 reals per link whatever the stored form
  double real_bytes = (double)sizeof(typename S::real) * (sizeof(typename S::elem) == 4 ? 0.5 : 1.0);
  double per_site = parity < 0 ? 48.0 * nrhs + 72.0 : 48.0 * nrhs + 144.0;
  ProfScope ps(dtype == MG_C128 ? "dslash_c128" : dtype == MG_C64 ? "dslash_c64"
               : dtype == MG_F16 ? "dslash_f16" : "dslash_bf16",
               per_site * real_bytes * nsites, 1320.0 * nsites * nrhs, st);
  run(v);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename E>
__global__ void link_to_lanes_kernel(E* dst, const zd* __restrict__ src, int V, int ne) {
  typedef typename VecT<E>::R R;
  size_t total = (size_t)4 * V * ne;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    // e enumerates the destination [mu][entry][site], entries 0 .. ne - 1 (row-major)
    size_t site = e % V, rest = e / V;
    int entry = (int)(rest % ne), mu = (int)(rest / ne);
    zd v = src[((size_t)mu * V + site) * 9 + entry];
    VecT<E>::st(dst, e, cplx<R>{(R)v.re, (R)v.im});
  }
}

}  // namespace

template <typename E>
int link_to_lanes_v(E* dst, const zd* src, int V, cudaStream_t st, int rows) {
  size_t total = (size_t)4 * V * 3 * rows;
  size_t g = (total + 255) / 256, cap = (size_t)num_sms() * 16;
  link_to_lanes_kernel<E><<<(unsigned)(g < cap ? g : cap), 256, 0, st>>>(dst, src, V, 3 * rows);
  WMG_LAUNCHED();
  return MG_OK;
}
template int link_to_lanes_v<zd>(zd*, const zd*, int, cudaStream_t, int);
template int link_to_lanes_v<zf>(zf*, const zd*, int, cudaStream_t, int);
template int link_to_lanes_v<zh>(zh*, const zd*, int, cudaStream_t, int);
template int link_to_lanes_v<zbf>(zbf*, const zd*, int, cudaStream_t, int);

namespace {
// Largest deviation of any link from SU(3): max over links of max(|U U^dag - 1|_max,
// |det U - 1|), as the bits of a non-negative double (ordered like the values) in *out.
__global__ void su3_deviation_kernel(unsigned long long* out, const zd* __restrict__ L, size_t n) {
  double worst = 0;
  for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (size_t)gridDim.x * blockDim.x) {
    zd u[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) u[i] = L[l * 9 + i];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        zd s = {0, 0};
#pragma unroll
        for (int c = 0; c < 3; ++c) s = s + u[a * 3 + c] * conj(u[b * 3 + c]);
        if (a == b) s.re -= 1.0;
        worst = fmax(worst, fmax(fabs(s.re), fabs(s.im)));
      }
    zd det = u[0] * (u[4] * u[8] - u[5] * u[7]) - u[1] * (u[3] * u[8] - u[5] * u[6]) +
             u[2] * (u[3] * u[7] - u[4] * u[6]);
    det.re -= 1.0;
    worst = fmax(worst, sqrt(det.re * det.re + det.im * det.im));
  }
  if (!(worst == worst)) worst = 1e300;   // NaN: not SU(3)
  // warp, then CTA maximum: one atomic per CTA (a single address taking one atomic per
  // thread serialises them)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  __shared__ double wmax[32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = wmax[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wmax[w]);
    atomicMax(out, (unsigned long long)__double_as_longlong(m));
  }
}
}  // namespace

// The same on a double-float copy of the links, in double-float arithmetic on the FP32 units
// (error-free products and sums, ~2^-48 relative: deviations are resolved far below 1e-9).
__global__ void su3_deviation_df_kernel(unsigned long long* out, const zdf* __restrict__ L,
                                        size_t n) {
  float worst = 0.f;
  for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
       l += (size_t)gridDim.x * blockDim.x) {
    zdf u[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) u[i] = L[l * 9 + i];
    // U U^dag - 1: the six entries a <= b of the Hermitian matrix
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) {
        zdfacc s{};
#pragma unroll
        for (int c = 0; c < 3; ++c) zdf_fmac(s, u[b * 3 + c], u[a * 3 + c]);   // u_ac conj(u_bc)
        zdf v = zdf_norm(s);
        if (a == b) v.re = df_add(v.re, {-1.0f, 0.0f});
        worst = fmaxf(worst, fmaxf(fabsf(v.re.hi), fabsf(v.im.hi)));
      }
    // det U - 1 by cofactors of the first row
    zdfacc t{};
    zdf_fma(t, u[4], u[8]);
    zdf_fma(t, zdf_neg(u[5]), u[7]);
    const zdf c0 = zdf_norm(t);
    t = zdfacc{};
    zdf_fma(t, u[3], u[8]);
    zdf_fma(t, zdf_neg(u[5]), u[6]);
    const zdf c1 = zdf_norm(t);
    t = zdfacc{};
    zdf_fma(t, u[3], u[7]);
    zdf_fma(t, zdf_neg(u[4]), u[6]);
    const zdf c2 = zdf_norm(t);
    t = zdfacc{};
    zdf_fma(t, u[0], c0);
    zdf_fma(t, zdf_neg(u[1]), c1);
    zdf_fma(t, u[2], c2);
    zdf det = zdf_norm(t);
    det.re = df_add(det.re, {-1.0f, 0.0f});
    worst = fmaxf(worst, sqrtf(det.re.hi * det.re.hi + det.im.hi * det.im.hi));
  }
  if (!(worst == worst)) worst = 3e38f;   // NaN: not SU(3)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  __shared__ float wmax[32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = wmax[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmax[w]);
    atomicMax(out, (unsigned long long)__double_as_longlong((double)m));
  }
}

int su3_deviation(double* dev_out, const zd* links, size_t nlinks, cudaStream_t st) {
  unsigned long long* d = nullptr;
  WMG_CUDA(cudaMallocAsync(&d, sizeof(*d), st));
  WMG_CUDA(cudaMemsetAsync(d, 0, sizeof(*d), st));
  size_t g = (nlinks + 255) / 256, cap = (size_t)num_sms() * 8;
  su3_deviation_kernel<<<(unsigned)(g < cap ? (g < 1 ? 1 : g) : cap), 256, 0, st>>>(d, links, nlinks);
  WMG_LAUNCHED();
  unsigned long long bits = 0;
  WMG_CUDA(cudaMemcpyAsync(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost, st));
  WMG_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(d, st);
  std::memcpy(dev_out, &bits, sizeof(double));
  return MG_OK;
}

int su3_deviation_df(double* dev_out, const zdf* links, size_t nlinks, cudaStream_t st) {
  unsigned long long* d = nullptr;
  WMG_CUDA(cudaMallocAsync(&d, sizeof(*d), st));
  WMG_CUDA(cudaMemsetAsync(d, 0, sizeof(*d), st));
  size_t g = (nlinks + 255) / 256, cap = (size_t)num_sms() * 8;
  su3_deviation_df_kernel<<<(unsigned)(g < cap ? (g < 1 ? 1 : g) : cap), 256, 0, st>>>(d, links, nlinks);
  WMG_LAUNCHED();
  unsigned long long bits = 0;
  WMG_CUDA(cudaMemcpyAsync(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost, st));
  WMG_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(d, st);
  std::memcpy(dev_out, &bits, sizeof(double));
  return MG_OK;
}

int dslash_launch(int dtype, void* out, const void* in, const void* links, const Geom& g,
                  int parity, int dagger, int nrhs, cudaStream_t st, size_t in_stride,
                  size_t out_stride, int link_layout, const void* sub) {
  size_t half = (size_t)12 * (parity < 0 ? g.V : g.V / 2);
  if (in_stride == 0) in_stride = half;
  if (out_stride == 0) out_stride = half;
  switch (dtype) {
    case MG_C128:
      return launch_typed<StC128>(out, in, links, g, parity, dagger, nrhs, st, in_stride, out_stride, dtype,
                                  link_layout, sub);
    case MG_C64:
      return launch_typed<StC64>(out, in, links, g, parity, dagger, nrhs, st, in_stride, out_stride, dtype,
                                  link_layout, sub);
    case MG_F16:
      return launch_typed<StF16>(out, in, links, g, parity, dagger, nrhs, st, in_stride, out_stride, dtype,
                                  link_layout, sub);
    case MG_BF16:
      return launch_typed<StBF16>(out, in, links, g, parity, dagger, nrhs, st, in_stride, out_stride, dtype,
                                  link_layout, sub);
  }
  return fail(MG_EINVAL, "dslash: unknown dtype");
}

}  // namespace wmg

extern "C" int wilson_dslash(void* out, const void* in, const void* links, const int dims[4],
                             double kappa, const double hop_weight[4], const int bc_phase[4],
                             int parity, int dagger, int dtype, int nrhs, void* stream) {
  using namespace wmg;
  if (!out || !in || !links || !dims) return fail(MG_EINVAL, "wilson_dslash: NULL pointer");
  if (nrhs < 1) return fail(MG_EINVAL, "wilson_dslash: nrhs < 1");
  if (parity < -1 || parity > 1) return fail(MG_EINVAL, "wilson_dslash: parity must be -1, 0 or 1");
  if (dtype < MG_C128 || dtype > MG_BF16) return fail(MG_EINVAL, "wilson_dslash: bad dtype");
  double w1[4] = {1, 1, 1, 1};
  int bc1[4] = {1, 1, 1, 1};
  Geom g;
  WMG_TRY(make_geom(g, dims, kappa, hop_weight ? hop_weight : w1, bc_phase ? bc_phase : bc1,
                    parity >= 0));
  if (out == in) return fail(MG_EINVAL, "wilson_dslash: out must not alias in");
  cudaStream_t st = (cudaStream_t)stream;
  size_t eb = dtype_bytes(dtype);
  size_t fsites = parity < 0 ? (size_t)g.V : (size_t)g.V / 2;
  size_t fbytes = fsites * 12 * eb * nrhs;
  size_t lbytes = (size_t)4 * g.V * 9 * eb;
  Staged sin, sl, sout;
  WMG_TRY(stage_in(sin, in, fbytes, st));
  WMG_TRY(stage_in(sl, links, lbytes, st));
  WMG_TRY(stage_out_alloc(sout, out, fbytes, st));
  if (((uintptr_t)sin.dev | (uintptr_t)sout.dev) & 15)
    return fail(MG_EINVAL, "wilson_dslash: spinor fields must be 16-byte aligned");
  if ((uintptr_t)sl.dev & (eb >= 8 ? 7 : 3))
    return fail(MG_EINVAL, "wilson_dslash: links misaligned for their dtype");
  WMG_TRY(dslash_launch(dtype, sout.dev, sin.dev, sl.dev, g, parity, dagger, nrhs, st, 0, 0));
  WMG_TRY(stage_out_finish(sout, out, fbytes, st));
  return MG_OK;
}
