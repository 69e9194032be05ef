// Wilson-Dirac stencil (the operator D of Eq. 1), full and single-parity, any storage.
//
// One thread per output site and right-hand side.  Each of the 8 hops loads the
// neighbour spinor, projects it to a 2-spin half spinor with (1 -/+ gamma_mu) in the
// chiral basis, multiplies by U_mu(x) or U_mu(x-mu)^dag, and reconstructs the lower
// spin pair from the upper one.  Spinor loads are 16-byte vector loads of the
// [site][spin][colour] layout; links are read through the read-only path.
#include "common.cuh"
#include "internal.h"
#include "vec.cuh"

namespace wmg {

namespace {

// 16-byte vector loads/stores of one site's 12 complex numbers.
template <typename S> struct SiteIO;

template <> struct SiteIO<StC128> {
  static __device__ __forceinline__ void load(const double2* p, size_t site, zd v[12]) {
    const double2* q = p + site * 12;
#pragma unroll
    for (int i = 0; i < 12; ++i) { double2 t = __ldg(q + i); v[i] = {t.x, t.y}; }
  }
  static __device__ __forceinline__ void store(double2* p, size_t site, const zd v[12]) {
    double2* q = p + site * 12;
#pragma unroll
    for (int i = 0; i < 12; ++i) q[i] = make_double2(v[i].re, v[i].im);
  }
};
template <> struct SiteIO<StC64> {
  static __device__ __forceinline__ void load(const float2* p, size_t site, zf v[12]) {
    const float4* q = reinterpret_cast<const float4*>(p + site * 12);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      float4 t = __ldg(q + i);
      v[2 * i] = {t.x, t.y};
      v[2 * i + 1] = {t.z, t.w};
    }
  }
  static __device__ __forceinline__ void store(float2* p, size_t site, const zf v[12]) {
    float4* q = reinterpret_cast<float4*>(p + site * 12);
#pragma unroll
    for (int i = 0; i < 6; ++i)
      q[i] = make_float4(v[2 * i].re, v[2 * i].im, v[2 * i + 1].re, v[2 * i + 1].im);
  }
};
template <typename H, typename S> struct SiteIOHalf {
  static __device__ __forceinline__ void load(const H* p, size_t site, zf v[12]) {
    const uint4* q = reinterpret_cast<const uint4*>(p + site * 12);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      uint4 t = __ldg(q + i);
      const H* h = reinterpret_cast<const H*>(&t);
#pragma unroll
      for (int j = 0; j < 4; ++j) v[4 * i + j] = S::ld(h, j);
    }
  }
  static __device__ __forceinline__ void store(H* p, size_t site, const zf v[12]) {
    uint4* q = reinterpret_cast<uint4*>(p + site * 12);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      uint4 t;
      H* h = reinterpret_cast<H*>(&t);
#pragma unroll
      for (int j = 0; j < 4; ++j) S::st(h, j, v[4 * i + j]);
      q[i] = t;
    }
  }
};
template <> struct SiteIO<StF16> : SiteIOHalf<__half2, StF16> {};
template <> struct SiteIO<StBF16> : SiteIOHalf<__nv_bfloat162, StBF16> {};

// Load the 3x3 link U_mu(site).  LL = 0: ABI layout [mu][site][3][3] (one link contiguous);
// LL = 1: lane-contiguous layout [mu][3x3 entry][site], so a warp reading one entry for 32
// consecutive sites touches one contiguous 32 x element_size span (the solver's copy).
template <typename S, int LL>
__device__ __forceinline__ void load_link(const typename S::elem* L, int V, int mu, int site,
                                          cplx<typename S::real> u[9]) {
  if (LL == 0) {
    size_t idx = ((size_t)mu * V + site) * 9;
#pragma unroll
    for (int i = 0; i < 9; ++i) u[i] = S::ld(L, idx + i);
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) u[i] = S::ld(L, ((size_t)mu * 9 + i) * V + site);
  }
}

// Project psi with (1 + s gamma_mu) to the upper spin pair h (2 spins x 3 colours),
// scaled by c.  mu = 0,1,2: h = psi_up - s i sigma_mu psi_dn; mu = 3: h = psi_up + s psi_dn.
template <int MU, int SGN, typename R>
__device__ __forceinline__ void project(const cplx<R> p[12], cplx<R> h[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cplx<R> u0 = p[0 * 3 + c], u1 = p[1 * 3 + c], d0 = p[2 * 3 + c], d1 = p[3 * 3 + c];
    cplx<R> a, b;  // i sigma psi_dn, components 0 and 1
    if (MU == 0) { a = ti(d1); b = ti(d0); }
    else if (MU == 1) { a = d1; b = -d0; }
    else if (MU == 2) { a = ti(d0); b = tmi(d1); }
    else { a = d0; b = d1; }
    if (MU < 3) {
      if (SGN > 0) { h[c] = u0 - a; h[3 + c] = u1 - b; }
      else { h[c] = u0 + a; h[3 + c] = u1 + b; }
    } else {
      if (SGN > 0) { h[c] = u0 + a; h[3 + c] = u1 + b; }
      else { h[c] = u0 - a; h[3 + c] = u1 - b; }
    }
  }
}

// acc += (1 + s gamma_mu) reconstructed from the transported half spinor g:
// upper = g; lower = s i sigma_mu g (mu < 3) or s g (mu = 3).
template <int MU, int SGN, typename R>
__device__ __forceinline__ void accumulate(cplx<R> acc[12], const cplx<R> g[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    cplx<R> g0 = g[c], g1 = g[3 + c];
    acc[0 * 3 + c] += g0;
    acc[1 * 3 + c] += g1;
    cplx<R> a, b;  // i sigma g or g
    if (MU == 0) { a = ti(g1); b = ti(g0); }
    else if (MU == 1) { a = g1; b = -g0; }
    else if (MU == 2) { a = ti(g0); b = tmi(g1); }
    else { a = g0; b = g1; }
    if (SGN > 0) { acc[2 * 3 + c] += a; acc[3 * 3 + c] += b; }
    else { acc[2 * 3 + c] -= a; acc[3 * 3 + c] -= b; }
  }
}

template <typename R>
__device__ __forceinline__ void mul_link(const cplx<R> u[9], const cplx<R> h[6], cplx<R> g[6]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cplx<R> t = u[a * 3 + 0] * h[s * 3 + 0];
      cfma(t, u[a * 3 + 1], h[s * 3 + 1]);
      cfma(t, u[a * 3 + 2], h[s * 3 + 2]);
      g[s * 3 + a] = t;
    }
}
template <typename R>
__device__ __forceinline__ void mul_link_dag(const cplx<R> u[9], const cplx<R> h[6], cplx<R> g[6]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cplx<R> t = {0, 0};
      cfmac(t, u[0 * 3 + a], h[s * 3 + 0]);
      cfmac(t, u[1 * 3 + a], h[s * 3 + 1]);
      cfmac(t, u[2 * 3 + a], h[s * 3 + 2]);
      g[s * 3 + a] = t;
    }
}

struct KGeom {
  int L[4];
  int stride[4];
  int V;
  float wf[4];
  double wd[4];
  int bc[4];
  double kappa;
};

template <typename R> __device__ __forceinline__ R wgt(const KGeom& g, int mu);
template <> __device__ __forceinline__ double wgt<double>(const KGeom& g, int mu) { return g.wd[mu]; }
template <> __device__ __forceinline__ float wgt<float>(const KGeom& g, int mu) { return g.wf[mu]; }

// forward hop of direction MU: (1 + SF gamma) U_mu(x) psi(x + mu)
template <int MU, int DAG, typename S, int LL>
__device__ __forceinline__ void hop_fwd(const KGeom& g, int site, const int c[4],
                                        const typename S::elem* in, size_t in_off,
                                        bool half_in, const typename S::elem* links,
                                        cplx<typename S::real> acc[12]) {
  typedef typename S::real R;
  constexpr int SF = DAG ? +1 : -1;  // forward projector sign
  R w = wgt<R>(g, MU);
  int nb = (c[MU] == g.L[MU] - 1) ? site - (g.L[MU] - 1) * g.stride[MU] : site + g.stride[MU];
  R cf = (c[MU] == g.L[MU] - 1 && g.bc[MU] < 0) ? -w : w;
  cplx<R> p[12], h[6], gg[6], u[9];
  SiteIO<S>::load(in + in_off, half_in ? (size_t)(nb >> 1) : (size_t)nb, p);
  project<MU, SF, R>(p, h);
#pragma unroll
  for (int i = 0; i < 6; ++i) h[i] = cf * h[i];
  load_link<S, LL>(links, g.V, MU, site, u);
  mul_link<R>(u, h, gg);
  accumulate<MU, SF, R>(acc, gg);
}

// backward hop of direction MU: (1 + SB gamma) U_mu(x - mu)^dag psi(x - mu)
template <int MU, int DAG, typename S, int LL>
__device__ __forceinline__ void hop_bwd(const KGeom& g, int site, const int c[4],
                                        const typename S::elem* in, size_t in_off,
                                        bool half_in, const typename S::elem* links,
                                        cplx<typename S::real> acc[12]) {
  typedef typename S::real R;
  constexpr int SB = DAG ? -1 : +1;  // backward projector sign
  R w = wgt<R>(g, MU);
  int nb = (c[MU] == 0) ? site + (g.L[MU] - 1) * g.stride[MU] : site - g.stride[MU];
  R cf = (c[MU] == 0 && g.bc[MU] < 0) ? -w : w;
  cplx<R> p[12], h[6], gg[6], u[9];
  SiteIO<S>::load(in + in_off, half_in ? (size_t)(nb >> 1) : (size_t)nb, p);
  project<MU, SB, R>(p, h);
#pragma unroll
  for (int i = 0; i < 6; ++i) h[i] = cf * h[i];
  load_link<S, LL>(links, g.V, MU, nb, u);
  mul_link_dag<R>(u, h, gg);
  accumulate<MU, SB, R>(acc, gg);
}

template <int MU, int DAG, typename S, int LL>
__device__ __forceinline__ void hop_pair(const KGeom& g, int site, const int c[4],
                                         const typename S::elem* in, size_t in_off,
                                         bool half_in, const typename S::elem* links,
                                         cplx<typename S::real> acc[12]) {
  hop_fwd<MU, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
  hop_bwd<MU, DAG, S, LL>(g, site, c, in, in_off, half_in, links, acc);
}

// Site index of thread i (parity < 0: lexicographic; else the i-th site of that parity)
// and its coordinates.
__device__ __forceinline__ int stencil_site(const KGeom& g, int parity, int i, int c[4]) {
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
  c[0] = site % g.L[0];
  int rest = site / g.L[0];
  c[1] = rest % g.L[1];
  rest /= g.L[1];
  c[2] = rest % g.L[2];
  c[3] = rest / g.L[2];
  return site;
}

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
    SiteIO<S>::store(out + rhs * out_stride, (size_t)i, res);
  }
}

KGeom to_kgeom(const Geom& g) {
  KGeom k;
  for (int m = 0; m < 4; ++m) {
    k.L[m] = g.L[m];
    k.wf[m] = (float)g.w[m];
    k.wd[m] = g.w[m];
    k.bc[m] = g.bc[m];
  }
  k.stride[0] = 1;
  k.stride[1] = g.L[0];
  k.stride[2] = g.L[0] * g.L[1];
  k.stride[3] = g.L[0] * g.L[1] * g.L[2];
  k.V = g.V;
  k.kappa = g.kappa;
  return k;
}

// Launch shapes: threads per CTA and the minimum resident CTAs per SM requested from
// the register allocator (register cap = 64K / (TPB * MINB)).  The autotuner below
// picks one per (dtype, parity, dagger, volume, nrhs).
struct Shape {
  int tpb, minb;
};
constexpr Shape kShapes[] = {{128, 1}, {128, 6}, {128, 8}, {256, 4}, {64, 16}, {128, 0}};
// the last entry is the two-threads-per-site kernel (dslash_split_kernel)
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

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
    default: launch_shape<S, DAG, 128, 1, LL>(out, in, links, k, parity, nsites, nrhs, st, is, os); break;
  }
}

template <typename S>
int launch_typed(void* out, const void* in, const void* links, const Geom& g, int parity,
                 int dagger, int nrhs, cudaStream_t st, size_t in_stride, size_t out_stride,
                 int dtype, int layout) {
  KGeom k = to_kgeom(g);
  int nsites = parity < 0 ? g.V : g.V / 2;
  auto run = [&](int v) {
    if (layout == 0) {
      if (dagger) launch_variant<S, 1, 0>(v, out, in, links, k, parity, nsites, nrhs, st, in_stride, out_stride);
      else launch_variant<S, 0, 0>(v, out, in, links, k, parity, nsites, nrhs, st, in_stride, out_stride);
    } else {
      if (dagger) launch_variant<S, 1, 1>(v, out, in, links, k, parity, nsites, nrhs, st, in_stride, out_stride);
      else launch_variant<S, 0, 1>(v, out, in, links, k, parity, nsites, nrhs, st, in_stride, out_stride);
    }
  };
  int v = tuned_variant(dtype + 16 * layout, parity, dagger, g.V, nrhs, st, kNumShapes, run);
  if (v < 0) return fail(MG_ECUDA, "dslash autotune failed");
  // algorithmic bytes: in + out spinors per rhs and each link once (parity: all 4V links)
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
__global__ void link_to_lanes_kernel(E* dst, const zd* __restrict__ src, int V) {
  typedef typename VecT<E>::R R;
  size_t total = (size_t)4 * V * 9;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    // e enumerates the destination [mu][entry][site]
    size_t site = e % V, rest = e / V;
    int entry = (int)(rest % 9), mu = (int)(rest / 9);
    zd v = src[((size_t)mu * V + site) * 9 + entry];
    VecT<E>::st(dst, e, cplx<R>{(R)v.re, (R)v.im});
  }
}

}  // namespace

template <typename E>
int link_to_lanes_v(E* dst, const zd* src, int V, cudaStream_t st) {
  size_t total = (size_t)4 * V * 9;
  size_t g = (total + 255) / 256, cap = (size_t)num_sms() * 16;
  link_to_lanes_kernel<E><<<(unsigned)(g < cap ? g : cap), 256, 0, st>>>(dst, src, V);
  WMG_LAUNCHED();
  return MG_OK;
}
template int link_to_lanes_v<zd>(zd*, const zd*, int, cudaStream_t);
template int link_to_lanes_v<zf>(zf*, const zd*, int, cudaStream_t);
template int link_to_lanes_v<zh>(zh*, const zd*, int, cudaStream_t);
template int link_to_lanes_v<zbf>(zbf*, const zd*, int, cudaStream_t);

int dslash_launch(int dtype, void* out, const void* in, const void* links, const Geom& g,
                  int parity, int dagger, int nrhs, cudaStream_t st, size_t in_stride,
                  size_t out_stride, int link_layout) {
  size_t half = (size_t)12 * (parity < 0 ? g.V : g.V / 2);
  if (in_stride == 0) in_stride = half;
  if (out_stride == 0) out_stride = half;
  switch (dtype) {
    case MG_C128:
      return launch_typed<StC128>(out, in, links, g, parity, dagger, nrhs, st, in_stride, out_stride, dtype,
                                  link_layout);
    case MG_C64:
      return launch_typed<StC64>(out, in, links, g, parity, dagger, nrhs, st, in_stride, out_stride, dtype,
                                  link_layout);
    case MG_F16:
      return launch_typed<StF16>(out, in, links, g, parity, dagger, nrhs, st, in_stride, out_stride, dtype,
                                  link_layout);
    case MG_BF16:
      return launch_typed<StBF16>(out, in, links, g, parity, dagger, nrhs, st, in_stride, out_stride, dtype,
                                  link_layout);
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
