// Device building blocks of the Wilson-Dirac stencil (the operator D of Eq. 1), shared by
// the single- and multi-right-hand-side kernels: site loads/stores of every storage type,
// link loads in both layouts, the spin projections (1 -/+ gamma_mu) of the chiral basis,
// colour transport by U or U^dag, reconstruction, and one hop in each direction.
#pragma once

#include "common.cuh"
#include "internal.h"
#include "vec.cuh"

namespace wmg {
namespace stencil {

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
// consecutive sites touches one contiguous 32 x element_size span (the solver's copy);
// LL = 2: the same with the first two rows only, [mu][6 entry][site]: for U in SU(3) the rows
// are orthonormal and det U = 1, so the third row is the complex conjugate of the cross
// product of the first two (12 of the 18 reals cross HBM).
template <typename S, int LL>
__device__ __forceinline__ void load_link(const typename S::elem* L, int V, int mu, int site,
                                          cplx<typename S::real> u[9]) {
  if (LL == 0) {
    size_t idx = ((size_t)mu * V + site) * 9;
#pragma unroll
    for (int i = 0; i < 9; ++i) u[i] = S::ld(L, idx + i);
  } else if (LL == 1) {
#pragma unroll
    for (int i = 0; i < 9; ++i) u[i] = S::ld(L, ((size_t)mu * 9 + i) * V + site);
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) u[i] = S::ld(L, ((size_t)mu * 6 + i) * V + site);
    u[6] = conj(u[1] * u[5] - u[2] * u[4]);
    u[7] = conj(u[2] * u[3] - u[0] * u[5]);
    u[8] = conj(u[0] * u[4] - u[1] * u[3]);
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
  // single-parity form only: when set, out_p = sub_p - (-kappa H_{p,1-p} in) (the even-odd
  // Schur complement and its source / reconstruction steps), sub with out's layout and stride
  const void* sub = nullptr;
};

// res <- sub[rhs][i] - res for the single-parity form with a subtrahend field
template <typename S>
__device__ __forceinline__ void apply_sub(const KGeom& g, size_t rhs_off, int i,
                                          cplx<typename S::real> res[12]);

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

template <typename S>
__device__ __forceinline__ void apply_sub(const KGeom& g, size_t rhs_off, int i,
                                          cplx<typename S::real> res[12]) {
  if (!g.sub) return;
  cplx<typename S::real> b[12];
  SiteIO<S>::load(static_cast<const typename S::elem*>(g.sub) + rhs_off, (size_t)i, b);
#pragma unroll
  for (int k = 0; k < 12; ++k) res[k] = b[k] - res[k];
}

inline KGeom to_kgeom(const Geom& g) {
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

// Stencil with 2 or 4 right-hand sides per thread (nr), defined in dslash_mrhs.cu for the four
// storage types; layout 0: ABI links, 1: lane-contiguous links.
template <typename S>
void launch_dslash_mrhs(int nr, int dagger, int layout, void* out, const void* in,
                        const void* links, const KGeom& k, int parity, int nsites, int nrhs,
                        cudaStream_t st, size_t in_stride, size_t out_stride);

}  // namespace stencil
}  // namespace wmg
