// Wilson-Dirac stencil (Eq. 1) for several right-hand sides per thread: each link is loaded
// once and applied to NR spinors (the test-vector streams of the setup smoothing, Eq. 2, and
// batched solves), so link bytes are shared across the right-hand sides and every thread
// keeps NR independent neighbour loads in flight per hop.
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "stencil.cuh"

namespace wmg {

namespace {

using namespace stencil;

template <int MU, int DAG, typename S, int LL, int NR>
__device__ __forceinline__ void hop_fwd_m(const KGeom& g, int site, const int c[4],
                                          const typename S::elem* in, size_t in_stride, int nr,
                                          bool half_in, const typename S::elem* links,
                                          cplx<typename S::real> acc[NR][12]) {
  typedef typename S::real R;
  constexpr int SF = DAG ? +1 : -1;
  R w = wgt<R>(g, MU);
  int nb = (c[MU] == g.L[MU] - 1) ? site - (g.L[MU] - 1) * g.stride[MU] : site + g.stride[MU];
  R cf = (c[MU] == g.L[MU] - 1 && g.bc[MU] < 0) ? -w : w;
  size_t idx = half_in ? (size_t)(nb >> 1) : (size_t)nb;
  cplx<R> u[9];
  load_link<S, LL>(links, g.V, MU, site, u);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    // a ragged last group re-reads its last right-hand side (discarded at the store), so the
    // loads carry no branch and all NR can be in flight at once
    {
      cplx<R> p[12], h[6], gg[6];
      SiteIO<S>::load(in + (r < nr ? r : nr - 1) * in_stride, idx, p);
      project<MU, SF, R>(p, h);
#pragma unroll
      for (int i = 0; i < 6; ++i) h[i] = cf * h[i];
      mul_link<R>(u, h, gg);
      accumulate<MU, SF, R>(acc[r], gg);
    }
  }
}

template <int MU, int DAG, typename S, int LL, int NR>
__device__ __forceinline__ void hop_bwd_m(const KGeom& g, int site, const int c[4],
                                          const typename S::elem* in, size_t in_stride, int nr,
                                          bool half_in, const typename S::elem* links,
                                          cplx<typename S::real> acc[NR][12]) {
  typedef typename S::real R;
  constexpr int SB = DAG ? -1 : +1;
  R w = wgt<R>(g, MU);
  int nb = (c[MU] == 0) ? site + (g.L[MU] - 1) * g.stride[MU] : site - g.stride[MU];
  R cf = (c[MU] == 0 && g.bc[MU] < 0) ? -w : w;
  size_t idx = half_in ? (size_t)(nb >> 1) : (size_t)nb;
  cplx<R> u[9];
  load_link<S, LL>(links, g.V, MU, nb, u);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    // a ragged last group re-reads its last right-hand side (discarded at the store), so the
    // loads carry no branch and all NR can be in flight at once
    {
      cplx<R> p[12], h[6], gg[6];
      SiteIO<S>::load(in + (r < nr ? r : nr - 1) * in_stride, idx, p);
      project<MU, SB, R>(p, h);
#pragma unroll
      for (int i = 0; i < 6; ++i) h[i] = cf * h[i];
      mul_link_dag<R>(u, h, gg);
      accumulate<MU, SB, R>(acc[r], gg);
    }
  }
}

// One thread per site and group of NR right-hand sides (grid.y = groups); the last group
// may hold fewer than NR.
template <typename S, int DAG, int NR, int LL, int MINB>
__global__ void __launch_bounds__(128, MINB)
dslash_mrhs_kernel(typename S::elem* __restrict__ out, const typename S::elem* __restrict__ in,
                   const typename S::elem* __restrict__ links, KGeom g, int parity, int nsites,
                   int nrhs, size_t in_stride, size_t out_stride) {
  dep_entry();
  typedef typename S::real R;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsites) return;
  const int r0 = blockIdx.y * NR;
  const int nr = min(NR, nrhs - r0);
  int c[4];
  const int site = stencil_site(g, parity, i, c);
  const bool half_in = parity >= 0;
  const typename S::elem* inr = in + (size_t)r0 * in_stride;
  cplx<R> acc[NR][12];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[r][k] = {0, 0};
  hop_fwd_m<0, DAG, S, LL, NR>(g, site, c, inr, in_stride, nr, half_in, links, acc);
  hop_bwd_m<0, DAG, S, LL, NR>(g, site, c, inr, in_stride, nr, half_in, links, acc);
  hop_fwd_m<1, DAG, S, LL, NR>(g, site, c, inr, in_stride, nr, half_in, links, acc);
  hop_bwd_m<1, DAG, S, LL, NR>(g, site, c, inr, in_stride, nr, half_in, links, acc);
  hop_fwd_m<2, DAG, S, LL, NR>(g, site, c, inr, in_stride, nr, half_in, links, acc);
  hop_bwd_m<2, DAG, S, LL, NR>(g, site, c, inr, in_stride, nr, half_in, links, acc);
  hop_fwd_m<3, DAG, S, LL, NR>(g, site, c, inr, in_stride, nr, half_in, links, acc);
  hop_bwd_m<3, DAG, S, LL, NR>(g, site, c, inr, in_stride, nr, half_in, links, acc);
  const R mk = (R)(-g.kappa);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (r < nr) {
      cplx<R> res[12];
      typename S::elem* o = out + (size_t)(r0 + r) * out_stride;
      if (parity < 0) {
        cplx<R> p[12];
        SiteIO<S>::load(inr + r * in_stride, (size_t)site, p);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          res[k].re = fma(mk, acc[r][k].re, p[k].re);
          res[k].im = fma(mk, acc[r][k].im, p[k].im);
        }
        SiteIO<S>::store(o, (size_t)site, res);
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) res[k] = mk * acc[r][k];
        apply_sub<S>(g, (size_t)(r0 + r) * out_stride, i, res);
        SiteIO<S>::store(o, (size_t)i, res);
      }
    }
  }
}

template <typename S, int DAG, int NR, int LL, int MINB>
void launch_nr(void* out, const void* in, const void* links, const KGeom& k, int parity,
               int nsites, int nrhs, cudaStream_t st, size_t is, size_t os) {
  typedef typename S::elem E;
  dim3 grid((nsites + 127) / 128, (nrhs + NR - 1) / NR);
  launch_dep(dslash_mrhs_kernel<S, DAG, NR, LL, MINB>, grid, 128, 0, st, (E*)out, (const E*)in,
             (const E*)links, k, parity, nsites, nrhs, is, os);
}

template <typename S, int DAG, int LL>
void launch_dl(int nr, void* out, const void* in, const void* links, const KGeom& k,
               int parity, int nsites, int nrhs, cudaStream_t st, size_t is, size_t os) {
  // register caps measured best on GB300: 2 per thread at <= 128 registers, 4 per thread
  // uncapped (a 168-register cap spills)
  if (nr == 4) launch_nr<S, DAG, 4, LL, 1>(out, in, links, k, parity, nsites, nrhs, st, is, os);
  else launch_nr<S, DAG, 2, LL, 4>(out, in, links, k, parity, nsites, nrhs, st, is, os);
}

}  // namespace

namespace stencil {

template <typename S>
void launch_dslash_mrhs(int nr, int dagger, int layout, void* out, const void* in,
                        const void* links, const KGeom& k, int parity, int nsites, int nrhs,
                        cudaStream_t st, size_t is, size_t os) {
  if (layout == 0) {
    if (dagger) launch_dl<S, 1, 0>(nr, out, in, links, k, parity, nsites, nrhs, st, is, os);
    else launch_dl<S, 0, 0>(nr, out, in, links, k, parity, nsites, nrhs, st, is, os);
  } else if (layout == 1) {
    if (dagger) launch_dl<S, 1, 1>(nr, out, in, links, k, parity, nsites, nrhs, st, is, os);
    else launch_dl<S, 0, 1>(nr, out, in, links, k, parity, nsites, nrhs, st, is, os);
  } else if constexpr (!std::is_same<S, StC128>::value) {
    if (dagger) launch_dl<S, 1, 2>(nr, out, in, links, k, parity, nsites, nrhs, st, is, os);
    else launch_dl<S, 0, 2>(nr, out, in, links, k, parity, nsites, nrhs, st, is, os);
  }
}

template void launch_dslash_mrhs<StC128>(int, int, int, void*, const void*, const void*,
                                         const KGeom&, int, int, int, cudaStream_t, size_t, size_t);
template void launch_dslash_mrhs<StC64>(int, int, int, void*, const void*, const void*,
                                        const KGeom&, int, int, int, cudaStream_t, size_t, size_t);
template void launch_dslash_mrhs<StF16>(int, int, int, void*, const void*, const void*,
                                        const KGeom&, int, int, int, cudaStream_t, size_t, size_t);
template void launch_dslash_mrhs<StBF16>(int, int, int, void*, const void*, const void*,
                                         const KGeom&, int, int, int, cudaStream_t, size_t, size_t);

}  // namespace stencil

}  // namespace wmg
