// Even-odd (Schur-complement) form of D x = b (even-odd preconditioning, Sec. 1).
//
// With the sites ordered (even, odd) the Wilson-Dirac operator is
//     D = [[1, -kappa H_eo], [-kappa H_oe, 1]]
// and eliminating the odd sites leaves D_hat = 1 - kappa^2 H_eo H_oe on the even sites:
//     b_hat = b_e + kappa H_eo b_o,   D_hat x_e = b_hat,   x_o = b_o + kappa H_oe x_e.
// The hops are the single-parity stencil (dslash_launch with parity 0 / 1: -kappa H_{p,1-p}
// on half-lattice fields indexed by site / 2).  This file holds the even/odd split and join
// of full-lattice fields and the D_hat operator; the K-cycle's Schur-form post-smoother
// (mg.cu) is built from them.
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "vec.cuh"

namespace wmg {
namespace {

// site of half index i with parity p: sites 2i and 2i + 1 share a row (Lx even) and have
// opposite parities
__device__ __forceinline__ int eo_site(const int L[4], int i, int p) {
  int s0 = 2 * i;
  int x0 = s0 % L[0];
  int rest = s0 / L[0];
  int y = rest % L[1];
  int z = (rest / L[1]) % L[2];
  int t = rest / (L[1] * L[2]);
  return s0 + (((x0 + y + z + t) & 1) != p ? 1 : 0);
}

struct Dims4 {
  int L[4];
};

// even[rhs][i] = full[rhs][eo_site(i, 0)], odd[rhs][i] = full[rhs][eo_site(i, 1)]
template <typename E>
__global__ void eo_split_kernel(E* __restrict__ even, E* __restrict__ odd,
                                const E* __restrict__ full, Dims4 d, int Vh, int nrhs) {
  size_t total = (size_t)nrhs * Vh * 12;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t rhs = e / ((size_t)Vh * 12), rem = e % ((size_t)Vh * 12);
    int i = (int)(rem / 12), c = (int)(rem % 12);
    size_t fb = rhs * (size_t)Vh * 24;
    if (even) even[e] = full[fb + (size_t)eo_site(d.L, i, 0) * 12 + c];
    if (odd) odd[e] = full[fb + (size_t)eo_site(d.L, i, 1) * 12 + c];
  }
}

template <typename E>
__global__ void eo_join_kernel(E* __restrict__ full, const E* __restrict__ even,
                               const E* __restrict__ odd, Dims4 d, int Vh, int nrhs) {
  size_t total = (size_t)nrhs * Vh * 12;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t rhs = e / ((size_t)Vh * 12), rem = e % ((size_t)Vh * 12);
    int i = (int)(rem / 12), c = (int)(rem % 12);
    size_t fb = rhs * (size_t)Vh * 24;
    full[fb + (size_t)eo_site(d.L, i, 0) * 12 + c] = even[e];
    full[fb + (size_t)eo_site(d.L, i, 1) * 12 + c] = odd[e];
  }
}

// even[rhs][i] = (a - b)[rhs][eo_site(i, 0)], odd[rhs][i] = (a - b)[rhs][eo_site(i, 1)]
template <typename E>
__global__ void eo_split_diff_kernel(E* __restrict__ even, E* __restrict__ odd,
                                     const E* __restrict__ a, const E* __restrict__ b, Dims4 d,
                                     int Vh, int nrhs) {
  size_t total = (size_t)nrhs * Vh * 12;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t rhs = e / ((size_t)Vh * 12), rem = e % ((size_t)Vh * 12);
    int i = (int)(rem / 12), c = (int)(rem % 12);
    size_t fb = rhs * (size_t)Vh * 24;
    const size_t se = fb + (size_t)eo_site(d.L, i, 0) * 12 + c;
    const size_t so = fb + (size_t)eo_site(d.L, i, 1) * 12 + c;
    even[e] = a[se] - b[se];
    odd[e] = a[so] - b[so];
  }
}

// full[rhs][eo_site(i, 0)] += even[rhs][i], full[rhs][eo_site(i, 1)] += odd[rhs][i]
template <typename E>
__global__ void eo_join_add_kernel(E* __restrict__ full, const E* __restrict__ even,
                                   const E* __restrict__ odd, Dims4 d, int Vh, int nrhs) {
  size_t total = (size_t)nrhs * Vh * 12;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t rhs = e / ((size_t)Vh * 12), rem = e % ((size_t)Vh * 12);
    int i = (int)(rem / 12), c = (int)(rem % 12);
    size_t fb = rhs * (size_t)Vh * 24;
    E* pe = full + fb + (size_t)eo_site(d.L, i, 0) * 12 + c;
    E* po = full + fb + (size_t)eo_site(d.L, i, 1) * 12 + c;
    *pe = *pe + even[e];
    *po = *po + odd[e];
  }
}

unsigned grid_for(size_t n) {
  size_t g = (n + 255) / 256, cap = (size_t)num_sms() * 16;
  return (unsigned)(g < cap ? (g < 1 ? 1 : g) : cap);
}

}  // namespace

template <typename E>
int eo_split(E* even, E* odd, const E* full, const Geom& g, int nrhs, cudaStream_t st) {
  Dims4 d{{g.L[0], g.L[1], g.L[2], g.L[3]}};
  int Vh = g.V / 2;
  eo_split_kernel<E><<<grid_for((size_t)nrhs * Vh * 12), 256, 0, st>>>(even, odd, full, d, Vh, nrhs);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename E>
int eo_join(E* full, const E* even, const E* odd, const Geom& g, int nrhs, cudaStream_t st) {
  Dims4 d{{g.L[0], g.L[1], g.L[2], g.L[3]}};
  int Vh = g.V / 2;
  eo_join_kernel<E><<<grid_for((size_t)nrhs * Vh * 12), 256, 0, st>>>(full, even, odd, d, Vh, nrhs);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename E>
int eo_join_add(E* full, const E* even, const E* odd, const Geom& g, int nrhs, cudaStream_t st) {
  Dims4 d{{g.L[0], g.L[1], g.L[2], g.L[3]}};
  int Vh = g.V / 2;
  eo_join_add_kernel<E><<<grid_for((size_t)nrhs * Vh * 12), 256, 0, st>>>(full, even, odd, d, Vh,
                                                                         nrhs);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename E>
int eo_split_diff(E* even, E* odd, const E* a, const E* b, const Geom& g, int nrhs,
                  cudaStream_t st) {
  Dims4 d{{g.L[0], g.L[1], g.L[2], g.L[3]}};
  int Vh = g.V / 2;
  eo_split_diff_kernel<E><<<grid_for((size_t)nrhs * Vh * 12), 256, 0, st>>>(even, odd, a, b, d,
                                                                           Vh, nrhs);
  WMG_LAUNCHED();
  return MG_OK;
}

// out = D_hat in = in - (-kappa H_eo)(-kappa H_oe) in on even half-lattice fields (dagger:
// D_hat^dag, both hops daggered); tmp: an odd half-lattice field per right-hand side.
template <typename E>
int schur_apply(E* out, const E* in, E* tmp, const void* links, int layout, const Geom& g,
                int dagger, int nrhs, cudaStream_t st) {
  constexpr int dt = std::is_same<E, zd>::value   ? MG_C128
                     : std::is_same<E, zf>::value ? MG_C64
                     : std::is_same<E, zh>::value ? MG_F16
                                                  : MG_BF16;
  size_t nh = (size_t)(g.V / 2) * 12;
  WMG_TRY(dslash_launch(dt, tmp, in, links, g, 1, dagger, nrhs, st, nh, nh, layout));
  // out = in - (-kappa H_eo) tmp, the subtraction fused into the second hop
  WMG_TRY(dslash_launch(dt, out, tmp, links, g, 0, dagger, nrhs, st, nh, nh, layout, in));
  return MG_OK;
}

#define INST_EO(E)                                                                        \
  template int eo_split<E>(E*, E*, const E*, const Geom&, int, cudaStream_t);             \
  template int eo_join<E>(E*, const E*, const E*, const Geom&, int, cudaStream_t);        \
  template int schur_apply<E>(E*, const E*, E*, const void*, int, const Geom&, int, int, \
                              cudaStream_t);
INST_EO(zd)
INST_EO(zf)
INST_EO(zh)
template int eo_join_add<zd>(zd*, const zd*, const zd*, const Geom&, int, cudaStream_t);
template int eo_join_add<zf>(zf*, const zf*, const zf*, const Geom&, int, cudaStream_t);
template int eo_split_diff<zd>(zd*, zd*, const zd*, const zd*, const Geom&, int, cudaStream_t);
template int eo_split_diff<zf>(zf*, zf*, const zf*, const zf*, const Geom&, int, cudaStream_t);
INST_EO(zbf)

}  // namespace wmg

extern "C" int wilson_schur(void* out, const void* in, const void* links, const int dims[4],
                            double kappa, const double hop_weight[4], const int bc_phase[4],
                            int dagger, int dtype, int nrhs, void* stream) {
  using namespace wmg;
  if (!out || !in || !links || !dims) return fail(MG_EINVAL, "wilson_schur: NULL pointer");
  if (nrhs < 1) return fail(MG_EINVAL, "wilson_schur: nrhs < 1");
  if (dtype < MG_C128 || dtype > MG_BF16) return fail(MG_EINVAL, "wilson_schur: bad dtype");
  if (out == in) return fail(MG_EINVAL, "wilson_schur: out must not alias in");
  double w1[4] = {1, 1, 1, 1};
  int bc1[4] = {1, 1, 1, 1};
  Geom g;
  WMG_TRY(make_geom(g, dims, kappa, hop_weight ? hop_weight : w1, bc_phase ? bc_phase : bc1, true));
  cudaStream_t st = (cudaStream_t)stream;
  size_t eb = dtype_bytes(dtype);
  size_t fbytes = (size_t)(g.V / 2) * 12 * eb * nrhs;
  Staged sin, sl, sout;
  WMG_TRY(stage_in(sin, in, fbytes, st));
  WMG_TRY(stage_in(sl, links, (size_t)4 * g.V * 9 * eb, st));
  WMG_TRY(stage_out_alloc(sout, out, fbytes, st));
  if (((uintptr_t)sin.dev | (uintptr_t)sout.dev) & 15)
    return fail(MG_EINVAL, "wilson_schur: spinor fields must be 16-byte aligned");
  void* tmp = nullptr;
  WMG_CUDA(cudaMallocAsync(&tmp, fbytes, st));
  int s = MG_OK;
  switch (dtype) {
    case MG_C128: s = schur_apply<zd>((zd*)sout.dev, (const zd*)sin.dev, (zd*)tmp, sl.dev, 0, g, dagger, nrhs, st); break;
    case MG_C64: s = schur_apply<zf>((zf*)sout.dev, (const zf*)sin.dev, (zf*)tmp, sl.dev, 0, g, dagger, nrhs, st); break;
    case MG_F16: s = schur_apply<zh>((zh*)sout.dev, (const zh*)sin.dev, (zh*)tmp, sl.dev, 0, g, dagger, nrhs, st); break;
    default: s = schur_apply<zbf>((zbf*)sout.dev, (const zbf*)sin.dev, (zbf*)tmp, sl.dev, 0, g, dagger, nrhs, st); break;
  }
  cudaFreeAsync(tmp, st);
  WMG_TRY(s);
  WMG_TRY(stage_out_finish(sout, out, fbytes, st));
  return MG_OK;
}
