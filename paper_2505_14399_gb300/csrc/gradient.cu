// Link-angle gradient of a loss through x = D^{-1} b (adjoint of the Wilson-Dirac stencil).
//
// With g_b = D^{-dag} g_x and U_mu(y) -> exp(i omega^a T^a) U_mu(y), only the two hops of
// D that use U_mu(y) change, and
//   dL/d omega^a_mu(y) = -Re[ g_b^dag dD x ] = -kappa w_mu phi Im tr( T^a C ),
//   C = U A - B U^dag,  A = sum_s x_s(y+mu) h_s^dag,  h = (1 - gamma_mu) g_b(y),
//                       B = sum_s x_s(y) h'_s^dag,   h' = (1 + gamma_mu) g_b(y+mu),
// with phi = bc[mu] when the hop wraps the lattice; T^a = lambda^a / 2 (Gell-Mann).
#include "common.cuh"
#include "internal.h"

namespace wmg {

namespace {

// (gamma_mu psi) in the chiral basis: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = [[0,1],[1,0]]
__device__ void gamma_apply(int mu, const zd p[12], zd out[12]) {
  for (int c = 0; c < 3; ++c) {
    zd u0 = p[c], u1 = p[3 + c], d0 = p[6 + c], d1 = p[9 + c];
    zd su0, su1, sd0, sd1;  // sigma applied to up / down pairs
    if (mu == 0) { su0 = u1; su1 = u0; sd0 = d1; sd1 = d0; }
    else if (mu == 1) { su0 = tmi(u1); su1 = ti(u0); sd0 = tmi(d1); sd1 = ti(d0); }
    else if (mu == 2) { su0 = u0; su1 = -u1; sd0 = d0; sd1 = -d1; }
    if (mu < 3) {
      out[c] = tmi(sd0);      // -i sigma psi_dn
      out[3 + c] = tmi(sd1);
      out[6 + c] = ti(su0);   // i sigma psi_up
      out[9 + c] = ti(su1);
    } else {
      out[c] = d0; out[3 + c] = d1; out[6 + c] = u0; out[9 + c] = u1;
    }
  }
}

__global__ void link_gradient_kernel(double* out, const zd* __restrict__ gb, const zd* __restrict__ x,
                                     const zd* __restrict__ links, Geom g, int sx, int sy, int sz,
                                     int st) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 4 * g.V) return;
  int mu = e / g.V, y = e % g.V;
  int c[4];
  c[0] = y % g.L[0];
  int r = y / g.L[0];
  c[1] = r % g.L[1]; r /= g.L[1];
  c[2] = r % g.L[2]; c[3] = r / g.L[2];
  int stride[4] = {sx, sy, sz, st};
  bool wrap = c[mu] == g.L[mu] - 1;
  int yp = wrap ? y - (g.L[mu] - 1) * stride[mu] : y + stride[mu];
  double phi = (wrap && g.bc[mu] < 0) ? -1.0 : 1.0;
  zd gy[12], gyp[12], xy[12], xyp[12], tg[12], tgp[12], U[9];
  for (int i = 0; i < 12; ++i) {
    gy[i] = gb[(size_t)y * 12 + i];
    gyp[i] = gb[(size_t)yp * 12 + i];
    xy[i] = x[(size_t)y * 12 + i];
    xyp[i] = x[(size_t)yp * 12 + i];
  }
  for (int i = 0; i < 9; ++i) U[i] = links[((size_t)mu * g.V + y) * 9 + i];
  gamma_apply(mu, gy, tg);
  gamma_apply(mu, gyp, tgp);
  zd h[12], hp[12];
  for (int i = 0; i < 12; ++i) {
    h[i] = gy[i] - tg[i];     // (1 - gamma) g(y)
    hp[i] = gyp[i] + tgp[i];  // (1 + gamma) g(y+mu)
  }
  zd A[9], B[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      zd sa = {0, 0}, sb = {0, 0};
      for (int s = 0; s < 4; ++s) {
        sa = sa + xyp[s * 3 + a] * conj(h[s * 3 + b]);
        sb = sb + xy[s * 3 + a] * conj(hp[s * 3 + b]);
      }
      A[a * 3 + b] = sa;
      B[a * 3 + b] = sb;
    }
  zd C[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      zd ua = {0, 0}, bu = {0, 0};
      for (int q = 0; q < 3; ++q) {
        ua = ua + U[a * 3 + q] * A[q * 3 + b];
        bu = bu + B[a * 3 + q] * conj(U[b * 3 + q]);  // (U^dag)_{qb} = conj(U_{bq})
      }
      C[a * 3 + b] = ua - bu;
    }
  // tr(lambda^a C)
  zd tr[8];
  tr[0] = C[1 * 3 + 0] + C[0 * 3 + 1];
  tr[1] = tmi(C[1 * 3 + 0]) + ti(C[0 * 3 + 1]);
  tr[2] = C[0] - C[4];
  tr[3] = C[2 * 3 + 0] + C[0 * 3 + 2];
  tr[4] = tmi(C[2 * 3 + 0]) + ti(C[0 * 3 + 2]);
  tr[5] = C[2 * 3 + 1] + C[1 * 3 + 2];
  tr[6] = tmi(C[2 * 3 + 1]) + ti(C[1 * 3 + 2]);
  zd d8 = C[0] + C[4] - 2.0 * C[8];
  tr[7] = (1.0 / sqrt(3.0)) * d8;
  double f = -g.kappa * g.w[mu] * phi * 0.5;
  for (int a = 0; a < 8; ++a) out[((size_t)mu * g.V + y) * 8 + a] = f * tr[a].im;
}

}  // namespace

int link_gradient_launch(double* out, const zd* gb, const zd* x, const zd* links, const Geom& g,
                         cudaStream_t st) {
  int tot = 4 * g.V;
  link_gradient_kernel<<<(tot + 127) / 128, 128, 0, st>>>(
      out, gb, x, links, g, 1, g.L[0], g.L[0] * g.L[1], g.L[0] * g.L[1] * g.L[2]);
  WMG_LAUNCHED();
  return MG_OK;
}

}  // namespace wmg

extern "C" int wilson_link_gradient(void* out, const void* g_b, const void* x, const void* links,
                                    const int dims[4], double kappa, const double hop_weight[4],
                                    const int bc_phase[4], void* stream) {
  using namespace wmg;
  if (!out || !g_b || !x || !links || !dims) return fail(MG_EINVAL, "wilson_link_gradient: NULL pointer");
  double w1[4] = {1, 1, 1, 1};
  int bc1[4] = {1, 1, 1, 1};
  Geom g;
  WMG_TRY(make_geom(g, dims, kappa, hop_weight ? hop_weight : w1, bc_phase ? bc_phase : bc1, false));
  cudaStream_t st = (cudaStream_t)stream;
  size_t fb = (size_t)g.V * 12 * sizeof(zd);
  Staged sg, sx, sl, so;
  WMG_TRY(stage_in(sg, g_b, fb, st));
  WMG_TRY(stage_in(sx, x, fb, st));
  WMG_TRY(stage_in(sl, links, (size_t)4 * g.V * 9 * sizeof(zd), st));
  WMG_TRY(stage_out_alloc(so, out, (size_t)4 * g.V * 8 * sizeof(double), st));
  WMG_TRY(link_gradient_launch((double*)so.dev, (const zd*)sg.dev, (const zd*)sx.dev,
                               (const zd*)sl.dev, g, st));
  WMG_TRY(stage_out_finish(so, out, (size_t)4 * g.V * 8 * sizeof(double), st));
  return MG_OK;
}
