// Wilson-clover term (Configuration B of Sec. 4 uses a clover-improved Wilson action whose term
// the paper does not write; this is the textbook Sheikholeslami-Wohlert form):
//
//   D_clover = D_W + C,   C(x) = -kappa c_sw sum_{mu < nu} sigma_mu_nu (x) F_mu_nu(x),
//
// sigma_mu_nu = (i/2)[gamma_mu, gamma_nu] in the chiral basis of the library (it commutes with
// gamma_5, so C is block diagonal in the chirality: two 6 x 6 Hermitian blocks per site), and
// F_mu_nu(x) the traceless part of (Q - Q^dag) / (8 i), Q the sum of the four plaquettes of the
// mu-nu plane that start and end at x, each taken counter-clockwise (mu first, then nu):
//   U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
//   U_nu(x) U_mu(x+nu-mu)^dag U_nu(x-mu)^dag U_mu(x-mu)
//   U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
//   U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag.
// The gauge field is periodic (fermion boundary phases do not enter F).
//
// Storage: C[site][alpha][6][6] row-major, rows and columns (spin within chirality, colour).
// Kernels: the field (FP64, one thread per site), the site-local apply out += C in, and the
// clover part of the Galerkin diagonal, X_j += sum_{x in Lambda_j} P(x)^dag C(x) P(x).
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace wmg {
namespace {

// the diagonal 2 x 2 blocks of sigma_mu_nu for the six planes: s[p][alpha][2][2]
struct SigmaBlocks {
  zd s[6][2][4];
};

__device__ __forceinline__ void m3_mul(zd* c, const zd* a, const zd* b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      zd t = a[i * 3] * b[j];
      cfma(t, a[i * 3 + 1], b[3 + j]);
      cfma(t, a[i * 3 + 2], b[6 + j]);
      c[i * 3 + j] = t;
    }
}
__device__ __forceinline__ void m3_dag(zd* c, const zd* a) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) c[i * 3 + j] = conj(a[j * 3 + i]);
}

struct LatG {
  int L[4];
  int V;
};

__device__ __forceinline__ int shift(const LatG& g, int s, int mu, int sgn) {
  int c[4];
  c[0] = s % g.L[0];
  int r = s / g.L[0];
  c[1] = r % g.L[1];
  r /= g.L[1];
  c[2] = r % g.L[2];
  c[3] = r / g.L[2];
  c[mu] = (c[mu] + sgn + g.L[mu]) % g.L[mu];
  return c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

__device__ __forceinline__ void ld_link(zd* u, const zd* __restrict__ L, int V, int mu, int s) {
  const zd* p = L + ((size_t)mu * V + s) * 9;
#pragma unroll
  for (int i = 0; i < 9; ++i) u[i] = p[i];
}

// a b c d, each optionally daggered, into out
__device__ __forceinline__ void leaf(zd* out, const zd* a, const zd* b, const zd* c, const zd* d) {
  zd t1[9], t2[9];
  m3_mul(t1, a, b);
  m3_mul(t2, t1, c);
  m3_mul(out, t2, d);
}

__global__ void clover_field_kernel(zd* __restrict__ C, const zd* __restrict__ L, LatG g,
                                    SigmaBlocks sb, double coef) {
  const int PA[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < g.V; x += gridDim.x * blockDim.x) {
    zd acc[2][36];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int e = 0; e < 36; ++e) acc[a][e] = {0, 0};
    for (int p = 0; p < 6; ++p) {
      const int mu = PA[p][0], nu = PA[p][1];
      const int xpm = shift(g, x, mu, +1), xpn = shift(g, x, nu, +1);
      const int xmm = shift(g, x, mu, -1), xmn = shift(g, x, nu, -1);
      const int xpn_mm = shift(g, xpn, mu, -1), xmm_mn = shift(g, xmm, nu, -1);
      const int xmn_pm = shift(g, xmn, mu, +1);
      zd A[9], B[9], Cc[9], D[9], T[9], Q[9];
      // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
      ld_link(A, L, g.V, mu, x);
      ld_link(B, L, g.V, nu, xpm);
      ld_link(T, L, g.V, mu, xpn);
      m3_dag(Cc, T);
      ld_link(T, L, g.V, nu, x);
      m3_dag(D, T);
      leaf(Q, A, B, Cc, D);
      // leaf 2: U_nu(x) U_mu(x+nu-mu)^dag U_nu(x-mu)^dag U_mu(x-mu)
      ld_link(A, L, g.V, nu, x);
      ld_link(T, L, g.V, mu, xpn_mm);
      m3_dag(B, T);
      ld_link(T, L, g.V, nu, xmm);
      m3_dag(Cc, T);
      ld_link(D, L, g.V, mu, xmm);
      leaf(T, A, B, Cc, D);
#pragma unroll
      for (int i = 0; i < 9; ++i) Q[i] += T[i];
      // leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
      ld_link(T, L, g.V, mu, xmm);
      m3_dag(A, T);
      ld_link(T, L, g.V, nu, xmm_mn);
      m3_dag(B, T);
      ld_link(Cc, L, g.V, mu, xmm_mn);
      ld_link(D, L, g.V, nu, xmn);
      leaf(T, A, B, Cc, D);
#pragma unroll
      for (int i = 0; i < 9; ++i) Q[i] += T[i];
      // leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag
      ld_link(T, L, g.V, nu, xmn);
      m3_dag(A, T);
      ld_link(B, L, g.V, mu, xmn);
      ld_link(Cc, L, g.V, nu, xmn_pm);
      ld_link(T, L, g.V, mu, x);
      m3_dag(D, T);
      leaf(T, A, B, Cc, D);
#pragma unroll
      for (int i = 0; i < 9; ++i) Q[i] += T[i];
      // F = traceless part of (Q - Q^dag) / (8 i)
      zd F[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          zd d = Q[i * 3 + j] - conj(Q[j * 3 + i]);
          F[i * 3 + j] = {d.im / 8.0, -d.re / 8.0};   // d / (8 i)
        }
      zd tr = F[0] + F[4] + F[8];
      tr = (1.0 / 3.0) * tr;
      F[0] = F[0] - tr;
      F[4] = F[4] - tr;
      F[8] = F[8] - tr;
      // acc_alpha[(s, c)][(t, d)] += s_alpha[s][t] F[c][d]
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            zd sg = sb.s[p][a][s * 2 + t];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
              for (int d = 0; d < 3; ++d) acc[a][(s * 3 + c) * 6 + t * 3 + d] += sg * F[c * 3 + d];
          }
    }
    zd* out = C + (size_t)x * 72;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int e = 0; e < 36; ++e) out[a * 36 + e] = coef * acc[a][e];
  }
}

// out[rhs][x] += C(x) in[rhs][x], the two chiral 6 x 6 blocks (spins 0,1 and 2,3)
template <typename R>
__global__ void clover_add_kernel(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in,
                                  const cplx<R>* __restrict__ C, int V, int nrhs) {
  const size_t total = (size_t)V * nrhs * 2;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(e & 1);
    const size_t rs = e >> 1;          // rhs * V + x
    const int x = (int)(rs % V);
    const cplx<R>* vin = in + rs * 12 + a * 6;
    cplx<R>* vout = out + rs * 12 + a * 6;
    const cplx<R>* Cx = C + (size_t)x * 72 + a * 36;
    cplx<R> v[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = vin[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      cplx<R> acc = vout[i];
#pragma unroll
      for (int j = 0; j < 6; ++j) cfma(acc, Cx[i * 6 + j], v[j]);
      vout[i] = acc;
    }
  }
}

// X_j[(alpha, a)][(alpha, b)] += sum_l sum_{r, s} conj(P[t][a][6 l + r]) C_alpha(x_l)[r][s]
// P[t][b][6 l + s], t = 2 j + alpha; one CTA per tile, one thread per (a, b); Op column-major
__global__ void clover_galerkin_kernel(zd* Op, const zd* __restrict__ P, const zd* __restrict__ C,
                                       int k, Blocking B) {
  extern __shared__ zd csh[];
  zd* Pl = csh;                    // [k][6]   P rows of one local site
  zd* Cl = Pl + (size_t)k * 6;     // [6][6]
  const int t = blockIdx.x, j = t >> 1, alpha = t & 1;
  const int n2k = 2 * k;
  zd acc = {0, 0};
  const int a = threadIdx.x / k, b = threadIdx.x % k;
  const bool act = threadIdx.x < k * k;
  for (int l = 0; l < B.nd; ++l) {
    const int x = B.site(j, l);
    __syncthreads();
    for (int e = threadIdx.x; e < k * 6; e += blockDim.x)
      Pl[e] = P[((size_t)t * k + e / 6) * B.M + (size_t)l * 6 + e % 6];
    for (int e = threadIdx.x; e < 36; e += blockDim.x) Cl[e] = C[(size_t)x * 72 + alpha * 36 + e];
    __syncthreads();
    if (act) {
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        zd cs = {0, 0};
#pragma unroll
        for (int s = 0; s < 6; ++s) cfma(cs, Cl[r * 6 + s], Pl[b * 6 + s]);
        cfmac(acc, Pl[a * 6 + r], cs);
      }
    }
  }
  if (act) {
    zd* X = Op + (size_t)j * 9 * n2k * n2k;
    const size_t idx = (size_t)(alpha * k + b) * n2k + alpha * k + a;   // column b, row a
    X[idx] = X[idx] + acc;
  }
}

SigmaBlocks sigma_blocks() {
  // chiral basis: gamma_k = [[0, -i s_k], [i s_k, 0]], gamma_4 = [[0, 1], [1, 0]]
  typedef zd M4[4][4];
  const zd I = {0, 1}, Z = {0, 0}, O = {1, 0};
  zd pauli[3][2][2] = {{{Z, O}, {O, Z}}, {{Z, {0, -1}}, {I, Z}}, {{O, Z}, {Z, {-1, 0}}}};
  M4 g[4];
  for (int m = 0; m < 4; ++m)
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) g[m][i][j] = Z;
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        g[k][i][2 + j] = zd{0, -1} * pauli[k][i][j];
        g[k][2 + i][j] = I * pauli[k][i][j];
      }
  for (int i = 0; i < 2; ++i) {
    g[3][i][2 + i] = O;
    g[3][2 + i][i] = O;
  }
  const int PA[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  SigmaBlocks sb;
  for (int p = 0; p < 6; ++p) {
    const int mu = PA[p][0], nu = PA[p][1];
    zd s[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        zd c = Z;
        for (int q = 0; q < 4; ++q) c = c + g[mu][i][q] * g[nu][q][j] - g[nu][i][q] * g[mu][q][j];
        s[i][j] = zd{0, 0.5} * c;      // (i/2) [gamma_mu, gamma_nu]
      }
    for (int a = 0; a < 2; ++a)
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) sb.s[p][a][i * 2 + j] = s[2 * a + i][2 * a + j];
  }
  return sb;
}

unsigned grid_for(size_t n) {
  size_t g = (n + 255) / 256, cap = (size_t)num_sms() * 16;
  return (unsigned)(g < cap ? (g < 1 ? 1 : g) : cap);
}

}  // namespace

int clover_field(zd* C, const zd* links, const Geom& g, double csw, cudaStream_t st) {
  LatG lg{{g.L[0], g.L[1], g.L[2], g.L[3]}, g.V};
  ProfScope ps("clover_field", 16.0 * (36.0 * g.V + 72.0 * g.V), 8.0 * 6 * 16 * 27 * g.V, st);
  clover_field_kernel<<<grid_for(g.V), 128, 0, st>>>(C, links, lg, sigma_blocks(), -g.kappa * csw);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int clover_add(cplx<R>* out, const cplx<R>* in, const cplx<R>* C, int V, int nrhs,
               cudaStream_t st) {
  ProfScope ps("clover_apply", (double)sizeof(cplx<R>) * ((double)V * 72 + 36.0 * V * nrhs),
               8.0 * 72 * V * nrhs, st);
  clover_add_kernel<R><<<grid_for((size_t)V * nrhs * 2), 256, 0, st>>>(out, in, C, V, nrhs);
  WMG_LAUNCHED();
  return MG_OK;
}
template int clover_add<double>(zd*, const zd*, const zd*, int, int, cudaStream_t);
template int clover_add<float>(zf*, const zf*, const zf*, int, int, cudaStream_t);

int clover_galerkin_add(zd* Op, const zd* P, const zd* C, int k, const Blocking& B,
                        cudaStream_t st) {
  size_t sh = sizeof(zd) * ((size_t)k * 6 + 36);
  int thr = ((k * k + 31) / 32) * 32;
  if (thr < 64) thr = 64;
  clover_galerkin_kernel<<<B.d * 2, thr, sh, st>>>(Op, P, C, k, B);
  WMG_LAUNCHED();
  return MG_OK;
}

}  // namespace wmg

extern "C" int wilson_clover_field(void* clover, const void* links, const int dims[4],
                                   double kappa, double csw, void* stream) {
  using namespace wmg;
  if (!clover || !links || !dims) return fail(MG_EINVAL, "wilson_clover_field: NULL pointer");
  double w1[4] = {1, 1, 1, 1};
  int bc1[4] = {1, 1, 1, 1};
  Geom g;
  WMG_TRY(make_geom(g, dims, kappa, w1, bc1, false));
  cudaStream_t st = (cudaStream_t)stream;
  Staged sl, so;
  WMG_TRY(stage_in(sl, links, (size_t)4 * g.V * 9 * sizeof(zd), st));
  WMG_TRY(stage_out_alloc(so, clover, (size_t)g.V * 72 * sizeof(zd), st));
  WMG_TRY(clover_field((zd*)so.dev, (const zd*)sl.dev, g, csw, st));
  WMG_TRY(stage_out_finish(so, clover, (size_t)g.V * 72 * sizeof(zd), st));
  return MG_OK;
}

extern "C" int wilson_clover_apply(void* out, const void* in, const void* links,
                                   const void* clover, const int dims[4], double kappa,
                                   const double hop_weight[4], const int bc_phase[4], int dagger,
                                   int dtype, int nrhs, void* stream) {
  using namespace wmg;
  if (!out || !in || !links || !clover || !dims)
    return fail(MG_EINVAL, "wilson_clover_apply: NULL pointer");
  if (dtype != MG_C128 && dtype != MG_C64)
    return fail(MG_EINVAL, "wilson_clover_apply: dtype must be MG_C128 or MG_C64");
  if (nrhs < 1) return fail(MG_EINVAL, "wilson_clover_apply: nrhs < 1");
  if (out == in) return fail(MG_EINVAL, "wilson_clover_apply: out must not alias in");
  double w1[4] = {1, 1, 1, 1};
  int bc1[4] = {1, 1, 1, 1};
  Geom g;
  WMG_TRY(make_geom(g, dims, kappa, hop_weight ? hop_weight : w1, bc_phase ? bc_phase : bc1, false));
  cudaStream_t st = (cudaStream_t)stream;
  size_t eb = dtype_bytes(dtype);
  size_t fbytes = (size_t)g.V * 12 * eb * nrhs;
  Staged si, sl, sc, so;
  WMG_TRY(stage_in(si, in, fbytes, st));
  WMG_TRY(stage_in(sl, links, (size_t)4 * g.V * 9 * eb, st));
  WMG_TRY(stage_in(sc, clover, (size_t)g.V * 72 * eb, st));
  WMG_TRY(stage_out_alloc(so, out, fbytes, st));
  WMG_TRY(dslash_launch(dtype, so.dev, si.dev, sl.dev, g, -1, dagger, nrhs, st, 0, 0));
  if (dtype == MG_C128)
    WMG_TRY(clover_add<double>((zd*)so.dev, (const zd*)si.dev, (const zd*)sc.dev, g.V, nrhs, st));
  else
    WMG_TRY(clover_add<float>((zf*)so.dev, (const zf*)si.dev, (const zf*)sc.dev, g.V, nrhs, st));
  WMG_TRY(stage_out_finish(so, out, fbytes, st));
  return MG_OK;
}
