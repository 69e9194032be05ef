// Restriction R = P^dag, prolongation, the Galerkin coarse operator D_c = P^dag D P
// (Eq. 5) and its application.
//
// P is kept as the final iCSVD tiles: P[t][i][row], t = 2 j + alpha, M = 6 n_d rows.
// D_c is a coarse nearest-neighbour stencil stored per coarse site as 9 column-major
// (2k)x(2k) blocks: blk 0 = X (self), blk 1 + dir = Y_dir, dir = 2 mu + (0: +mu, 1: -mu).
//
// Galerkin assembly: CTA (j, mu) walks the n_d fine sites x of aggregate j; for each,
// the forward hop x -> x + mu of D applied to the 2k columns of P at the neighbour is
// reduced to a 6 x 2k half-spinor block chi (spin projection, colour transport), P(x)
// is folded with the matching reconstruction into a 6 x 2k block Ptil, and
// Ptil^dag chi is accumulated in FP64 -- into Y_+mu(j) if the hop leaves the
// aggregate, else into a per-direction partial of X(j).  Backward hops are not
// computed: gamma_5 D gamma_5 = D^dag and gamma_5 P = P sigma_3 make each backward
// contribution sigma_3 C^dag sigma_3 of a forward one C (exactly, up to rounding), which
// halves the FP64 work.  A second kernel adds the diagonal term P_j^dag P_j and the
// mirrored blocks in a fixed order.
#include <type_traits>

#include "common.cuh"
#include "df64.cuh"
#include "galerkin.cuh"
#include "internal.h"

namespace wmg {

namespace {

template <typename R>
__global__ void __launch_bounds__(256)
restrict_kernel(cplx<R>* vc, const cplx<R>* __restrict__ v, const cplx<R>* __restrict__ P,
                int k, Blocking B) {
  dep_entry();
  extern __shared__ unsigned char smraw[];
  cplx<R>* sv = reinterpret_cast<cplx<R>*>(smraw);
  int t = blockIdx.x, rhs = blockIdx.y;
  int j = t >> 1, alpha = t & 1;
  size_t V = (size_t)B.nd * B.d;
  const cplx<R>* vr = v + (size_t)rhs * V * 12;
  for (int row = threadIdx.x; row < B.M; row += blockDim.x) {
    int l = row / 6, sp = (row / 3) & 1, c = row % 3;
    int s = B.site(j, l);
    sv[row] = vr[(size_t)s * 12 + (2 * alpha + sp) * 3 + c];
  }
  __syncthreads();
  // warp work items (column i, half h of the rows): 2k items spread evenly over the warps
  // (k = 12: three per warp), each lane with two independent accumulators; the two halves of
  // a column meet in shared memory
  cplx<R>* sred = sv + B.M;   // [2k]
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const cplx<R>* Pt = P + (size_t)t * k * B.M;
  const int half_rows = (B.M + 1) / 2;
  for (int it = wid; it < 2 * k; it += nw) {
    const int i = it >> 1, r0 = (it & 1) * half_rows;
    const int r1 = min(B.M, r0 + half_rows);
    const cplx<R>* col = Pt + (size_t)i * B.M;
    cplx<R> a0 = {0, 0}, a1 = {0, 0};
    int row = r0 + lane;
    for (; row + 32 < r1; row += 64) {
      cfmac(a0, col[row], sv[row]);
      cfmac(a1, col[row + 32], sv[row + 32]);
    }
    for (; row < r1; row += 32) cfmac(a0, col[row], sv[row]);
    a0 += a1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0.re += __shfl_down_sync(0xffffffffu, a0.re, o);
      a0.im += __shfl_down_sync(0xffffffffu, a0.im, o);
    }
    if (lane == 0) sred[it] = a0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    vc[(size_t)rhs * B.d * 2 * k + (size_t)t * k + i] = sred[2 * i] + sred[2 * i + 1];
}

template <typename R>
__global__ void prolong_kernel(cplx<R>* v, const cplx<R>* __restrict__ vc,
                               const cplx<R>* __restrict__ P, int k, Blocking B, size_t total) {
  dep_entry();
  size_t V12 = (size_t)B.nd * B.d * 12;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t rhs = e / V12, rem = e % V12;
    int s = (int)(rem / 12), comp = (int)(rem % 12);
    int spin = comp / 3, c = comp % 3;
    int j, l;
    B.block_of(s, &j, &l);
    int t = 2 * j + (spin >> 1);
    int row = (l * 2 + (spin & 1)) * 3 + c;
    const cplx<R>* Pt = P + (size_t)t * k * B.M + row;
    const cplx<R>* cv = vc + rhs * B.d * 2 * k + (size_t)t * k;
    cplx<R> acc = {0, 0};
    for (int i = 0; i < k; ++i) cfma(acc, Pt[(size_t)i * B.M], cv[i]);
    v[e] = acc;
  }
}


// (i sigma_mu psi)[s] for a 2-spinor given by its two components: returns component s.
__device__ __forceinline__ zd isigma(int mu, int s, zd p0, zd p1) {
  if (mu == 0) return s == 0 ? ti(p1) : ti(p0);
  if (mu == 1) return s == 0 ? p1 : -p0;
  return s == 0 ? ti(p0) : tmi(p1);
}

constexpr int GTH = 256;     // threads
constexpr int GMAXE = 16;    // accumulator entries per thread ((2k)^2 <= 4096)


// Forward hops x -> y = x + mu of D = 1 - kappa sum_mu w_mu [(1 - gamma_mu) U_mu(x) delta_{x+mu}
// + ...]: the spin projector (1 - gamma_mu) reduces the 2k columns of P at y to a half
// spinor (2 spins x 3 colours), U_mu(x) transports its colour, and the reconstruction folds
// into P(x).  Staged per fine site h and half-spinor row r (6 rows):
//   sCh[h][r][b] = +-(U P_b(y))_r   (sign -1 for an antiperiodic wrapping hop)
//   sPt[h][r][a] = (L P_a(x))_r     (L = reconstruction adjoint)
// and every block accumulates sum_{h,r} conj(sPt[h][r][a]) sCh[h][r][b]; the factor
// -kappa w_mu multiplies the finished block.  DF: P, links, staging and accumulation in
// double-float on the FP32 units (P and links pre-split into (hi, lo) pairs); otherwise FP64.
// NE: accumulator entries per thread (ceil((2k)^2 / GTH), rounded up to a launched size).
template <bool DF, int NE>
__global__ void __launch_bounds__(GTH)
galerkin_hop_kernel(zd* Op, zd* Xpart, const zd* __restrict__ P, const zdf* __restrict__ Pdf,
                    int k, const zd* __restrict__ links, const zdf* __restrict__ Ldf, HopGeom g,
                    Blocking B) {
  typedef typename std::conditional<DF, zdf, zd>::type T;
  typedef typename std::conditional<DF, zdfacc, zd>::type TA;
  extern __shared__ zd gsm_raw[];
  T* gsm = reinterpret_cast<T*>(gsm_raw);
  int n2k = 2 * k;
  T* sPt = gsm;                        // [GNB][6][n2k]
  T* sCh = gsm + GNB * 6 * n2k;        // [GNB][6][n2k]
  __shared__ int ssite[GNB], snb[GNB], sneg[GNB];
  __shared__ size_t sox[GNB], soy[GNB];   // tile offsets (chirality 0, column 0) of x and y
  __shared__ int slx[GNB], sly[GNB];      // local site of x and y in their aggregates
  int j = blockIdx.x, mu = blockIdx.y, dir = 2 * mu;
  double coef = -g.kappa * g.w[mu];
  int ne = n2k * n2k;
  int bmu = B.b[mu];
  const int* bb = B.b;
  size_t V = (size_t)B.nd * B.d;
  for (int pass = 0; pass < 2; ++pass) {  // 0: hops inside the aggregate, 1: crossing hops
    TA acc[NE];
#pragma unroll
    for (int q = 0; q < NE; ++q) acc[q] = TA{};
    int l = 0;
    while (true) {
      // collect the next batch of local sites of this pass (same scan in every thread)
      int nb = 0;
      int lsel[GNB];
      while (l < B.nd && nb < GNB) {
        int lm;
        {
          int q = l;
          int lc[4];
          lc[0] = q % bb[0]; q /= bb[0];
          lc[1] = q % bb[1]; q /= bb[1];
          lc[2] = q % bb[2]; lc[3] = q / bb[2];
          lm = lc[mu];
        }
        bool cross = lm == bmu - 1;
        if ((pass == 1) == cross) lsel[nb++] = l;
        ++l;
      }
      if (nb == 0) break;
      __syncthreads();
      if (threadIdx.x < nb) {
        int x = B.site(j, lsel[threadIdx.x]);
        int c[4];
        c[0] = x % g.L[0];
        int r = x / g.L[0];
        c[1] = r % g.L[1]; r /= g.L[1];
        c[2] = r % g.L[2]; c[3] = r / g.L[2];
        bool wrap = c[mu] == g.L[mu] - 1;
        int y = wrap ? x - (g.L[mu] - 1) * g.stride[mu] : x + g.stride[mu];
        ssite[threadIdx.x] = x;
        snb[threadIdx.x] = y;
        sneg[threadIdx.x] = (wrap && g.bc[mu] < 0) ? 1 : 0;
        int jy, ly, jx, lx;
        B.block_of(y, &jy, &ly);
        B.block_of(x, &jx, &lx);
        soy[threadIdx.x] = (size_t)(2 * jy) * k * B.M;
        sox[threadIdx.x] = (size_t)(2 * jx) * k * B.M;
        sly[threadIdx.x] = ly;
        slx[threadIdx.x] = lx;
      }
      __syncthreads();
      // stage chi and Ptil
      for (int e = threadIdx.x; e < nb * 6 * n2k; e += GTH) {
        int h = e / (6 * n2k);
        int r = (e / n2k) % 6;
        int bcol = e % n2k;
        int s = r / 3, cc = r % 3;
        int beta = bcol / k;
        int x = ssite[h];
        int ly = sly[h], lx = slx[h];
        // column bcol = beta k + i of the tile pair (chirality beta follows chirality 0)
        size_t oy = soy[h] + (size_t)bcol * B.M;
        size_t ox = sox[h] + (size_t)bcol * B.M;
        if constexpr (DF) {
          // half spinor of column bcol at y: chirality 0 keeps spin s of the upper pair;
          // chirality 1 gives i sigma_mu psi_dn (mu < 3) or -psi_dn (mu = 3)
          zdf hv[3];
#pragma unroll
          for (int c2 = 0; c2 < 3; ++c2) {
            if (beta == 0) {
              hv[c2] = zdf_ld(Pdf + oy + (ly * 2 + s) * 3 + c2);
            } else {
              zdf p0 = zdf_ld(Pdf + oy + (ly * 2 + 0) * 3 + c2);
              zdf p1 = zdf_ld(Pdf + oy + (ly * 2 + 1) * 3 + c2);
              hv[c2] = mu < 3 ? isigma_df(mu, s, p0, p1) : zdf_neg(s == 0 ? p0 : p1);
            }
          }
          const zdf* U = Ldf + ((size_t)mu * V + x) * 9 + cc * 3;
          zdfacc t{};
#pragma unroll
          for (int c2 = 0; c2 < 3; ++c2) zdf_fma(t, zdf_ld(U + c2), hv[c2]);
          zdf ch = zdf_norm(t);
          sCh[(h * 6 + r) * n2k + bcol] = sneg[h] ? zdf_neg(ch) : ch;
          zdf pt;
          if (beta == 0) {
            pt = zdf_ld(Pdf + ox + (lx * 2 + s) * 3 + cc);
          } else {
            zdf p0 = zdf_ld(Pdf + ox + (lx * 2 + 0) * 3 + cc);
            zdf p1 = zdf_ld(Pdf + ox + (lx * 2 + 1) * 3 + cc);
            pt = mu < 3 ? isigma_df(mu, s, p0, p1) : zdf_neg(s == 0 ? p0 : p1);
          }
          sPt[(h * 6 + r) * n2k + bcol] = pt;
        } else {
          const zd* Py = P + oy;
          zd hv[3];
#pragma unroll
          for (int c2 = 0; c2 < 3; ++c2) {
            if (beta == 0) {
              hv[c2] = Py[(ly * 2 + s) * 3 + c2];
            } else {
              zd p0 = Py[(ly * 2 + 0) * 3 + c2], p1 = Py[(ly * 2 + 1) * 3 + c2];
              hv[c2] = mu < 3 ? isigma(mu, s, p0, p1) : -(s == 0 ? p0 : p1);
            }
          }
          const zd* U = links + ((size_t)mu * V + x) * 9;
          zd ch = {0, 0};
#pragma unroll
          for (int c2 = 0; c2 < 3; ++c2) cfma(ch, U[cc * 3 + c2], hv[c2]);
          sCh[(h * 6 + r) * n2k + bcol] = sneg[h] ? -ch : ch;
          const zd* Px = P + ox;
          zd pt;
          if (beta == 0) {
            pt = Px[(lx * 2 + s) * 3 + cc];
          } else {
            zd p0 = Px[(lx * 2 + 0) * 3 + cc], p1 = Px[(lx * 2 + 1) * 3 + cc];
            pt = mu < 3 ? isigma(mu, s, p0, p1) : -(s == 0 ? p0 : p1);
          }
          sPt[(h * 6 + r) * n2k + bcol] = pt;
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < NE; ++q) {
        int e = threadIdx.x + q * GTH;
        if (e < ne) {
          int a = e / n2k, b = e % n2k;
          TA t = acc[q];
          for (int h = 0; h < nb; ++h)
#pragma unroll
            for (int r = 0; r < 6; ++r)
            {
              if constexpr (DF) zdf_fmac(t, sPt[(h * 6 + r) * n2k + a], sCh[(h * 6 + r) * n2k + b]);
              else cfmac(t, sPt[(h * 6 + r) * n2k + a], sCh[(h * 6 + r) * n2k + b]);
            }
          acc[q] = t;
        }
      }
    }
    zd* out = pass == 1 ? Op + ((size_t)j * 9 + 1 + dir) * ne
                        : Xpart + ((size_t)mu * B.d + j) * ne;
#pragma unroll
    for (int q = 0; q < NE; ++q) {
      int e = threadIdx.x + q * GTH;
      if (e < ne) {
        int a = e / n2k, b = e % n2k;
        zd v;
        if constexpr (DF) v = zdf_result(acc[q]);
        else v = acc[q];
        out[(size_t)b * n2k + a] = coef * v;   // column-major
      }
    }
    __syncthreads();
  }
}

// complex double -> (hi, lo) float pairs
__global__ void to_df_kernel(zdf* out, const zd* __restrict__ in, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    zdf v = zdf_from(in[i]);
    reinterpret_cast<float4*>(out)[i] = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo);
  }
}

// Completes D_c from the forward hops.  gamma_5-hermiticity of D with gamma_5 P = P sigma_3
// gives, hop by hop, backward contribution = sigma_3 (forward contribution)^dag sigma_3, so
//   X(j)      = P_j^dag P_j + sum_mu [F_mu(j) + sigma_3 F_mu(j)^dag sigma_3]
//   Y_-mu(j)  = sigma_3 Y_+mu(j - mu)^dag sigma_3
// with F_mu(j) the forward hops that stay inside aggregate j.  Element (a, b) of
// sigma_3 M^dag sigma_3 is s_a s_b conj(M(b, a)), s = +1 / -1 for chirality 0 / 1.
__global__ void __launch_bounds__(GTH)
galerkin_finish_kernel(zd* Op, const zd* __restrict__ Xpart, const zd* __restrict__ PtP, int k,
                       Blocking B) {
  int j = blockIdx.x;
  int n2k = 2 * k, ne = n2k * n2k;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    int b = e / n2k, a = e % n2k;  // column-major element (a, b)
    int et = a * n2k + b;          // element (b, a)
    int aa = a / k, bb = b / k;
    double sab = (aa == bb) ? 1.0 : -1.0;
    zd acc = {0, 0};
    if (aa == bb) acc = PtP[((size_t)(2 * j + aa) * k + a % k) * k + b % k];   // P_a^dag P_b
    for (int mu = 0; mu < 4; ++mu) {
      const zd* F = Xpart + ((size_t)mu * B.d + j) * ne;
      acc += F[e];
      acc += sab * conj(F[et]);
      int jm = B.coarse_nbr(j, 2 * mu + 1);
      zd yv = Op[((size_t)jm * 9 + 1 + 2 * mu) * ne + et];
      Op[((size_t)j * 9 + 2 + 2 * mu) * ne + e] = sab * conj(yv);
    }
    Op[(size_t)j * 9 * ne + e] = acc;
  }
}

// y(j) = sum_blk Op[j][blk] x(src(blk)).  One CTA per (coarse site, rhs) with 9 x 2k
// threads: thread (blk, a) stages x(src(blk))[a] in shared memory, forms row a of
// block blk times that vector (column-major blocks: coalesced over a), and the nine
// partial rows are summed in a fixed order.
template <typename R>
__global__ void __launch_bounds__(576)
coarse_apply_kernel(cplx<R>* y, const cplx<R>* __restrict__ x, const cplx<R>* __restrict__ Op,
                    int n2k, Blocking B) {
  dep_entry();
  extern __shared__ unsigned char csm[];
  cplx<R>* sx = reinterpret_cast<cplx<R>*>(csm);     // [9][n2k]
  cplx<R>* sp = sx + 9 * n2k;                         // [9][n2k] partial rows
  int j = blockIdx.x, rhs = blockIdx.y;
  int blk = threadIdx.x / n2k, a = threadIdx.x % n2k;
  size_t nc = (size_t)B.d * n2k;
  const cplx<R>* xr = x + (size_t)rhs * nc;
  int src = blk == 0 ? j : B.coarse_nbr(j, blk - 1);
  sx[threadIdx.x] = xr[(size_t)src * n2k + a];
  __syncthreads();
  const cplx<R>* O = Op + ((size_t)j * 9 + blk) * n2k * n2k + a;
  const cplx<R>* xs = sx + blk * n2k;
  cplx<R> acc = {0, 0};
  for (int b = 0; b < n2k; ++b) cfma(acc, O[(size_t)b * n2k], xs[b]);
  sp[threadIdx.x] = acc;
  __syncthreads();
  if (blk == 0) {
    cplx<R> t = sp[a];
#pragma unroll
    for (int q = 1; q < 9; ++q) t += sp[q * n2k + a];
    y[(size_t)rhs * nc + (size_t)j * n2k + a] = t;
  }
}

}  // namespace

template <typename R>
int restrict_launch(cplx<R>* vc, const cplx<R>* v, const cplx<R>* P, int k, const Blocking& B,
                    int nrhs, cudaStream_t st) {
  dim3 grid(B.d * 2, nrhs);
  size_t sh = sizeof(cplx<R>) * (B.M + 2 * k);   // v's aggregate rows, half-column sums
  if (sh > 200 * 1024) return fail(MG_EINVAL, "restrict: aggregate too large");
  WMG_TRY(smem_attr(restrict_kernel<R>, sh));
  ProfScope ps("restrict", (double)sizeof(cplx<R>) * (12.0 * B.nd * B.d * (k + nrhs) + 2.0 * B.d * k * nrhs),
               8.0 * 12 * B.nd * B.d * k * nrhs, st);
  WMG_LAUNCH_DEP(restrict_kernel<R>, grid, 256, sh, st, vc, v, P, k, B);
  return MG_OK;
}

template <typename R>
int prolong_launch(cplx<R>* v, const cplx<R>* vc, const cplx<R>* P, int k, const Blocking& B,
                   int nrhs, cudaStream_t st) {
  size_t total = (size_t)nrhs * B.nd * B.d * 12;
  size_t gsz = (total + 255) / 256;
  size_t cap = (size_t)num_sms() * 16;
  ProfScope ps("prolong", (double)sizeof(cplx<R>) * (12.0 * B.nd * B.d * (k + nrhs) + 2.0 * B.d * k * nrhs),
               8.0 * 12 * B.nd * B.d * k * nrhs, st);
  WMG_LAUNCH_DEP(prolong_kernel<R>, (unsigned)(gsz < cap ? gsz : cap), 256, 0, st, v, vc, P, k, B, total);
  return MG_OK;
}

int to_df(zdf* out, const zd* in, size_t n, cudaStream_t st) {
  size_t g = (n + 255) / 256, cap = (size_t)num_sms() * 16;
  to_df_kernel<<<(unsigned)(g < cap ? (g < 1 ? 1 : g) : cap), 256, 0, st>>>(out, in, n);
  WMG_LAUNCHED();
  return MG_OK;
}

namespace {
template <bool DF, int NE>
int launch_hop(dim3 grid, size_t sh, cudaStream_t st, zd* Op, zd* Xpart, const zd* P,
               const zdf* Pdf, int k, const zd* links, const zdf* Ldf, const HopGeom& hg,
               const Blocking& B) {
  WMG_TRY(smem_attr(galerkin_hop_kernel<DF, NE>, sh));
  galerkin_hop_kernel<DF, NE><<<grid, GTH, sh, st>>>(Op, Xpart, P, Pdf, k, links, Ldf, hg, B);
  WMG_LAUNCHED();
  return MG_OK;
}

template <bool DF>
int launch_hop_ne(dim3 grid, size_t sh, cudaStream_t st, zd* Op, zd* Xpart, const zd* P,
                  const zdf* Pdf, int k, const zd* links, const zdf* Ldf, const HopGeom& hg,
                  const Blocking& B) {
  int ne = (4 * k * k + GTH - 1) / GTH;
  if (ne <= 2) return launch_hop<DF, 2>(grid, sh, st, Op, Xpart, P, Pdf, k, links, Ldf, hg, B);
  if (ne <= 4) return launch_hop<DF, 4>(grid, sh, st, Op, Xpart, P, Pdf, k, links, Ldf, hg, B);
  if (ne <= 8) return launch_hop<DF, 8>(grid, sh, st, Op, Xpart, P, Pdf, k, links, Ldf, hg, B);
  if (ne <= 12) return launch_hop<DF, 12>(grid, sh, st, Op, Xpart, P, Pdf, k, links, Ldf, hg, B);
  return launch_hop<DF, 16>(grid, sh, st, Op, Xpart, P, Pdf, k, links, Ldf, hg, B);
}
}  // namespace

int galerkin_build(zd* Op, zd* Xpart, const zd* P, zdf* Pdf, zd* PtP, int k, const zd* links,
                   const zdf* Ldf, const Geom& g, const Blocking& B, cudaStream_t st, bool df64,
                   bool pdf_ready, int* range_flag) {
  if (4 * k * k > GTH * GMAXE) return fail(MG_EINVAL, "galerkin: k > 32");
  if (df64 && (!Pdf || !Ldf)) return fail(MG_EINVAL, "galerkin: double-float copies missing");
  HopGeom hg;
  for (int m = 0; m < 4; ++m) {
    hg.L[m] = g.L[m];
    hg.w[m] = g.w[m];
    hg.bc[m] = g.bc[m];
  }
  hg.stride[0] = 1;
  hg.stride[1] = g.L[0];
  hg.stride[2] = g.L[0] * g.L[1];
  hg.stride[3] = g.L[0] * g.L[1] * g.L[2];
  hg.kappa = g.kappa;
  size_t sh = sizeof(zd) * 2 * GNB * 6 * 2 * k;
  dim3 grid(B.d, 4);
  // diagonal term P_j^dag P_j: the Gram matrix of every P tile (profiled as a Gram launch)
  if (df64) {
    if (!pdf_ready) WMG_TRY(to_df(Pdf, P, (size_t)B.d * 2 * k * B.M, st));
    WMG_TRY(tile_gram(PtP, Pdf, k, k, B, st, true));
  } else {
    WMG_TRY(tile_gram(PtP, P, k, k, B, st, false));
  }
  const bool tc = df64 && galerkin_tc_supported(k, B);
  // flops: the method's work, 768 k^2 FP64-equivalent flops per fine site (4 forward hops x
  // 6 rows x (2k)^2 complex multiply-adds); the tensor path also records the bf16 digit-plane
  // products it issues for them
  if (tc && !range_flag) return fail(MG_EINVAL, "galerkin: no range flag");
  int tc_nb = 0;
  if (tc) WMG_TRY(galerkin_tc_batch(&tc_nb, Op, Xpart, Pdf, k, Ldf, hg, B, range_flag, st));
  const double tc_flops = tc ? galerkin_tc_issued_flops(k, B, tc_nb) : 0.0;
  ProfScope ps(tc ? "galerkin_tc" : df64 ? "galerkin_df64" : "galerkin_fp64",
               16.0 * (12.0 * B.nd * B.d * k * 5 + 36.0 * B.nd * B.d),
               768.0 * k * k * B.nd * B.d, tc ? tc_flops : 0.0, st);
  if (tc) {
    // tensor pipe (exact digit-plane products); entries outside its fixed-point range (links
    // that are not unitary, a prolongator that is not orthonormal) fall back to the FP32 units
    int* flag = range_flag;
    WMG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    WMG_TRY(galerkin_hops_tc(Op, Xpart, Pdf, k, Ldf, hg, B, tc_nb, flag, st));
    int h_flag = 0;
    WMG_CUDA(cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    WMG_CUDA(cudaStreamSynchronize(st));
    if (h_flag) {
      ProfScope pf("galerkin_tc_range_fallback", 0.0, 0.0, st);
      WMG_TRY(launch_hop_ne<true>(grid, sh, st, Op, Xpart, P, Pdf, k, links, Ldf, hg, B));
    }
  } else if (df64) {
    WMG_TRY(launch_hop_ne<true>(grid, sh, st, Op, Xpart, P, Pdf, k, links, Ldf, hg, B));
  } else {
    WMG_TRY(launch_hop_ne<false>(grid, sh, st, Op, Xpart, P, Pdf, k, links, Ldf, hg, B));
  }
  galerkin_finish_kernel<<<B.d, GTH, 0, st>>>(Op, Xpart, PtP, k, B);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int coarse_apply_launch(cplx<R>* y, const cplx<R>* x, const cplx<R>* Op, int k, const Blocking& B,
                        int nrhs, cudaStream_t st) {
  if (2 * k > 64) return fail(MG_EINVAL, "coarse_apply: 2k > 64");
  dim3 grid(B.d, nrhs);
  size_t sh = sizeof(cplx<R>) * 18 * 2 * k;
  ProfScope ps("coarse_apply", (double)sizeof(cplx<R>) * B.d * (9.0 * 4 * k * k + 4.0 * k * nrhs),
               8.0 * 9 * 4 * k * k * B.d * nrhs, st);
  WMG_LAUNCH_DEP(coarse_apply_kernel<R>, grid, 9 * 2 * k, sh, st, y, x, Op, 2 * k, B);
  return MG_OK;
}

template int restrict_launch<float>(zf*, const zf*, const zf*, int, const Blocking&, int, cudaStream_t);
template int restrict_launch<double>(zd*, const zd*, const zd*, int, const Blocking&, int, cudaStream_t);
template int prolong_launch<float>(zf*, const zf*, const zf*, int, const Blocking&, int, cudaStream_t);
template int prolong_launch<double>(zd*, const zd*, const zd*, int, const Blocking&, int, cudaStream_t);
template int coarse_apply_launch<float>(zf*, const zf*, const zf*, int, const Blocking&, int, cudaStream_t);
template int coarse_apply_launch<double>(zd*, const zd*, const zd*, int, const Blocking&, int, cudaStream_t);

}  // namespace wmg
