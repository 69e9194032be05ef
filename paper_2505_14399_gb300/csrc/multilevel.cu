// Deeper levels of the hierarchy (Sec. 2.1 end, Algorithm 4, Sec. 4): the Galerkin operator
// of Eq. 5 takes the place of D on the next level, with sigma_3 as its chirality
// (gamma_5 P = P sigma_3), and the same setup -- test vectors by smoothing, chiral split,
// streaming SVD -- and Galerkin product build the level below it.
//
// A level-l operator (l >= 1) is a nearest-neighbour stencil on its lattice: blocks X(j) and
// Y_dir(j), dir = 2 mu + (0: +mu, 1: -mu), each n x n (n = 2 k_l, entries ordered
// (chirality alpha, i)), stored [j][9][col][row] (column-major blocks, X first) -- the layout
// of the level-1 operator.  Aggregates of a coarse lattice are blocks of its sites,
// lexicographic inside and across (Blocking, with M = n_d k_l rows per tile: row = l k_l + i
// for local site l and component i of chirality alpha).
//
// Kernels here: the chiral split of coarse vectors into tiles, restriction and prolongation
// between level l and l + 1, and the Galerkin product of a coarse stencil.  The SVD of the
// tiles is the fine level's (chiral_svd.cu); the solves run the Krylov engine on
// coarse_apply_launch.
#include <type_traits>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"

namespace wmg {
namespace {

unsigned grid_for(size_t n) {
  size_t g = (n + 255) / 256, cap = (size_t)num_sms() * 16;
  return (unsigned)(g < cap ? (g < 1 ? 1 : g) : cap);
}

// tiles[(t cmax + col0 + v) M + l k + i] = f[v][s][alpha k + i], t = 2 J + alpha, (J, l) the
// aggregate and local index of site s
template <typename R, typename TO>
__global__ void cgather_kernel(TO* tiles, int cmax, int col0, const cplx<R>* __restrict__ f,
                               int nvec, Blocking B, int k) {
  const int Ld = B.L[0] * B.L[1] * B.L[2] * B.L[3];
  const size_t per = (size_t)Ld * 2 * k;
  const size_t total = (size_t)nvec * per;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int v = (int)(e / per);
    size_t rem = e % per;
    int s = (int)(rem / (2 * k)), c = (int)(rem % (2 * k));
    int alpha = c / k, i = c % k;
    int J, l;
    B.block_of(s, &J, &l);
    size_t t = (size_t)J * 2 + alpha;
    cplx<R> x = f[e];
    size_t o = (t * cmax + col0 + v) * B.M + (size_t)l * k + i;
    if constexpr (std::is_same<TO, zdf>::value) tiles[o] = zdf_from(x);
    else tiles[o] = {(double)x.re, (double)x.im};
  }
}

// vc[rhs][J][alpha][i'] = sum_{l, i} conj(P[2J + alpha][i'][l k + i]) v[rhs][site(J, l)][alpha][i]
template <typename R>
__global__ void crestrict_kernel(cplx<R>* vc, const cplx<R>* __restrict__ v,
                                 const cplx<R>* __restrict__ P, Blocking B, int k, int kp,
                                 int nrhs) {
  const size_t nout = (size_t)B.d * 2 * kp;
  const size_t nin = (size_t)B.d * B.nd * 2 * k;
  const size_t total = (size_t)nrhs * nout;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t rhs = e / nout, rem = e % nout;
    int J = (int)(rem / (2 * kp)), c = (int)(rem % (2 * kp));
    int alpha = c / kp, ip = c % kp;
    const cplx<R>* Pc = P + (((size_t)J * 2 + alpha) * kp + ip) * B.M;
    const cplx<R>* vr = v + rhs * nin;
    cplx<R> acc = {0, 0};
    for (int l = 0; l < B.nd; ++l) {
      const cplx<R>* vs = vr + (size_t)B.site(J, l) * 2 * k + alpha * k;
      for (int i = 0; i < k; ++i) cfmac(acc, Pc[(size_t)l * k + i], vs[i]);
    }
    vc[e] = acc;
  }
}

// v[rhs][s][alpha][i] = sum_{i'} P[2J + alpha][i'][l k + i] vc[rhs][J][alpha][i']
template <typename R>
__global__ void cprolong_kernel(cplx<R>* v, const cplx<R>* __restrict__ vc,
                                const cplx<R>* __restrict__ P, Blocking B, int k, int kp,
                                int nrhs) {
  const size_t nout = (size_t)B.d * B.nd * 2 * k;
  const size_t nin = (size_t)B.d * 2 * kp;
  const size_t total = (size_t)nrhs * nout;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t rhs = e / nout, rem = e % nout;
    int s = (int)(rem / (2 * k)), c = (int)(rem % (2 * k));
    int alpha = c / k, i = c % k;
    int J, l;
    B.block_of(s, &J, &l);
    const cplx<R>* Pc = P + ((size_t)J * 2 + alpha) * kp * B.M + (size_t)l * k + i;
    const cplx<R>* xr = vc + rhs * nin + (size_t)J * 2 * kp + alpha * kp;
    cplx<R> acc = {0, 0};
    for (int ip = 0; ip < kp; ++ip) cfma(acc, Pc[(size_t)ip * B.M], xr[ip]);
    v[e] = acc;
  }
}

// local coordinate of site s inside its aggregate along mu, and whether the hop dir leaves it
__device__ __forceinline__ bool hop_leaves(const Blocking& B, int s, int dir) {
  int c[4];
  c[0] = s % B.L[0];
  int r = s / B.L[0];
  c[1] = r % B.L[1];
  r /= B.L[1];
  c[2] = r % B.L[2];
  c[3] = r / B.L[2];
  int mu = dir >> 1;
  int lc = c[mu] % B.b[mu];
  return (dir & 1) ? lc == 0 : lc == B.b[mu] - 1;
}

// neighbour of site s on the level-l lattice B.L in direction dir (periodic)
__device__ __forceinline__ int lat_nbr(const Blocking& B, int s, int dir) {
  int c[4];
  c[0] = s % B.L[0];
  int r = s / B.L[0];
  c[1] = r % B.L[1];
  r /= B.L[1];
  c[2] = r % B.L[2];
  c[3] = r / B.L[2];
  int mu = dir >> 1;
  c[mu] = (dir & 1) ? (c[mu] + B.L[mu] - 1) % B.L[mu] : (c[mu] + 1) % B.L[mu];
  return c[0] + B.L[0] * (c[1] + B.L[1] * (c[2] + B.L[2] * c[3]));
}

constexpr int GC_T = 256;

// One CTA per (aggregate J, target block tb): tb = 0 collects P(j)^dag X(j) P(j) and the hops
// that stay inside J, tb = 1 + dir the hops dir that leave J (Eq. 5 term by term), member
// sites in local order and sources in a fixed order (deterministic).  P(j) is the site
// restriction of P, block diagonal in the chirality: P(j)[(alpha, i)][(alpha, i')] =
// P[2J + alpha][i'][l k + i].  Shared memory: T = B_src P(j') (n x n'), the two site blocks
// of P, and the n' x n' accumulator.
__global__ void __launch_bounds__(GC_T)
cgalerkin_kernel(zd* Op2, const zd* __restrict__ Op, const zd* __restrict__ P, Blocking B, int k,
                 int kp) {
  extern __shared__ zd gsm[];
  const int n = 2 * k, np = 2 * kp;
  zd* T = gsm;                    // [np][n]   T[b'][a] = (B_src P(j'))[a][b']
  zd* Pa = T + (size_t)np * n;    // [2][kp][k]  P(j) blocks: Pa[(alpha kp + i') k + i]
  zd* Pb = Pa + (size_t)2 * kp * k;   // P(j') blocks
  zd* C = Pb + (size_t)2 * kp * k;    // [np][np] column-major accumulator C[b'][a']
  const int J = blockIdx.x, tb = blockIdx.y;
  for (int e = threadIdx.x; e < np * np; e += GC_T) C[e] = {0, 0};
  for (int l = 0; l < B.nd; ++l) {
    const int j = B.site(J, l);
    // sources of this target at site j: (block index in Op, neighbour site)
    for (int q = 0; q < 9; ++q) {
      int blk, jn;
      if (tb == 0) {
        if (q == 0) { blk = 0; jn = j; }
        else {
          if (hop_leaves(B, j, q - 1)) continue;
          blk = q;
          jn = lat_nbr(B, j, q - 1);
        }
      } else {
        if (q > 0) break;
        if (!hop_leaves(B, j, tb - 1)) break;
        blk = tb;
        jn = lat_nbr(B, j, tb - 1);
      }
      int Jn, ln;
      B.block_of(jn, &Jn, &ln);
      __syncthreads();
      for (int e = threadIdx.x; e < 2 * kp * k; e += GC_T) {
        int ai = e / k, i = e % k;   // ai = alpha kp + i'
        int alpha = ai / kp, ip = ai % kp;
        Pa[e] = P[(((size_t)J * 2 + alpha) * kp + ip) * B.M + (size_t)l * k + i];
        Pb[e] = P[(((size_t)Jn * 2 + alpha) * kp + ip) * B.M + (size_t)ln * k + i];
      }
      __syncthreads();
      // T[(alpha', i')][a] = sum_m Bsrc[a][(alpha', m)] Pb[alpha'][i'][m]
      const zd* Bs = Op + ((size_t)j * 9 + blk) * n * n;   // Bs[col * n + row]
      for (int e = threadIdx.x; e < np * n; e += GC_T) {
        int bp = e / n, a = e % n;
        int alpha = bp / kp;
        const zd* pb = Pb + (size_t)bp * k;
        zd acc = {0, 0};
        for (int m = 0; m < k; ++m) cfma(acc, Bs[(size_t)(alpha * k + m) * n + a], pb[m]);
        T[e] = acc;
      }
      __syncthreads();
      // C[(alpha', i')][(alpha, i'')] += sum_i conj(Pa[alpha][i''][i]) T[(alpha', i')][(alpha, i)]
      for (int e = threadIdx.x; e < np * np; e += GC_T) {
        int bp = e / np, ap = e % np;
        int alpha = ap / kp;
        const zd* pa = Pa + (size_t)ap * k;
        const zd* tt = T + (size_t)bp * n + alpha * k;
        zd acc = C[e];
        for (int i = 0; i < k; ++i) cfmac(acc, pa[i], tt[i]);
        C[e] = acc;
      }
    }
  }
  __syncthreads();
  zd* out = Op2 + ((size_t)J * 9 + tb) * np * np;
  for (int e = threadIdx.x; e < np * np; e += GC_T) out[e] = C[e];
}

}  // namespace

template <typename R>
int coarse_gather(void* tiles, int cmax, int col0, const cplx<R>* fields, int nvec,
                  const Blocking& B, int k, cudaStream_t st, bool df64) {
  size_t total = (size_t)nvec * B.d * B.nd * 2 * k;
  if (df64)
    cgather_kernel<R, zdf><<<grid_for(total), 256, 0, st>>>((zdf*)tiles, cmax, col0, fields, nvec, B, k);
  else
    cgather_kernel<R, zd><<<grid_for(total), 256, 0, st>>>((zd*)tiles, cmax, col0, fields, nvec, B, k);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int coarse_restrict(cplx<R>* vc, const cplx<R>* v, const cplx<R>* P, const Blocking& B, int k,
                    int kp, int nrhs, cudaStream_t st) {
  size_t total = (size_t)nrhs * B.d * 2 * kp;
  crestrict_kernel<R><<<grid_for(total), 256, 0, st>>>(vc, v, P, B, k, kp, nrhs);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int coarse_prolong(cplx<R>* v, const cplx<R>* vc, const cplx<R>* P, const Blocking& B, int k,
                   int kp, int nrhs, cudaStream_t st) {
  size_t total = (size_t)nrhs * B.d * B.nd * 2 * k;
  cprolong_kernel<R><<<grid_for(total), 256, 0, st>>>(v, vc, P, B, k, kp, nrhs);
  WMG_LAUNCHED();
  return MG_OK;
}

int coarse_galerkin(zd* Op2, const zd* Op, const zd* P, const Blocking& B, int k, int kp,
                    cudaStream_t st) {
  const size_t n = 2 * k, np = 2 * kp;
  size_t sh = sizeof(zd) * (np * n + 4 * (size_t)kp * k + np * np);
  if (sh > (size_t)220 * 1024) return fail(MG_EINVAL, "coarse Galerkin: k too large");
  WMG_TRY(smem_attr(cgalerkin_kernel, sh));
  ProfScope ps("galerkin_coarse_fp64", 16.0 * ((double)B.d * B.nd * 9 * n * n + 2.0 * B.d * kp * B.M),
               8.0 * B.d * B.nd * 9 * ((double)n * n * kp * 2 + (double)np * np * k), st);
  cgalerkin_kernel<<<dim3(B.d, 9), GC_T, sh, st>>>(Op2, Op, P, B, k, kp);
  WMG_LAUNCHED();
  return MG_OK;
}

template int coarse_gather<float>(void*, int, int, const zf*, int, const Blocking&, int, cudaStream_t, bool);
template int coarse_gather<double>(void*, int, int, const zd*, int, const Blocking&, int, cudaStream_t, bool);
template int coarse_restrict<float>(zf*, const zf*, const zf*, const Blocking&, int, int, int, cudaStream_t);
template int coarse_restrict<double>(zd*, const zd*, const zd*, const Blocking&, int, int, int, cudaStream_t);
template int coarse_prolong<float>(zf*, const zf*, const zf*, const Blocking&, int, int, int, cudaStream_t);
template int coarse_prolong<double>(zd*, const zd*, const zd*, const Blocking&, int, int, int, cudaStream_t);

}  // namespace wmg
