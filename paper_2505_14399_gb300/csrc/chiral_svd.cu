// Batched streaming chiral SVD (Algorithm 3, Eqs. 7-8) over all aggregates and both
// chiralities at once.
//
// Every (aggregate j, chirality alpha) owns a tile A = [Phi_{s-1} | Psi_s] of M = 6 n_d
// rows (Eq. 3 split) stored column-major in FP64, or in double-float (zdf, the same 16 bytes)
// when the sums run in double-float: those tiles then stay double-float from the gather to
// the final prolongator, so no kernel converts them on the FP64 units.  One stream is:
//   gather   : chiral split of the r new smoothed vectors into columns kk.. of all tiles
//   gram     : G = A^dag A (c x c Hermitian, c = kk + r), one CTA per tile
//   eig      : parallel cyclic Jacobi (Brent-Luk ordering) on G in shared memory,
//              eigenvalues sorted descending (ties by index) -> Sigma^2 and V
//   update   : Phi_s = A V_k (= U_k Sigma_k, Eq. 7), or U_k = A V_k Sigma_k^{-1} at the end
// An optional second pass (G of A V over all c columns, eig, rotate) restores the
// accuracy lost by forming A^dag A (its rotations are relative to sigma_i sigma_j).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"

namespace wmg {

namespace {

template <typename R, typename TO>
__global__ void gather_kernel(TO* tiles, int cmax, int col0, const cplx<R>* __restrict__ f,
                              int nvec, Blocking B) {
  size_t total = (size_t)nvec * B.L[0] * B.L[1] * B.L[2] * B.L[3] * 12;
  size_t V12 = total / nvec;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int v = (int)(e / V12);
    size_t rem = e % V12;
    int s = (int)(rem / 12), comp = (int)(rem % 12);
    int spin = comp / 3, col = comp % 3;
    int j, l;
    B.block_of(s, &j, &l);
    int alpha = spin >> 1;
    int row = (l * 2 + (spin & 1)) * 3 + col;
    size_t t = (size_t)j * 2 + alpha;
    cplx<R> x = f[e];
    if constexpr (std::is_same<TO, zdf>::value) tiles[(t * cmax + col0 + v) * B.M + row] = zdf_from(x);
    else tiles[(t * cmax + col0 + v) * B.M + row] = {(double)x.re, (double)x.im};
  }
}

constexpr int GT = 256;   // threads per tile CTA
// threads per Jacobi CTA: a round's work is about (c/2)(c/2 + 1)/2 A blocks and c^2/2 V
// entries, a few per thread at 128, and 128-thread CTAs keep every tile of a launch resident
// at once (8 per SM)
constexpr int JT = 128;
constexpr int GR = 32;    // rows staged per chunk
constexpr int MAXC = 64;  // max columns per tile

// G = A^dag A, upper triangle computed, mirrored.  DF: df64 arithmetic (FP32 units,
// error-free transformations) instead of FP64.  MAXP: column pairs per thread
// (>= pairs / blockDim), which sets the accumulator registers.
// The first kd columns may be known to be orthogonal with squared norms lamp[t][0..kd-1]
// (the previous stream's Phi = A V_k, whose Gram matrix is V_k^dag G V_k = Lambda_k): their
// block is then written as that diagonal and only the pairs (i, j), i <= j, j >= kd are summed.
template <bool DF, int MAXP>
__global__ void __launch_bounds__(GT) gram_kernel(zd* G, const void* __restrict__ tiles, int cmax,
                                                  int c, int M, int kd, const double* lamp,
                                                  int cprev) {
  typedef typename std::conditional<DF, zdf, zd>::type T;
  typedef typename std::conditional<DF, zdfacc, zd>::type TA;
  extern __shared__ zd smraw_g[];
  T* sA = reinterpret_cast<T*>(smraw_g);  // [GR][c]
  int t = blockIdx.x;
  const T* A = reinterpret_cast<const T*>(tiles) + (size_t)t * cmax * M;
  const int nth = blockDim.x;
  const int npairs = c * (c + 1) / 2 - kd * (kd + 1) / 2;
  TA acc[MAXP];
  int pi[MAXP], pj[MAXP];
#pragma unroll
  for (int q = 0; q < MAXP; ++q) {
    acc[q] = TA{};
    int p = threadIdx.x + q * nth;
    // p -> (i, j) with i <= j and j >= kd, column by column (column j holds j + 1 pairs)
    int j = kd, rem = p;
    while (j < c && rem >= j + 1) { rem -= j + 1; ++j; }
    pi[q] = rem;
    pj[q] = j;
  }
  zd* Gt = G + (size_t)t * c * c;
  for (int e = threadIdx.x; e < kd * kd; e += nth) {
    const int i = e / kd, j = e % kd;
    Gt[i * c + j] = i == j ? zd{lamp[(size_t)t * cprev + i], 0.0} : zd{0.0, 0.0};
  }
  for (int r0 = 0; r0 < M; r0 += GR) {
    int nr = min(GR, M - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * c; e += nth) {
      int col = e / nr, rr = e % nr;
      if constexpr (DF) sA[rr * c + col] = zdf_ld(A + (size_t)col * M + r0 + rr);
      else sA[rr * c + col] = A[(size_t)col * M + r0 + rr];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MAXP; ++q) {
      int p = threadIdx.x + q * nth;
      if (p < npairs) {
        TA a = acc[q];
        for (int rr = 0; rr < nr; ++rr) {
          if constexpr (DF) zdf_fmac(a, sA[rr * c + pi[q]], sA[rr * c + pj[q]]);
          else cfmac(a, sA[rr * c + pi[q]], sA[rr * c + pj[q]]);
        }
        acc[q] = a;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < MAXP; ++q) {
    int p = threadIdx.x + q * nth;
    if (p < npairs) {
      zd v;
      if constexpr (DF) v = zdf_result(acc[q]);
      else v = acc[q];
      Gt[pi[q] * c + pj[q]] = v;
      if (pi[q] != pj[q]) Gt[pj[q] * c + pi[q]] = conj(v);
    }
  }
}

// Parallel cyclic Jacobi on a Hermitian c x c matrix per CTA (Brent-Luk round robin).
// Rotation angles are computed in FP64 from the current entries; DF applies the rotations
// to the matrix and the eigenvector basis in double-float arithmetic on the FP32 units
// (this GPU's FP64 rate is ~1/64 of its FP32 rate), otherwise in FP64.
template <typename T> struct JacOps;
template <> struct JacOps<zd> {
  static __device__ __forceinline__ zd from(zd v) { return v; }
  static __device__ __forceinline__ zd val(zd v) { return v; }
  static __device__ __forceinline__ zd zero() { return {0, 0}; }
  static __device__ __forceinline__ zd one() { return {1, 0}; }
  static __device__ __forceinline__ zd cj(zd v) { return {v.re, -v.im}; }
};
template <> struct JacOps<zdf> {
  static __device__ __forceinline__ zdf from(zd v) { return zdf_from(v); }
  static __device__ __forceinline__ zd val(zdf v) { return {df_val(v.re), df_val(v.im)}; }
  static __device__ __forceinline__ zdf zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
  static __device__ __forceinline__ zdf one() { return {{1.f, 0.f}, {0.f, 0.f}}; }
  static __device__ __forceinline__ zdf cj(zdf v) { return {v.re, df_neg(v.im)}; }
};

// (xa, xb) <- (c xa - s ph xb, s xa + c ph xb), c and s real, ph a unit phase
__device__ __forceinline__ void rot_pair(zd& xa, zd& xb, double c, double s, zd ph) {
  zd e = ph * xb;
  zd na = c * xa - s * e;
  xb = s * xa + c * e;
  xa = na;
}
__device__ __forceinline__ void rot_pair(zdf& xa, zdf& xb, df c, df s, zdf ph) {
  zdf e = {df_dot2(ph.re, xb.re, df_neg(ph.im), xb.im), df_dot2(ph.re, xb.im, ph.im, xb.re)};
  df ms = df_neg(s);
  zdf na = {df_dot2(c, xa.re, ms, e.re), df_dot2(c, xa.im, ms, e.im)};
  xb = {df_dot2(s, xa.re, c, e.re), df_dot2(s, xa.im, c, e.im)};
  xa = na;
}

template <bool DF>
__global__ void __launch_bounds__(JT) jacobi_kernel(double* lam, zd* Vec, const zd* G, int c,
                                                    double rtol) {
  typedef typename std::conditional<DF, zdf, zd>::type T;
  typedef typename std::conditional<DF, df, double>::type TR;
  typedef JacOps<T> J;
  extern __shared__ zd sm[];
  int ce = c + (c & 1);              // padded to even
  int np = ce / 2;
  T* A = reinterpret_cast<T*>(sm);    // ce x ce
  T* Vv = A + ce * ce;                // ce x ce
  T* rph = Vv + ce * ce;              // [np] e^{-i phi}
  TR* rcT = reinterpret_cast<TR*>(rph + np);   // [np] cos
  TR* rsT = rcT + np;                          // [np] sin
  int* pa = reinterpret_cast<int*>(rsT + np);    // [ce - 1][np] pair (a < b) of each round
  int* pb = pa + (ce - 1) * np;
  int* rflag = pb + (ce - 1) * np;               // [np] pair rotated in this round
  __shared__ double dg[MAXC];
  int t = blockIdx.x;
  const zd* Gt = G + (size_t)t * c * c;
  const float rtol2 = (float)(rtol * rtol);
  for (int e = threadIdx.x; e < ce * ce; e += blockDim.x) {
    int i = e / ce, j = e % ce;
    A[e] = (i < c && j < c) ? J::from(Gt[i * c + j]) : J::zero();
    Vv[e] = (i == j) ? J::one() : J::zero();
  }
  // the round-robin schedule of all ce - 1 rounds of a sweep, once: pairs (top[p], bot[p])
  // start as (2p, 2p + 1); after each round top[0] stays, the others move one place
  if (threadIdx.x == 0) {
    int top[MAXC / 2], bot[MAXC / 2];
    for (int p = 0; p < np; ++p) { top[p] = 2 * p; bot[p] = 2 * p + 1; }
    for (int round = 0; round < ce - 1; ++round) {
      for (int p = 0; p < np; ++p) {
        pa[round * np + p] = min(top[p], bot[p]);
        pb[round * np + p] = max(top[p], bot[p]);
      }
      if (np > 1) {
        int tlast = top[np - 1];
        int b0 = bot[0];
        for (int p = np - 1; p > 1; --p) top[p] = top[p - 1];
        top[1] = b0;
        for (int p = 0; p < np - 1; ++p) bot[p] = bot[p + 1];
        bot[np - 1] = tlast;
      }
    }
  }
  __syncthreads();
  for (int sweep = 0; sweep < 30; ++sweep) {
    int rotated = 0;   // this thread computed a rotation in this sweep
    for (int round = 0; round < ce - 1; ++round) {
      // rotation parameters
      for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int a = pa[round * np + p], b = pb[round * np + p];
        int f = 0;
        if constexpr (DF) {
          // The angle comes from FP32 copies (the diagonal difference formed in df64 first,
          // so close eigenvalues keep their separation); cos, sin and the phase are then
          // made an exact rotation in df64 (c = (1 + t^2)^-1/2, s = t c, |phase| = 1) by
          // Newton reciprocal square roots on the FP32 units.  An angle good to FP32 leaves
          // ~1e-7 of the pair's coupling, removed when the pair comes round again; the
          // rotation applied is unitary to df64 accuracy either way.
          df cT = {1.f, 0.f}, sT = {0.f, 0.f};
          zdf phT = {{1.f, 0.f}, {0.f, 0.f}};
          if (b < c) {
            zdf g = A[a * ce + b];
            df da = A[a * ce + a].re, db = A[b * ce + b].re;
            float gr = df_to_float(g.re), gi = df_to_float(g.im);
            float ag2 = fmaf(gr, gr, gi * gi);
            if (ag2 > rtol2 * fabsf(da.hi * db.hi) && ag2 > 0.f) {
              float ia = rsqrtf(ag2);            // 1 / |g|
              float zeta = 0.5f * df_to_float(df_add(db, df_neg(da))) * ia;
              float tt = fabsf(zeta) > 1e18f
                             ? 0.5f / zeta
                             : copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
              cT = df_rsqrt(df_add({1.f, 0.f}, df_two_prod(tt, tt)));
              sT = df_mul_f(cT, tt);
              float pr = gr * ia, pi = -gi * ia;   // e^{-i phi} to FP32, then normalised
              df q = df_rsqrt(df_add(df_two_prod(pr, pr), df_two_prod(pi, pi)));
              phT = {df_mul_f(q, pr), df_mul_f(q, pi)};
              f = 1;
            }
          }
          rcT[p] = cT;
          rsT[p] = sT;
          rph[p] = phT;
        } else {
          double c0 = 1.0, s = 0.0;
          zd ph = {1, 0};
          if (b < c) {
            zd g = J::val(A[a * ce + b]);
            double ag = sqrt(norm2(g));
            double da = J::val(A[a * ce + a]).re, db = J::val(A[b * ce + b]).re;
            if (ag > rtol * sqrt(fabs(da * db)) && ag > 1e-300) {
              double zeta = (db - da) / (2.0 * ag);
              double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
              c0 = 1.0 / sqrt(1.0 + tt * tt);
              s = tt * c0;
              ph = {g.re / ag, -g.im / ag};  // e^{-i phi}
              f = 1;
            }
          }
          rcT[p] = c0;
          rsT[p] = s;
          rph[p] = J::from(ph);
        }
        rflag[p] = f;
        rotated |= f;
      }
      __syncthreads();
      // A <- J^dag A J and V <- V J in one pass.  The pairs of a round are disjoint, so the
      // 2 x 2 block of A on the rows of pair p and the columns of pair p' is closed under both
      // rotations: its rows turn with pair p (new_a = c A_a - s e^{i phi} A_b, new_b = s A_a +
      // c e^{i phi} A_b), then its columns with pair p' (phase e^{-i phi}).  A stays Hermitian,
      // so only blocks p <= p' are computed and each p < p' block is mirrored (conjugate
      // transpose) into (p', p); V's columns turn like A's.
      {
        const int nblk = np * (np + 1) / 2;
        for (int e = threadIdx.x; e < nblk + np * ce; e += blockDim.x) {
          if (e < nblk) {
            // block (p, p2), p <= p2, from the packed upper-triangle index
            int p = 0, rem = e;
            while (rem >= np - p) { rem -= np - p; ++p; }
            const int p2 = p + rem;
            const bool fr = rflag[p] != 0, fc = rflag[p2] != 0;
            if (!fr && !fc) continue;
            const int a = pa[round * np + p], b = pb[round * np + p];
            const int a2 = pa[round * np + p2], b2 = pb[round * np + p2];
            T x00 = A[a * ce + a2], x01 = A[a * ce + b2];
            T x10 = A[b * ce + a2], x11 = A[b * ce + b2];
            if (fr) {
              T eph = rph[p];
              if constexpr (DF) eph.im = df_neg(eph.im);
              else eph.im = -eph.im;
              rot_pair(x00, x10, rcT[p], rsT[p], eph);
              rot_pair(x01, x11, rcT[p], rsT[p], eph);
            }
            if (fc) {
              const T mph = rph[p2];
              rot_pair(x00, x01, rcT[p2], rsT[p2], mph);
              rot_pair(x10, x11, rcT[p2], rsT[p2], mph);
            }
            if (p == p2) {
              if constexpr (!DF) {
                // with the exact FP64 angle the rotated pair's coupling is zero
                if (fr) x01 = x10 = J::zero();
              }
            } else {
              A[a2 * ce + a] = J::cj(x00);
              A[b2 * ce + a] = J::cj(x01);
              A[a2 * ce + b] = J::cj(x10);
              A[b2 * ce + b] = J::cj(x11);
            }
            A[a * ce + a2] = x00;
            A[a * ce + b2] = x01;
            A[b * ce + a2] = x10;
            A[b * ce + b2] = x11;
          } else {
            const int ev = e - nblk;
            const int p = ev / ce, k = ev % ce;
            if (!rflag[p]) continue;
            const int a = pa[round * np + p], b = pb[round * np + p];
            T va = Vv[k * ce + a], vb = Vv[k * ce + b];
            rot_pair(va, vb, rcT[p], rsT[p], rph[p]);
            Vv[k * ce + a] = va;
            Vv[k * ce + b] = vb;
          }
        }
      }
      __syncthreads();
    }
    // a barrier that also ORs the flags: every thread takes the same exit decision
    if (!__syncthreads_or(rotated)) break;
  }
  for (int i = threadIdx.x; i < c; i += blockDim.x) dg[i] = J::val(A[i * ce + i]).re;
  __syncthreads();
  // sort eigenvalues descending (stable by index), thread 0; the df64 path compares the
  // normalised (hi, lo) pairs on the FP32 units
  __shared__ int order[MAXC];
  if (threadIdx.x == 0) {
    // stable insertion sort by value descending (ties keep index order)
    for (int i = 0; i < c; ++i) order[i] = i;
    for (int i = 1; i < c; ++i) {
      int key = order[i];
      int j = i - 1;
      if constexpr (DF) {
        df kv = A[key * ce + key].re;
        while (j >= 0 && df_less(A[order[j] * ce + order[j]].re, kv)) {
          order[j + 1] = order[j];
          --j;
        }
      } else {
        double kv = dg[key];
        while (j >= 0 && dg[order[j]] < kv) {
          order[j + 1] = order[j];
          --j;
        }
      }
      order[j + 1] = key;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < c; i += blockDim.x) lam[(size_t)t * c + i] = dg[order[i]];
  zd* Vt = Vec + (size_t)t * c * c;
  for (int e = threadIdx.x; e < c * c; e += blockDim.x) {
    int row = e / c, i = e % c;
    Vt[row * c + i] = J::val(Vv[row * ce + order[i]]);
  }
}

constexpr int UK = 64;  // max output columns per update

template <bool DF>
__global__ void __launch_bounds__(GT) update_kernel(void* out, int cmax_out,
                                                    const void* __restrict__ tiles, int cmax, int c,
                                                    const zd* __restrict__ Vec, const double* lam,
                                                    int kout, int scale_inv, int M) {
  typedef typename std::conditional<DF, zdf, zd>::type T;
  typedef typename std::conditional<DF, zdfacc, zd>::type TA;
  extern __shared__ zd smraw_u[];
  T* sV = reinterpret_cast<T*>(smraw_u);  // [c][kout]
  int t = blockIdx.x;
  const zd* Vt = Vec + (size_t)t * c * c;
  for (int e = threadIdx.x; e < c * kout; e += blockDim.x) {
    int row = e / kout, i = e % kout;
    zd v = Vt[row * c + i];
    if (scale_inv) {
      double l = lam[(size_t)t * c + i];
      double f = l > 0 ? 1.0 / sqrt(l) : 0.0;
      v = f * v;
    }
    if constexpr (DF) sV[e] = zdf_from(v);
    else sV[e] = v;
  }
  __syncthreads();
  const T* A = reinterpret_cast<const T*>(tiles) + (size_t)t * cmax * M;
  T* O = reinterpret_cast<T*>(out) + (size_t)t * cmax_out * M;
  for (int r = threadIdx.x; r < M; r += blockDim.x) {
    for (int i0 = 0; i0 < kout; i0 += 16) {
      TA acc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = TA{};
      for (int col = 0; col < c; ++col) {
        if constexpr (DF) {
          zdf a = zdf_ld(A + (size_t)col * M + r);
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (i0 + q < kout) zdf_fma(acc[q], a, sV[col * kout + i0 + q]);
        } else {
          zd a0 = A[(size_t)col * M + r];
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (i0 + q < kout) cfma(acc[q], a0, sV[col * kout + i0 + q]);
        }
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        if (i0 + q < kout) {
          if constexpr (DF) O[(size_t)(i0 + q) * M + r] = zdf_norm(acc[q]);
          else O[(size_t)(i0 + q) * M + r] = acc[q];
        }
      }
    }
  }
}

__global__ void __launch_bounds__(GT) phase_kernel(zd* tiles, int cmax, int k, int M) {
  __shared__ double sh[64];
  __shared__ zd q;
  int t = blockIdx.x;
  zd* A = tiles + (size_t)t * cmax * M;
  for (int i = 0; i < k; ++i) {
    zd* col = A + (size_t)i * M;
    double a = 0, b = 0;
    for (int r = threadIdx.x; r < M; r += blockDim.x) {
      a += col[r].re;
      b += col[r].im;
    }
    // block sum
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sh[2 * wid] = a; sh[2 * wid + 1] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sa = 0, sb = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sa += sh[2 * w]; sb += sh[2 * w + 1]; }
      double m = sqrt(sa * sa + sb * sb);
      q = m > 0 ? zd{sa / m, -sb / m} : zd{1, 0};
    }
    __syncthreads();
    zd f = q;
    for (int r = threadIdx.x; r < M; r += blockDim.x) col[r] = col[r] * f;
    __syncthreads();
  }
}

// The same canonical phase on double-float tiles, in double-float arithmetic: the column sum
// accumulated error-free on the FP32 units, q = conj(s) / |s| normalised by a Newton
// reciprocal square root, each entry multiplied by q.
// OUT: instead of writing the phased columns back, write them as the outputs P [tile][k][M]
// in complex double, complex float (rounded) and, if Pdf is not null, double-float.
template <bool OUT>
__global__ void __launch_bounds__(GT) phase_df_kernel(zdf* tiles, int cmax, int k, int M, zd* P,
                                                      zf* P32, zdf* Pdf) {
  __shared__ df sh[2][GT / 32];
  __shared__ zdf q;
  int t = blockIdx.x;
  zdf* A = tiles + (size_t)t * cmax * M;
  const df one = {1.0f, 0.0f};
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < k; ++i) {
    zdf* col = A + (size_t)i * M;
    dfacc a{0.f, 0.f}, b{0.f, 0.f};
    for (int r = threadIdx.x; r < M; r += blockDim.x) {
      zdf v = col[r];
      df_fma(a, v.re, one);
      df_fma(b, v.im, one);
    }
    df ar = df_norm(a), br = df_norm(b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      df x = {__shfl_down_sync(0xffffffffu, ar.hi, o), __shfl_down_sync(0xffffffffu, ar.lo, o)};
      df y = {__shfl_down_sync(0xffffffffu, br.hi, o), __shfl_down_sync(0xffffffffu, br.lo, o)};
      ar = df_add(ar, x);
      br = df_add(br, y);
    }
    if (lane == 0) { sh[0][wid] = ar; sh[1][wid] = br; }
    __syncthreads();
    if (threadIdx.x == 0) {
      df sa = {0.f, 0.f}, sb = {0.f, 0.f};
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        sa = df_add(sa, sh[0][w]);
        sb = df_add(sb, sh[1][w]);
      }
      df n2 = df_add(df_mul(sa, sa), df_mul(sb, sb));
      if (n2.hi > 0.f) {
        df inv = df_rsqrt(n2);
        q = {df_mul(sa, inv), df_neg(df_mul(sb, inv))};
      } else {
        q = {one, {0.f, 0.f}};
      }
    }
    __syncthreads();
    zdf f = q;
    const size_t o = ((size_t)t * k + i) * M;
    for (int r = threadIdx.x; r < M; r += blockDim.x) {
      zdf v = col[r];
      zdf w = {df_dot2(v.re, f.re, df_neg(v.im), f.im), df_dot2(v.re, f.im, v.im, f.re)};
      if (OUT) {
        P[o + r] = {df_val(w.re), df_val(w.im)};
        P32[o + r] = {df_to_float(w.re), df_to_float(w.im)};
        if (Pdf) Pdf[o + r] = w;
      } else {
        col[r] = w;
      }
    }
    __syncthreads();
  }
}

// Least-squares interpolation weights (Eq. 9): with the tile A = U Sigma V^dag (V and
// Sigma^2 from the Gram eigen-decomposition), V_c = Sigma_k V_k^dag and Omega = diag(omega),
//   P = A Omega V_c^dag (V_c Omega V_c^dag)^{-1} = A W,  W = Omega V_k B^{-1} Sigma_k^{-1},
//   B = V_k^dag Omega V_k (k x k, Hermitian positive definite for omega > 0).
// One CTA per tile: B in shared memory, inverted by Gauss-Jordan elimination with partial
// pivoting in FP64; W[t][row][i] (leading dimension c, columns i < k) for tile_update.
__global__ void __launch_bounds__(GT) ls_weights_kernel(zd* W, const zd* __restrict__ Vec,
                                                        const double* __restrict__ lam,
                                                        const double* __restrict__ omega, int c,
                                                        int k) {
  extern __shared__ zd lsm[];
  zd* Bm = lsm;                  // [k][2k]: B | I, reduced to I | B^-1
  zd* fc = Bm + (size_t)k * 2 * k;   // [k] the pivot column's factors of one elimination step
  __shared__ int piv;
  const int t = blockIdx.x, w2 = 2 * k;
  const zd* V = Vec + (size_t)t * c * c;   // V[row * c + i]
  for (int e = threadIdx.x; e < k * w2; e += blockDim.x) {
    int a = e / w2, b = e % w2;
    zd s = {0, 0};
    if (b < k) {
      for (int r = 0; r < c; ++r) cfmac(s, V[r * c + a], omega[r] * V[r * c + b]);
    } else {
      s = {(b - k) == a ? 1.0 : 0.0, 0.0};
    }
    Bm[e] = s;
  }
  __syncthreads();
  for (int col = 0; col < k; ++col) {
    if (threadIdx.x == 0) {
      int p = col;
      double m = -1;
      for (int r = col; r < k; ++r) {
        double v = norm2(Bm[r * w2 + col]);
        if (v > m) { m = v; p = r; }
      }
      piv = p;
    }
    __syncthreads();
    if (piv != col)
      for (int b = threadIdx.x; b < w2; b += blockDim.x) {
        zd x = Bm[col * w2 + b];
        Bm[col * w2 + b] = Bm[piv * w2 + b];
        Bm[piv * w2 + b] = x;
      }
    __syncthreads();
    zd pv = Bm[col * w2 + col];
    double d = norm2(pv);
    zd inv = d > 0 ? zd{pv.re / d, -pv.im / d} : zd{0, 0};
    __syncthreads();
    for (int b = threadIdx.x; b < w2; b += blockDim.x) Bm[col * w2 + b] = Bm[col * w2 + b] * inv;
    for (int r = threadIdx.x; r < k; r += blockDim.x) fc[r] = Bm[r * w2 + col];
    __syncthreads();
    for (int e = threadIdx.x; e < k * w2; e += blockDim.x) {
      int r = e / w2, b = e % w2;
      if (r == col) continue;
      Bm[e] = Bm[e] - fc[r] * Bm[col * w2 + b];
    }
    __syncthreads();
  }
  zd* Wt = W + (size_t)t * c * c;
  for (int e = threadIdx.x; e < c * k; e += blockDim.x) {
    int r = e / k, i = e % k;
    zd s = {0, 0};
    for (int a = 0; a < k; ++a) cfma(s, V[r * c + a], Bm[a * w2 + k + i]);
    double l = lam[(size_t)t * c + i];
    double f = l > 0 ? omega[r] / sqrt(l) : 0.0;
    Wt[r * c + i] = f * s;
  }
}

__global__ void sigma_kernel(double* sig, int ldsig, const double* lam, int c, int kk, int ntiles) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ntiles * kk) return;
  int t = e / kk, i = e % kk;
  double l = lam[(size_t)t * c + i];
  sig[(size_t)t * ldsig + i] = l > 0 ? sqrt(l) : 0.0;
}

}  // namespace

int make_blocking(Blocking& B, const int dims[4], const int block[4]) {
  B.nd = 1;
  B.d = 1;
  for (int m = 0; m < 4; ++m) {
    if (block[m] < 1 || dims[m] % block[m] != 0)
      return fail(MG_EINVAL, "aggregate extents must divide the lattice extents");
    B.L[m] = dims[m];
    B.b[m] = block[m];
    B.C[m] = dims[m] / block[m];
    B.nd *= block[m];
    B.d *= B.C[m];
  }
  B.M = 6 * B.nd;
  return MG_OK;
}

template <typename R>
int chiral_gather(void* tiles, int cmax, int col0, const cplx<R>* fields, int nvec,
                  const Blocking& B, cudaStream_t st, bool df64) {
  size_t total = (size_t)nvec * B.nd * B.d * 12;
  size_t g = (total + 255) / 256;
  size_t cap = (size_t)num_sms() * 16;
  unsigned grid = (unsigned)(g < cap ? g : cap);
  if (df64) gather_kernel<R, zdf><<<grid, 256, 0, st>>>((zdf*)tiles, cmax, col0, fields, nvec, B);
  else gather_kernel<R, zd><<<grid, 256, 0, st>>>((zd*)tiles, cmax, col0, fields, nvec, B);
  WMG_LAUNCHED();
  return MG_OK;
}
template int chiral_gather<float>(void*, int, int, const zf*, int, const Blocking&, cudaStream_t, bool);
template int chiral_gather<double>(void*, int, int, const zd*, int, const Blocking&, cudaStream_t, bool);

int tile_gram(zd* G, const void* tiles, int cmax, int c, const Blocking& B, cudaStream_t st,
              bool df64, int kd, const double* lam_prev, int c_prev) {
  if (c > MAXC) return fail(MG_EINVAL, "tile_gram: more than 64 columns");
  if (kd < 0 || kd > c || (kd > 0 && (!lam_prev || c_prev < kd)))
    return fail(MG_EINVAL, "tile_gram: bad known-diagonal block");
  size_t sh = sizeof(zd) * GR * c;
  const int npairs = c * (c + 1) / 2 - kd * (kd + 1) / 2;
  // one thread per summed pair where they fit one CTA (whole warps, at least two)
  const int nth = npairs >= GT ? GT : std::max(64, (npairs + 31) / 32 * 32);
  ProfScope ps(df64 ? "svd_gram_df64" : "svd_gram_fp64", 16.0 * B.M * c * B.d * 2,
               8.0 * B.M * npairs * B.d * 2, st);
  int np = (npairs + nth - 1) / nth;
#define WMG_GRAM(DFV, MP) \
  gram_kernel<DFV, MP><<<B.d * 2, nth, sh, st>>>(G, tiles, cmax, c, B.M, kd, lam_prev, c_prev)
  if (df64) {
    if (np <= 1) WMG_GRAM(true, 1);
    else if (np <= 2) WMG_GRAM(true, 2);
    else if (np <= 4) WMG_GRAM(true, 4);
    else WMG_GRAM(true, 9);
  } else {
    if (np <= 1) WMG_GRAM(false, 1);
    else if (np <= 2) WMG_GRAM(false, 2);
    else if (np <= 4) WMG_GRAM(false, 4);
    else WMG_GRAM(false, 9);
  }
#undef WMG_GRAM
  WMG_LAUNCHED();
  return MG_OK;
}

int tile_eig(double* lam, zd* Vec, zd* G, int c, int ntiles, cudaStream_t st, double rtol,
             bool df64) {
  if (c > MAXC) return fail(MG_EINVAL, "tile_eig: more than 64 columns");
  int ce = c + (c & 1), np = ce / 2;
  // A, V, phases (16-byte complex in both arithmetics), cos, sin (8 bytes), the round-robin
  // schedule and the rotation flags
  size_t sh = sizeof(zd) * (2 * ce * ce + np) + sizeof(double) * 2 * np +
              sizeof(int) * (2 * (ce - 1) * np + np) + 64;
  WMG_TRY(smem_attr(df64 ? jacobi_kernel<true> : jacobi_kernel<false>, sh));
  ProfScope ps(df64 ? "svd_jacobi_df64" : "svd_jacobi_fp64", 32.0 * c * c * ntiles, 0.0, st);
  if (df64) jacobi_kernel<true><<<ntiles, JT, sh, st>>>(lam, Vec, G, c, rtol);
  else jacobi_kernel<false><<<ntiles, JT, sh, st>>>(lam, Vec, G, c, rtol);
  WMG_LAUNCHED();
  return MG_OK;
}

int tile_update(void* out, int cmax_out, const void* tiles, int cmax, int c, const zd* Vec,
                const double* lam, int kout, int scale_inv, const Blocking& B, cudaStream_t st,
                bool df64) {
  if (kout > UK || c > MAXC) return fail(MG_EINVAL, "tile_update: too many columns");
  size_t sh = sizeof(zd) * c * kout;
  WMG_TRY(smem_attr(df64 ? update_kernel<true> : update_kernel<false>, sh));
  ProfScope ps(df64 ? "svd_update_df64" : "svd_update_fp64", 16.0 * B.M * (c + kout) * B.d * 2,
               8.0 * B.M * c * kout * B.d * 2, st);
  if (df64)
    update_kernel<true><<<B.d * 2, GT, sh, st>>>(out, cmax_out, tiles, cmax, c, Vec, lam, kout,
                                                 scale_inv, B.M);
  else
    update_kernel<false><<<B.d * 2, GT, sh, st>>>(out, cmax_out, tiles, cmax, c, Vec, lam, kout,
                                                  scale_inv, B.M);
  WMG_LAUNCHED();
  return MG_OK;
}

int tile_canonical_phase(void* tiles, int cmax, int k, const Blocking& B, cudaStream_t st,
                         bool df64) {
  if (df64) phase_df_kernel<false><<<B.d * 2, GT, 0, st>>>((zdf*)tiles, cmax, k, B.M, nullptr, nullptr, nullptr);
  else phase_kernel<<<B.d * 2, GT, 0, st>>>((zd*)tiles, cmax, k, B.M);
  WMG_LAUNCHED();
  return MG_OK;
}

int tile_phase_outputs(zd* P, zf* P32, zdf* Pdf, void* tiles, int cmax, int k,
                       const Blocking& B, cudaStream_t st) {
  phase_df_kernel<true><<<B.d * 2, GT, 0, st>>>((zdf*)tiles, cmax, k, B.M, P, P32, Pdf);
  WMG_LAUNCHED();
  return MG_OK;
}

int tile_ls_weights(zd* W, const zd* Vec, const double* lam, const double* omega, int c, int k,
                    int ntiles, cudaStream_t st) {
  if (k > c || c > MAXC) return fail(MG_EINVAL, "tile_ls_weights: bad sizes");
  size_t sh = sizeof(zd) * ((size_t)k * 2 * k + k);
  WMG_TRY(smem_attr(ls_weights_kernel, sh));
  ls_weights_kernel<<<ntiles, GT, sh, st>>>(W, Vec, lam, omega, c, k);
  WMG_LAUNCHED();
  return MG_OK;
}

int tile_sigma(double* sig, int ldsig, const double* lam, int c, int kk, int ntiles,
               cudaStream_t st) {
  int tot = ntiles * kk;
  sigma_kernel<<<(tot + 255) / 256, 256, 0, st>>>(sig, ldsig, lam, c, kk, ntiles);
  WMG_LAUNCHED();
  return MG_OK;
}

}  // namespace wmg
