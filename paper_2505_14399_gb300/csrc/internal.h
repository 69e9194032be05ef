// Internal interfaces between the library's translation units.
#pragma once

#include <functional>
#include <vector>

#include "common.cuh"
#include "vec.cuh"
#include "df64.cuh"

namespace wmg {

// ------------------------------------------------------------------ Dslash
// in/out strides are in complex elements between right-hand sides (0 = field size).
// link_layout 0: ABI [mu][site][3][3]; 1: lane-contiguous [mu][9][site] (link_to_lanes);
// 2: lane-contiguous first two rows [mu][6][site], third row rebuilt (SU(3) links, not C128).
// sub (single-parity form only, may be NULL): out_p = sub_p - (-kappa H_{p,1-p} in), sub with
// out's layout and stride.
int dslash_launch(int dtype, void* out, const void* in, const void* links, const Geom& g,
                  int parity, int dagger, int nrhs, cudaStream_t st, size_t in_stride,
                  size_t out_stride, int link_layout = 0, const void* sub = nullptr);
// dst[mu][e][site] = src[mu][site][e] (e < 3 rows, rows 3 or 2), converting complex double to E
// (vec.cuh); link_layout 1 reads rows = 3, link_layout 2 rows = 2.
template <typename E>
int link_to_lanes_v(E* dst, const zd* src, int V, cudaStream_t st, int rows = 3);
template <typename To>
inline int link_to_lanes(cplx<To>* dst, const zd* src, int V, cudaStream_t st, int rows = 3) {
  return link_to_lanes_v<cplx<To>>(dst, src, V, st, rows);
}
// *dev = the largest deviation of the nlinks 3x3 complex-double links from SU(3):
// max(|U U^dag - 1|_max, |det U - 1|) (synchronises st).
int su3_deviation(double* dev, const zd* links, size_t nlinks, cudaStream_t st);
// the same from a double-float copy of the links, in double-float arithmetic
int su3_deviation_df(double* dev, const zdf* links, size_t nlinks, cudaStream_t st);

// Autotuned launch shape for a kernel with `nvar` candidate shapes; `run(v)` launches
// shape v on the caller's arguments.  Returns the chosen shape or -1 on a CUDA error.
int tuned_variant(int dtype, int parity, int dagger, int V, int nrhs, cudaStream_t st, int nvar,
                  const std::function<void(int)>& run);
const char* tune_report();

// ------------------------------------------------------------------ BLAS-1 (batched)
// All vectors are nrhs contiguous complex arrays of length n (stride n).
// Reductions are deterministic: fixed partition, fixed tree order, FP64 combination.
struct ReduceWork {
  double* partial = nullptr;   // [nrhs][maxvec][nblk] (re, im interleaved)
  unsigned* counter = nullptr; // [nrhs]
  int nblk = 0;
  int cap = 0;        // partial slots per vector: >= nblk, and one per 128 sites of a fine
                      // field, so the fused stencil kernel may launch a CTA per 128 sites
  int maxvec = 0;
  int nrhs_cap = 0;
  int alloc(size_t n, int nrhs, int maxvec);
  void release();
};

// Routines on vectors of element type E (vec.cuh: zd, zf, zh, zbf); the wrappers without
// the _v suffix take cplx<R> vectors.
// out[rhs*ldo + i] = scale * sum_k conj(V_i[rhs][k]) w[rhs][k], i < nv; V_i = V + i*vstride.
template <typename E>
int multi_dot_v(zd* out, int ldo, const E* V, size_t vstride, int nv, const E* w, size_t n,
                int nrhs, ReduceWork& rw, cudaStream_t st, double scale = 1.0);
// w[rhs] += sgn * sum_i c[rhs*ldc + i] V_i[rhs]   (coefficients read on the device)
template <typename E>
int multi_axpy_v(E* w, const E* V, size_t vstride, int nv, const zd* c, int ldc, double sgn,
                 size_t n, int nrhs, cudaStream_t st);
// nrm[rhs*ldn] = sqrt(scale) ||w[rhs]||_2
template <typename E>
int norm2_v(double* nrm, int ldn, const E* w, size_t n, int nrhs, ReduceWork& rw,
            cudaStream_t st, double scale = 1.0);
// y[rhs] = x[rhs] / s[rhs*lds]   (s = 0 gives y = 0)
template <typename E>
int scale_inv_v(E* y, const E* x, const double* s, int lds, size_t n, int nrhs, cudaStream_t st);
// y = a*x + b*y with real scalars
template <typename E>
int axpby_v(E* y, double a, const E* x, double b, size_t n, int nrhs, cudaStream_t st);
// y += a*x, x in another storage (arithmetic of y)
template <typename Ey, typename Ex>
int axpy_mixed(Ey* y, double a, const Ex* x, size_t n, cudaStream_t st);
// y = a*x1 + b*x2, y in another storage than x1, x2 (arithmetic of x)
template <typename Eo, typename Ei>
int lincomb_v(Eo* y, double a, const Ei* x1, double b, const Ei* x2, size_t n, cudaStream_t st);
// y = x * s[rhs] (device scale) where inv 0: s, inv 1: 1/s; s = nullptr: plain copy
template <typename Eo, typename Ei>
int convert_v(Eo* y, const Ei* x, const double* s, int inv, size_t n, int nrhs, cudaStream_t st);
// y += s[rhs] * x (x in lower precision, y FP64)
template <typename Ei>
int accumulate_scaled_v(zd* y, const Ei* x, const double* s, size_t n, int nrhs, cudaStream_t st);
template <typename E>
int fill_zero_v(E* y, size_t n, cudaStream_t st);
// multiply spins 2,3 by -1 (gamma_5 in the chiral basis) on fields of V sites
template <typename E>
int apply_gamma5_v(E* y, const E* x, size_t nsites_total, cudaStream_t st);

template <typename R>
inline int multi_dot(zd* out, int ldo, const cplx<R>* V, size_t vstride, int nv,
                     const cplx<R>* w, size_t n, int nrhs, ReduceWork& rw, cudaStream_t st) {
  return multi_dot_v<cplx<R>>(out, ldo, V, vstride, nv, w, n, nrhs, rw, st);
}
template <typename R>
inline int multi_axpy(cplx<R>* w, const cplx<R>* V, size_t vstride, int nv, const zd* c,
                      int ldc, double sgn, size_t n, int nrhs, cudaStream_t st) {
  return multi_axpy_v<cplx<R>>(w, V, vstride, nv, c, ldc, sgn, n, nrhs, st);
}
template <typename R>
inline int norm2(double* nrm, int ldn, const cplx<R>* w, size_t n, int nrhs, ReduceWork& rw,
                 cudaStream_t st) {
  return norm2_v<cplx<R>>(nrm, ldn, w, n, nrhs, rw, st);
}
template <typename R>
inline int scale_inv(cplx<R>* y, const cplx<R>* x, const double* s, int lds, size_t n, int nrhs,
                     cudaStream_t st) {
  return scale_inv_v<cplx<R>>(y, x, s, lds, n, nrhs, st);
}
template <typename R>
inline int axpby(cplx<R>* y, double a, const cplx<R>* x, double b, size_t n, int nrhs,
                 cudaStream_t st) {
  return axpby_v<cplx<R>>(y, a, x, b, n, nrhs, st);
}
template <typename Ro, typename Ri>
inline int convert(cplx<Ro>* y, const cplx<Ri>* x, const double* s, int inv, size_t n, int nrhs,
                   cudaStream_t st) {
  return convert_v<cplx<Ro>, cplx<Ri>>(y, x, s, inv, n, nrhs, st);
}
template <typename Ri>
inline int accumulate_scaled(zd* y, const cplx<Ri>* x, const double* s, size_t n, int nrhs,
                             cudaStream_t st) {
  return accumulate_scaled_v<cplx<Ri>>(y, x, s, n, nrhs, st);
}
template <typename R>
inline int fill_zero(cplx<R>* y, size_t n, cudaStream_t st) {
  return fill_zero_v<cplx<R>>(y, n, st);
}
template <typename R>
inline int apply_gamma5(cplx<R>* y, const cplx<R>* x, size_t nsites_total, cudaStream_t st) {
  return apply_gamma5_v<cplx<R>>(y, x, nsites_total, st);
}

// ------------------------------------------------------------------ Krylov engine
// Vectors of element type E (vec.cuh).  Bases in half storage use the (1/n) inner product
// (unit root-mean-square columns); norms and tolerances are relative, so callers see no
// difference.
template <typename E>
using OpV = std::function<int(E* out, const E* in, cudaStream_t st)>;
template <typename R>
using Op = OpV<cplx<R>>;

// The fine Wilson-Dirac operator in FP32 with lane-contiguous links ([mu][3x3 entry][site]),
// for fixed-step GMRES runs that fuse it with their projection sweeps.
struct FusedStencil {
  const void* links;
  Geom g;
  int layout = 1;   // 1: [mu][9][site]; 2: first two rows [mu][6][site] (SU(3) links)
  // the even-odd Schur operator D_hat on even half-lattice fields instead of D: its first
  // hop into the odd field `odd` (nrhs of them), the second fused with the projections
  bool schur = false;
  void* odd = nullptr;
};

template <typename E>
class GmresV {
 public:
  ~GmresV() { release(); }
  int alloc(size_t n, int nrhs, int m, bool flexible);
  void release();
  // x = argmin ||b - A x|| over K_m(A, b), x0 = 0 (fixed number of steps, no host sync);
  // accumulate: x += xsign * that minimiser instead (x holds the caller's vector on entry)
  // fused: A is this FP32 fine stencil, applied by one kernel together with each step's
  // projection sweep (complex-float bases only; otherwise ignored)
  int fixed(const OpV<E>& A, E* x, const E* b, int m, cudaStream_t st, bool accumulate = false,
            const FusedStencil* fused = nullptr, double xsign = 1.0);
  // Restarted (F)GMRES from x0 = 0 until ||b - A x|| <= rtol ||b|| for every rhs.
  // M == nullptr: plain GMRES.  Returns MG_OK or MG_ENOCONV; *its = iterations.
  // check_every: host convergence check interval in Arnoldi steps; steps taken past
  // convergence are discarded from the least-squares update, so the iterate and the
  // iteration count equal those of a per-step check.
  int solve(const OpV<E>& A, const OpV<E>* M, E* x, const E* b, double rtol, int restart,
            int maxiter, int* its, cudaStream_t st, int check_every = 1);
  size_t n = 0;
  int nrhs = 0, m = 0;
  bool flexible = false;

 private:
  // b0 (fused first step only): the unscaled right-hand side, scaled and written as v_0 there;
  // next = false: column j + 1 of the basis is not needed (the last step of a fixed run), so
  // only the Givens step of column j runs, not the normalised update
  int arnoldi_step(const OpV<E>& A, const OpV<E>* M, int j, cudaStream_t st,
                   bool single_pass = false, const FusedStencil* fused = nullptr,
                   const E* b0 = nullptr, bool next = true);
  double ip_scale() const { return VecT<E>::rms ? 1.0 / (double)n : 1.0; }
  E* V = nullptr;         // (m+1) x nrhs x n
  E* Z = nullptr;         // m x nrhs x n
  E* w = nullptr;         // nrhs x n
  zd* small = nullptr;    // device scalars (Hessenberg, rotations, rhs)
  double* dnorm = nullptr;
  double* reshist = nullptr;   // [m][nrhs] residual estimate after each Arnoldi step
  double* host_res = nullptr;  // pinned, (m + 2) * nrhs
  ReduceWork rw;
};
template <typename R>
using Gmres = GmresV<cplx<R>>;

// ------------------------------------------------------------------ persistent coarse GMRES
struct Blocking;
// Restarted GMRES on the coarse stencil operator in one cooperative launch (one system).
template <typename R>
class CoarseSolver {
 public:
  ~CoarseSolver() { release(); }
  int alloc(size_t nc, int m);
  void release();
  // Enqueues the solve on `st` without waiting for it: a barrier wait that gives up raises
  // the device error word, and the iteration count accumulates on the device.
  int solve(const cplx<R>* Op, const Blocking& B, int k, cplx<R>* x, const cplx<R>* b,
            double rtol, int restart, int maxiter, cudaStream_t st);
  // iterations of the solves since the last call (synchronises `st`), then resets the count
  int take_iterations(long long* its, cudaStream_t st);
  // whether one cooperative grid holds the coarse system (each CTA keeps its rows in
  // registers: at most 2048 rows per CTA, one CTA per SM)
  bool fits(const Blocking& B, int k) const;
  size_t nc = 0;
  int m = 0;

 private:
  cplx<R>* V = nullptr;
  cplx<R>* W = nullptr;
  R* partial = nullptr;
  void* state = nullptr;
  void* host_state = nullptr;
  int max_grid = 0;
};

// ------------------------------------------------------------------ aggregates
// Aggregates (Lambda_j of Sec. 2.1) are blocks of extent b[mu]; coarse site j is
// lexicographic over C = L / b; local site l is lexicographic inside the block.
// Tile t = 2 j + alpha holds M = 6 n_d rows, row = (l * 2 + spin - 2 alpha) * 3 + colour.
struct Blocking {
  int L[4], b[4], C[4];
  int nd, d, M;
  __host__ __device__ int site(int j, int l) const {
    int cx = j % C[0], r = j / C[0];
    int cy = r % C[1]; r /= C[1];
    int cz = r % C[2], ct = r / C[2];
    int lx = l % b[0], q = l / b[0];
    int ly = q % b[1]; q /= b[1];
    int lz = q % b[2], lt = q / b[2];
    int x = cx * b[0] + lx, y = cy * b[1] + ly, z = cz * b[2] + lz, t = ct * b[3] + lt;
    return x + L[0] * (y + L[1] * (z + L[2] * t));
  }
  __host__ __device__ void block_of(int s, int* j, int* l) const {
    int x = s % L[0], r = s / L[0];
    int y = r % L[1]; r /= L[1];
    int z = r % L[2], t = r / L[2];
    *j = (x / b[0]) + C[0] * ((y / b[1]) + C[1] * ((z / b[2]) + C[2] * (t / b[3])));
    *l = (x % b[0]) + b[0] * ((y % b[1]) + b[1] * ((z % b[2]) + b[2] * (t % b[3])));
  }
  __host__ __device__ int coarse_nbr(int j, int dir) const {
    int c[4];
    c[0] = j % C[0]; int r = j / C[0];
    c[1] = r % C[1]; r /= C[1];
    c[2] = r % C[2]; c[3] = r / C[2];
    int mu = dir >> 1;
    c[mu] = (dir & 1) ? (c[mu] + C[mu] - 1) % C[mu] : (c[mu] + 1) % C[mu];
    return c[0] + C[0] * (c[1] + C[1] * (c[2] + C[2] * c[3]));
  }
};
int make_blocking(Blocking& B, const int dims[4], const int block[4]);

// ------------------------------------------------------------------ chiral SVD
// Tile buffers: [tile][column][row], column stride M, tile stride cmax*M; complex double, or
// complex double-float (zdf, the same 16 bytes) when df64 is set: the double-float setup keeps
// its tiles in that form from the gather to the prolongator, so nothing converts them on the
// FP64 units.
// gather: columns col0 .. col0+nvec-1 of every tile from nvec fields [v][site][12].
template <typename R>
int chiral_gather(void* tiles, int cmax, int col0, const cplx<R>* fields, int nvec,
                  const Blocking& B, cudaStream_t st, bool df64 = false);
// G[t][c][c] = A_t^dag A_t over the first c columns (df64: double-float tiles and sums).
// kd > 0: the first kd columns are the previous stream's Phi = A V_k, orthogonal with squared
// norms lam_prev[t][0..kd-1] (row stride c_prev): that block is written as the diagonal and
// only the pairs with a column j >= kd are summed.
int tile_gram(zd* G, const void* tiles, int cmax, int c, const Blocking& B, cudaStream_t st,
              bool df64 = false, int kd = 0, const double* lam_prev = nullptr, int c_prev = 0);
// Hermitian eigen-decomposition of every G_t (c x c) by parallel cyclic Jacobi; returns
// eigenvalues descending in lam[t][c] and eigenvectors in Vec[t][c][c] (column i at
// Vec[t][*][i], row-major c x c).
// rtol: a pair is rotated while |G_ab| > rtol sqrt(|G_aa G_bb|) (relative accuracy target).
int tile_eig(double* lam, zd* Vec, zd* G, int c, int ntiles, cudaStream_t st, double rtol,
             bool df64 = false);
// out[t][i][row] = sum_c A[t][c][row] Vec[t][c][i] * (scale_inv ? 1/sqrt(lam[t][i]) : 1)
// for i < kout; out tile stride cmax_out*M.
// df64: double-float tiles in and out, sums of products in double-float arithmetic.
int tile_update(void* out, int cmax_out, const void* tiles, int cmax, int c, const zd* Vec,
                const double* lam, int kout, int scale_inv, const Blocking& B, cudaStream_t st,
                bool df64 = false);
// Multiply every column i < k of every tile by conj(q)/|q|, q = sum of its entries.
int tile_canonical_phase(void* tiles, int cmax, int k, const Blocking& B, cudaStream_t st,
                         bool df64 = false);
// For double-float tiles, the canonical phase of every column applied on the way to the
// outputs: the first k columns as P [tile][k][M] in complex double, complex float (rounded)
// and, if Pdf is not null, double-float (the tiles keep their unphased values).
int tile_phase_outputs(zd* P, zf* P32, zdf* Pdf, void* tiles, int cmax, int k,
                       const Blocking& B, cudaStream_t st);
// Eq. 9 weights: W[t][row][i] = omega_row (V_k B^-1)[row][i] / sqrt(lam_i), B = V_k^dag Omega V_k,
// so that A W is the least-squares interpolation prolongator (leading dimension c, i < k)
int tile_ls_weights(zd* W, const zd* Vec, const double* lam, const double* omega, int c, int k,
                    int ntiles, cudaStream_t st);
// sig[t*ldsig + i] = sqrt(max(lam[t][i], 0)), i < kk
int tile_sigma(double* sig, int ldsig, const double* lam, int c, int kk, int ntiles,
               cudaStream_t st);

// ------------------------------------------------------------------ coarse operator
// P: [tile][i][row] with k columns (tile stride k*M).  Coarse vectors [rhs][j][alpha][i].
template <typename R>
int restrict_launch(cplx<R>* vc, const cplx<R>* v, const cplx<R>* P, int k, const Blocking& B,
                    int nrhs, cudaStream_t st);
template <typename R>
int prolong_launch(cplx<R>* v, const cplx<R>* vc, const cplx<R>* P, int k, const Blocking& B,
                   int nrhs, cudaStream_t st);
// Galerkin: Op[j][blk][b][a] (column-major blocks; blk 0 = X, 1 + dir = Y_dir), FP64.
// Scratch: Xpart (4 d (2k)^2), PtP (2 d k^2), and with df64 Pdf (P as (hi, lo) pairs, filled
// here unless pdf_ready says the setup wrote it), Ldf (the links as (hi, lo) pairs, filled
// by the caller) and range_flag (one device int of the caller's, for the tensor path's range
// check; synchronises `st` when that path runs).
int galerkin_build(zd* Op, zd* Xpart, const zd* P, zdf* Pdf, zd* PtP, int k, const zd* links,
                   const zdf* Ldf, const Geom& g, const Blocking& B, cudaStream_t st, bool df64,
                   bool pdf_ready, int* range_flag);
// complex double -> (hi, lo) float pairs
int to_df(zdf* out, const zd* in, size_t n, cudaStream_t st);
template <typename R>
int coarse_apply_launch(cplx<R>* y, const cplx<R>* x, const cplx<R>* Op, int k, const Blocking& B,
                        int nrhs, cudaStream_t st);

// ------------------------------------------------------------------ deeper levels
// B: L = level-l lattice, b = aggregate, C = level-(l+1) lattice, M = n_d k (k = k_l); level-l
// vectors [site][alpha][k], level-(l+1) vectors [J][alpha][kp]; P tiles [2J + alpha][kp][M].
template <typename R>
int coarse_gather(void* tiles, int cmax, int col0, const cplx<R>* fields, int nvec,
                  const Blocking& B, int k, cudaStream_t st, bool df64);
template <typename R>
int coarse_restrict(cplx<R>* vc, const cplx<R>* v, const cplx<R>* P, const Blocking& B, int k,
                    int kp, int nrhs, cudaStream_t st);
template <typename R>
int coarse_prolong(cplx<R>* v, const cplx<R>* vc, const cplx<R>* P, const Blocking& B, int k,
                   int kp, int nrhs, cudaStream_t st);
// Op2 = P^dag Op P (Eq. 5) as the level-(l+1) stencil, from the level-l stencil Op; FP64
int coarse_galerkin(zd* Op2, const zd* Op, const zd* P, const Blocking& B, int k, int kp,
                    cudaStream_t st);

// ------------------------------------------------------------------ even-odd (Schur) form
// even/odd half-lattice fields (checkerboard index site / 2) of nrhs full-lattice fields;
// split skips a NULL output
template <typename E>
int eo_split(E* even, E* odd, const E* full, const Geom& g, int nrhs, cudaStream_t st);
template <typename E>
int eo_join(E* full, const E* even, const E* odd, const Geom& g, int nrhs, cudaStream_t st);
// full += join(even, odd) (complex double / float fields)
template <typename E>
int eo_join_add(E* full, const E* even, const E* odd, const Geom& g, int nrhs, cudaStream_t st);
// (even, odd) = split(a - b) of full fields (complex double / float fields)
template <typename E>
int eo_split_diff(E* even, E* odd, const E* a, const E* b, const Geom& g, int nrhs,
                  cudaStream_t st);
// out = D_hat in = (1 - kappa^2 H_eo H_oe) in on even fields (dagger: D_hat^dag); tmp: odd
// field per rhs; links in `layout` (dslash_launch)
template <typename E>
int schur_apply(E* out, const E* in, E* tmp, const void* links, int layout, const Geom& g,
                int dagger, int nrhs, cudaStream_t st);

// ------------------------------------------------------------------ Wilson-clover term
// C[site][alpha][6][6] = -kappa c_sw sum_{mu<nu} sigma_mu_nu (x) F_mu_nu (chiral blocks), FP64
int clover_field(zd* C, const zd* links, const Geom& g, double csw, cudaStream_t st);
// out[rhs][x] += C(x) in[rhs][x]
template <typename R>
int clover_add(cplx<R>* out, const cplx<R>* in, const cplx<R>* C, int V, int nrhs, cudaStream_t st);
// X_j += sum_{x in Lambda_j} P(x)^dag C(x) P(x) on the chirality-diagonal blocks of Op
int clover_galerkin_add(zd* Op, const zd* P, const zd* C, int k, const Blocking& B, cudaStream_t st);

// ------------------------------------------------------------------ gradient
int link_gradient_launch(double* out, const zd* gb, const zd* x, const zd* links, const Geom& g,
                         cudaStream_t st);

// ------------------------------------------------------------------ RNG
// out[v][site][12] complex Gaussian (Philox4x32-10 + Box-Muller) for vector ids
// id0 .. id0+nvec-1.
template <typename R>
int gaussian_fill(cplx<R>* out, unsigned long long seed, unsigned id0, int nvec, int V,
                  cudaStream_t st);
// out[v][site][c] for nsites sites of ncomp components, counter (site, c, id0 + v, word3)
// (word3: 0 on the fine lattice, the level index on a coarse level)
template <typename R>
int gaussian_fill_n(cplx<R>* out, unsigned long long seed, unsigned id0, int nvec, int nsites,
                    int ncomp, unsigned word3, cudaStream_t st);

}  // namespace wmg
