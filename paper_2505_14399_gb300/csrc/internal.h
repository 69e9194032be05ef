// Internal interfaces between the library's translation units.
#pragma once

#include <functional>
#include <vector>

#include "common.cuh"

namespace wmg {

// ------------------------------------------------------------------ Dslash
// in/out strides are in complex elements between right-hand sides (0 = field size).
// link_layout 0: ABI [mu][site][3][3]; 1: lane-contiguous [mu][9][site] (link_to_lanes).
int dslash_launch(int dtype, void* out, const void* in, const void* links, const Geom& g,
                  int parity, int dagger, int nrhs, cudaStream_t st, size_t in_stride,
                  size_t out_stride, int link_layout = 0);
// dst[mu][e][site] = src[mu][site][e] (e < 9), converting complex double to To.
template <typename To>
int link_to_lanes(cplx<To>* dst, const zd* src, int V, cudaStream_t st);

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
  int maxvec = 0;
  int nrhs_cap = 0;
  int alloc(size_t n, int nrhs, int maxvec);
  void release();
};

// out[rhs*ldo + i] = sum_k conj(V_i[rhs][k]) w[rhs][k], i < nv; V_i = V + i*vstride.
template <typename R>
int multi_dot(zd* out, int ldo, const cplx<R>* V, size_t vstride, int nv, const cplx<R>* w,
              size_t n, int nrhs, ReduceWork& rw, cudaStream_t st);
// w[rhs] += sgn * sum_i c[rhs*ldc + i] V_i[rhs]   (coefficients read on the device)
template <typename R>
int multi_axpy(cplx<R>* w, const cplx<R>* V, size_t vstride, int nv, const zd* c, int ldc,
               double sgn, size_t n, int nrhs, cudaStream_t st);
// multi_axpy followed by nrm[rhs*ldn] = ||w[rhs]||_2, in one pass over w
template <typename R>
int multi_axpy_norm(cplx<R>* w, const cplx<R>* V, size_t vstride, int nv, const zd* c, int ldc,
                    double sgn, size_t n, int nrhs, double* nrm, int ldn, ReduceWork& rw,
                    cudaStream_t st);
// nrm[rhs*ldn] = ||w[rhs]||_2
template <typename R>
int norm2(double* nrm, int ldn, const cplx<R>* w, size_t n, int nrhs, ReduceWork& rw,
          cudaStream_t st);
// y[rhs] = x[rhs] / s[rhs*lds]   (s = 0 gives y = 0)
template <typename R>
int scale_inv(cplx<R>* y, const cplx<R>* x, const double* s, int lds, size_t n, int nrhs,
              cudaStream_t st);
// y = a*x + b*y with real scalars
template <typename R>
int axpby(cplx<R>* y, double a, const cplx<R>* x, double b, size_t n, int nrhs,
          cudaStream_t st);
// y = x * s[rhs] (device scale) where mode 0: s, mode 1: 1/s
template <typename Ro, typename Ri>
int convert(cplx<Ro>* y, const cplx<Ri>* x, const double* s, int inv, size_t n, int nrhs,
            cudaStream_t st);
// y += a * s[rhs] * x (x in lower precision, y FP64)
template <typename Ri>
int accumulate_scaled(zd* y, const cplx<Ri>* x, const double* s, size_t n, int nrhs,
                      cudaStream_t st);
template <typename R>
int fill_zero(cplx<R>* y, size_t n, cudaStream_t st);
// multiply spins 2,3 by -1 (gamma_5 in the chiral basis) on fields of V sites
template <typename R>
int apply_gamma5(cplx<R>* y, const cplx<R>* x, size_t nsites_total, cudaStream_t st);

// ------------------------------------------------------------------ Krylov engine
template <typename R>
using Op = std::function<int(cplx<R>* out, const cplx<R>* in, cudaStream_t st)>;

template <typename R>
class Gmres {
 public:
  ~Gmres() { release(); }
  int alloc(size_t n, int nrhs, int m, bool flexible);
  void release();
  // x = argmin ||b - A x|| over K_m(A, b), x0 = 0 (fixed number of steps, no host sync)
  int fixed(const Op<R>& A, cplx<R>* x, const cplx<R>* b, int m, cudaStream_t st);
  // Restarted (F)GMRES from x0 = 0 until ||b - A x|| <= rtol ||b|| for every rhs.
  // M == nullptr: plain GMRES.  Returns MG_OK or MG_ENOCONV; *its = iterations.
  // check_every: host convergence check interval in Arnoldi steps; steps taken past
  // convergence are discarded from the least-squares update, so the iterate and the
  // iteration count equal those of a per-step check.
  int solve(const Op<R>& A, const Op<R>* M, cplx<R>* x, const cplx<R>* b, double rtol,
            int restart, int maxiter, int* its, cudaStream_t st, int check_every = 1);
  size_t n = 0;
  int nrhs = 0, m = 0;
  bool flexible = false;

 private:
  int arnoldi_step(const Op<R>& A, const Op<R>* M, int j, cudaStream_t st);
  cplx<R>* V = nullptr;   // (m+1) x nrhs x n
  cplx<R>* Z = nullptr;   // m x nrhs x n
  cplx<R>* w = nullptr;   // nrhs x n
  zd* small = nullptr;    // device scalars (Hessenberg, rotations, rhs)
  double* dnorm = nullptr;
  double* reshist = nullptr;   // [m][nrhs] residual estimate after each Arnoldi step
  double* host_res = nullptr;  // pinned, (m + 2) * nrhs
  ReduceWork rw;
  size_t off_H = 0, off_h2 = 0, off_cs = 0, off_g = 0, off_y = 0;
};

// ------------------------------------------------------------------ persistent coarse GMRES
struct Blocking;
// Restarted GMRES on the coarse stencil operator in one cooperative launch (one system).
template <typename R>
class CoarseSolver {
 public:
  ~CoarseSolver() { release(); }
  int alloc(size_t nc, int m);
  void release();
  int solve(const cplx<R>* Op, const Blocking& B, int k, cplx<R>* x, const cplx<R>* b,
            double rtol, int restart, int maxiter, int* its, cudaStream_t st);
  size_t nc = 0;
  int m = 0;

 private:
  size_t smem_bytes() const;
  cplx<R>* V = nullptr;
  cplx<R>* W = nullptr;
  double* partial = nullptr;
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
// Tile buffers: [tile][column][row] complex double, column stride M, tile stride cmax*M.
// gather: columns col0 .. col0+nvec-1 of every tile from nvec fields [v][site][12].
template <typename R>
int chiral_gather(zd* tiles, int cmax, int col0, const cplx<R>* fields, int nvec,
                  const Blocking& B, cudaStream_t st);
// G[t][c][c] = A_t^dag A_t over the first c columns.
int tile_gram(zd* G, const zd* tiles, int cmax, int c, const Blocking& B, cudaStream_t st,
              bool df64 = false);
// Hermitian eigen-decomposition of every G_t (c x c) by parallel cyclic Jacobi; returns
// eigenvalues descending in lam[t][c] and eigenvectors in Vec[t][c][c] (column i at
// Vec[t][*][i], row-major c x c).
// rtol: a pair is rotated while |G_ab| > rtol sqrt(|G_aa G_bb|) (relative accuracy target).
int tile_eig(double* lam, zd* Vec, zd* G, int c, int ntiles, cudaStream_t st,
             double rtol = 1e-15);
// out[t][i][row] = sum_c A[t][c][row] Vec[t][c][i] * (scale_inv ? 1/sqrt(lam[t][i]) : 1)
// for i < kout; out tile stride cmax_out*M.
// df64: sums of products in double-float arithmetic (df64.cuh) instead of FP64.
int tile_update(zd* out, int cmax_out, const zd* tiles, int cmax, int c, const zd* Vec,
                const double* lam, int kout, int scale_inv, const Blocking& B, cudaStream_t st,
                bool df64 = false);
// Multiply every column i < k of every tile by conj(q)/|q|, q = sum of its entries.
int tile_canonical_phase(zd* tiles, int cmax, int k, const Blocking& B, cudaStream_t st);
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
int galerkin_build(zd* Op, zd* Xpart, const zd* P, int k, const zd* links, const Geom& g,
                   const Blocking& B, cudaStream_t st, bool df64 = false);
template <typename R>
int coarse_apply_launch(cplx<R>* y, const cplx<R>* x, const cplx<R>* Op, int k, const Blocking& B,
                        int nrhs, cudaStream_t st);

// ------------------------------------------------------------------ gradient
int link_gradient_launch(double* out, const zd* gb, const zd* x, const zd* links, const Geom& g,
                         cudaStream_t st);

// ------------------------------------------------------------------ RNG
// out[v][site][12] complex Gaussian (Philox4x32-10 + Box-Muller) for vector ids
// id0 .. id0+nvec-1.
template <typename R>
int gaussian_fill(cplx<R>* out, unsigned long long seed, unsigned id0, int nvec, int V,
                  cudaStream_t st);

}  // namespace wmg
