// Batched GMRES / flexible GMRES with all Krylov scalars resident on the device.
//
// Arnoldi uses classical Gram-Schmidt applied twice (CGS2: two batched dot passes and
// two batched updates per step), the Hessenberg column is reduced by complex Givens
// rotations in a one-thread-per-system kernel, and the residual estimates |g_{j+1}|
// (one per step, kept on the device) are the only values the host reads, every
// `check_every` steps of a tolerance-driven solve.  All nrhs systems advance in lockstep.
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace wmg {

namespace {

// Per-system layout of the device scalar block (units of zd):
//   H[(m+1) x m] column-major | h2[m+1] | cs[m] (real in .re) | sn[m] | g[m+1] | y[m]
struct SmallLayout {
  int m;
  __host__ __device__ int stride() const { return (m + 1) * m + (m + 1) + m + m + (m + 1) + m; }
  __host__ __device__ int H() const { return 0; }
  __host__ __device__ int h2() const { return (m + 1) * m; }
  __host__ __device__ int cs() const { return h2() + m + 1; }
  __host__ __device__ int sn() const { return cs() + m; }
  __host__ __device__ int g() const { return sn() + m; }
  __host__ __device__ int y() const { return g() + m + 1; }
};

__global__ void init_kernel(zd* small, SmallLayout L, const double* beta, double* res, int nrhs) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  zd* s = small + (size_t)r * L.stride();
  for (int i = 0; i < L.stride(); ++i) s[i] = {0, 0};
  s[L.g()] = {beta[r], 0};
  res[r] = beta[r];
}

// Finish column j: H[:, j] += h2, H[j+1, j] = ||w||, rotate, new rotation, residual.
__global__ void givens_kernel(zd* small, SmallLayout L, int j, const double* wnorm, double* res,
                              int nrhs) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  zd* s = small + (size_t)r * L.stride();
  zd* col = s + L.H() + (size_t)j * (L.m + 1);
  const zd* h2 = s + L.h2();
  for (int i = 0; i <= j; ++i) col[i] = col[i] + h2[i];
  col[j + 1] = {wnorm[r], 0};
  zd* cs = s + L.cs();
  zd* sn = s + L.sn();
  for (int i = 0; i < j; ++i) {
    double c = cs[i].re;
    zd sv = sn[i];
    zd a = col[i], b = col[i + 1];
    zd na = c * a + sv * b;
    zd nb = c * b - cmulc(sv, a);  // -conj(s) a + c b
    col[i] = na;
    col[i + 1] = nb;
  }
  zd a = col[j], b = col[j + 1];
  double na = sqrt(norm2(a)), nbv = sqrt(norm2(b));
  double rho = hypot(na, nbv);
  double c;
  zd sv;
  if (rho == 0.0) {
    c = 1.0;
    sv = {0, 0};
  } else if (na == 0.0) {
    c = 0.0;
    sv = {b.re / rho, -b.im / rho};  // s b = |b|^2/rho: choose s = conj(b)/rho
  } else {
    c = na / rho;
    // s = (a/|a|) conj(b) / rho
    zd ua = {a.re / na, a.im / na};
    sv = (1.0 / rho) * (ua * conj(b));
  }
  zd top = c * a + sv * b;
  col[j] = top;
  col[j + 1] = {0, 0};
  cs[j] = {c, 0};
  sn[j] = sv;
  zd* g = s + L.g();
  zd gj = g[j];
  g[j] = c * gj;
  g[j + 1] = -cmulc(sv, gj);  // -conj(s) g_j
  res[r] = sqrt(norm2(g[j + 1]));
}

// Back substitution R y = g over the first `steps` columns.
__global__ void solve_kernel(zd* small, SmallLayout L, int steps, int nrhs) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  zd* s = small + (size_t)r * L.stride();
  const zd* H = s + L.H();
  const zd* g = s + L.g();
  zd* y = s + L.y();
  for (int i = steps - 1; i >= 0; --i) {
    zd acc = g[i];
    for (int k = i + 1; k < steps; ++k) acc = acc - H[(size_t)k * (L.m + 1) + i] * y[k];
    zd d = H[(size_t)i * (L.m + 1) + i];
    double dd = norm2(d);
    y[i] = dd > 0 ? (1.0 / dd) * cmulc(d, acc) : zd{0, 0};
  }
}

}  // namespace

template <typename R>
int Gmres<R>::alloc(size_t n_, int nrhs_, int m_, bool flexible_) {
  if (n == n_ && nrhs >= nrhs_ && m >= m_ && (flexible || !flexible_)) return MG_OK;
  release();
  n = n_;
  nrhs = nrhs_;
  m = m_;
  flexible = flexible_;
  size_t fb = sizeof(cplx<R>) * n * nrhs;
  WMG_CUDA(cudaMalloc(&V, fb * (m + 1)));
  if (flexible) WMG_CUDA(cudaMalloc(&Z, fb * m));
  WMG_CUDA(cudaMalloc(&w, fb));
  SmallLayout L{m};
  WMG_CUDA(cudaMalloc(&small, sizeof(zd) * L.stride() * nrhs));
  WMG_CUDA(cudaMalloc(&dnorm, sizeof(double) * nrhs * 4));
  WMG_CUDA(cudaMalloc(&reshist, sizeof(double) * nrhs * m));
  WMG_CUDA(cudaMallocHost(&host_res, sizeof(double) * nrhs * (m + 2)));
  WMG_TRY(rw.alloc(n, nrhs, m + 1));
  return MG_OK;
}

template <typename R>
void Gmres<R>::release() {
  if (V) cudaFree(V);
  if (Z) cudaFree(Z);
  if (w) cudaFree(w);
  if (small) cudaFree(small);
  if (dnorm) cudaFree(dnorm);
  if (reshist) cudaFree(reshist);
  if (host_res) cudaFreeHost(host_res);
  V = Z = w = nullptr;
  small = nullptr;
  dnorm = nullptr;
  reshist = nullptr;
  host_res = nullptr;
  rw.release();
  n = 0;
  nrhs = 0;
  m = 0;
}

// dnorm layout: [0..nrhs) current ||w||, [nrhs..2nrhs) beta, [2nrhs..3nrhs) residual estimate
template <typename R>
int Gmres<R>::arnoldi_step(const Op<R>& A, const Op<R>* M, int j, cudaStream_t st) {
  SmallLayout L{m};
  size_t fs = n * nrhs;
  cplx<R>* vj = V + (size_t)j * fs;
  if (M) {
    cplx<R>* zj = Z + (size_t)j * fs;
    WMG_TRY((*M)(zj, vj, st));
    WMG_TRY(A(w, zj, st));
  } else {
    WMG_TRY(A(w, vj, st));
  }
  zd* Hcol = small + L.H() + (size_t)j * (m + 1);
  WMG_TRY(multi_dot<R>(Hcol, L.stride(), V, fs, j + 1, w, n, nrhs, rw, st));
  WMG_TRY(multi_axpy<R>(w, V, fs, j + 1, Hcol, L.stride(), -1.0, n, nrhs, st));
  WMG_TRY(multi_dot<R>(small + L.h2(), L.stride(), V, fs, j + 1, w, n, nrhs, rw, st));
  WMG_TRY(multi_axpy<R>(w, V, fs, j + 1, small + L.h2(), L.stride(), -1.0, n, nrhs, st));
  WMG_TRY(norm2<R>(dnorm, 1, w, n, nrhs, rw, st));
  givens_kernel<<<(nrhs + 31) / 32, 32, 0, st>>>(small, L, j, dnorm, reshist + (size_t)j * nrhs,
                                                 nrhs);
  WMG_LAUNCHED();
  WMG_TRY(scale_inv<R>(V + (size_t)(j + 1) * fs, w, dnorm, 1, n, nrhs, st));
  return MG_OK;
}

template <typename R>
int Gmres<R>::fixed(const Op<R>& A, cplx<R>* x, const cplx<R>* b, int steps, cudaStream_t st) {
  if (steps > m) return fail(MG_EINVAL, "gmres: more steps than allocated");
  SmallLayout L{m};
  size_t fs = n * nrhs;
  WMG_TRY(fill_zero<R>(x, fs, st));
  if (steps == 0) return MG_OK;
  WMG_TRY(norm2<R>(dnorm + nrhs, 1, b, n, nrhs, rw, st));
  init_kernel<<<(nrhs + 31) / 32, 32, 0, st>>>(small, L, dnorm + nrhs, dnorm + 2 * nrhs, nrhs);
  WMG_LAUNCHED();
  WMG_TRY(scale_inv<R>(V, b, dnorm + nrhs, 1, n, nrhs, st));
  for (int j = 0; j < steps; ++j) WMG_TRY(arnoldi_step(A, nullptr, j, st));
  solve_kernel<<<(nrhs + 31) / 32, 32, 0, st>>>(small, L, steps, nrhs);
  WMG_LAUNCHED();
  WMG_TRY(multi_axpy<R>(x, V, fs, steps, small + L.y(), L.stride(), 1.0, n, nrhs, st));
  return MG_OK;
}

template <typename R>
int Gmres<R>::solve(const Op<R>& A, const Op<R>* M, cplx<R>* x, const cplx<R>* b, double rtol,
                    int restart, int maxiter, int* its_out, cudaStream_t st, int check_every) {
  if (restart > m) return fail(MG_EINVAL, "gmres: restart longer than allocated");
  if (M && !flexible) return fail(MG_EINVAL, "gmres: flexible space not allocated");
  SmallLayout L{m};
  size_t fs = n * nrhs;
  WMG_TRY(fill_zero<R>(x, fs, st));
  // bnorm on host
  std::vector<double> bn(nrhs), res(nrhs);
  WMG_TRY(norm2<R>(dnorm + nrhs, 1, b, n, nrhs, rw, st));
  WMG_CUDA(cudaMemcpyAsync(host_res, dnorm + nrhs, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  WMG_CUDA(cudaStreamSynchronize(st));
  for (int r = 0; r < nrhs; ++r) bn[r] = host_res[r];
  // r = b (x0 = 0); the residual lives in w between cycles
  cplx<R>* rvec = w;
  WMG_CUDA(cudaMemcpyAsync(rvec, b, sizeof(cplx<R>) * fs, cudaMemcpyDeviceToDevice, st));
  int its = 0;
  bool converged = false;
  for (int r = 0; r < nrhs; ++r) res[r] = bn[r];
  auto all_done = [&](const double* rr) {
    for (int r = 0; r < nrhs; ++r)
      if (!(rr[r] <= rtol * bn[r])) return false;
    return true;
  };
  if (all_done(res.data())) converged = true;
  while (!converged && its < maxiter) {
    WMG_TRY(norm2<R>(dnorm + nrhs, 1, rvec, n, nrhs, rw, st));
    init_kernel<<<(nrhs + 31) / 32, 32, 0, st>>>(small, L, dnorm + nrhs, dnorm + 2 * nrhs, nrhs);
    WMG_LAUNCHED();
    WMG_TRY(scale_inv<R>(V, rvec, dnorm + nrhs, 1, n, nrhs, st));
    int steps = 0, checked = 0;
    if (check_every < 1) check_every = 1;
    for (int j = 0; j < restart && its < maxiter; ++j) {
      WMG_TRY(arnoldi_step(A, M, j, st));
      ++steps;
      ++its;
      bool check = ((j + 1 - checked) >= check_every) || j + 1 == restart || its >= maxiter;
      if (!check) continue;
      WMG_CUDA(cudaMemcpyAsync(host_res, reshist + (size_t)checked * nrhs,
                               sizeof(double) * nrhs * (j + 1 - checked), cudaMemcpyDeviceToHost,
                               st));
      WMG_CUDA(cudaStreamSynchronize(st));
      bool stop = false;
      for (int jj = checked; jj <= j && !stop; ++jj) {
        const double* rr = host_res + (size_t)(jj - checked) * nrhs;
        for (int r = 0; r < nrhs; ++r)
          if (!std::isfinite(rr[r])) return fail(MG_ENAN, "gmres: non-finite residual");
        if (all_done(rr)) {
          its -= j - jj;     // steps past convergence are discarded
          steps = jj + 1;
          stop = true;
        }
      }
      checked = j + 1;
      if (stop) break;
    }
    solve_kernel<<<(nrhs + 31) / 32, 32, 0, st>>>(small, L, steps, nrhs);
    WMG_LAUNCHED();
    WMG_TRY(multi_axpy<R>(x, M ? Z : V, fs, steps, small + L.y(), L.stride(), 1.0, n, nrhs, st));
    // true residual r = b - A x
    WMG_TRY(A(rvec, x, st));
    WMG_TRY(axpby<R>(rvec, 1.0, b, -1.0, fs, 1, st));
    WMG_TRY(norm2<R>(dnorm + 3 * nrhs, 1, rvec, n, nrhs, rw, st));
    WMG_CUDA(cudaMemcpyAsync(host_res + nrhs, dnorm + 3 * nrhs, sizeof(double) * nrhs,
                             cudaMemcpyDeviceToHost, st));
    WMG_CUDA(cudaStreamSynchronize(st));
    if (all_done(host_res + nrhs)) converged = true;
  }
  if (its_out) *its_out = its;
  if (!converged) return fail(MG_ENOCONV, "gmres: no convergence within maxiter");
  return MG_OK;
}

template class Gmres<float>;
template class Gmres<double>;

}  // namespace wmg
