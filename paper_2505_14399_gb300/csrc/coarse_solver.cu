// Coarse-level GMRES (the coarse solve of the K-cycle, Sec. 2.1 / Sec. 4: ||r|| <= 0.03 ||b||)
// as one persistent cooperative kernel.
//
// The coarse system (d coarse sites x 2k unknowns) is small and its solve needs hundreds of
// Arnoldi steps, each a stencil apply and a handful of global inner products.  Launching a
// kernel per operation is latency-bound, so the whole restarted GMRES runs inside a single
// cooperative grid: every CTA owns whole coarse sites (rows), keeps its rows of the Krylov
// basis, and holds a private copy of the small Hessenberg least-squares problem in shared
// memory.  Global quantities (dot products, norms) are reduced with per-CTA partials and a
// fixed-order sum that every CTA performs identically, so all CTAs take identical decisions.
//
// Per Arnoldi step: apply (reads neighbours' raw direction W), CGS2 pass 1 (barrier),
// pass 2 (barrier), norm (barrier): three grid barriers.  Only W is read across CTAs; V rows
// are private to their owner.  Every barrier wait is bounded; on timeout the kernel raises
// an error word and all CTAs return (the host maps it to MG_ETIMEOUT).
#include <cmath>

#include "common.cuh"
#include "grid.cuh"
#include "internal.h"

namespace wmg {

namespace {

constexpr int CT = 256;       // threads per CTA
constexpr int RPT = 8;        // rows per thread (registers)
constexpr int MAXM = 48;      // restart length supported in shared memory

// L1-bypassing load of a complex value written by another CTA.
__device__ __forceinline__ zf ldcg_c(const zf* p) {
  float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ zd ldcg_c(const zd* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

template <typename R>
struct CArgs {
  const cplx<R>* Op;
  Blocking B;
  int n2k;
  cplx<R>* x;          // [nc]
  const cplx<R>* b;    // [nc]
  cplx<R>* V;          // [(m+1)][nc]
  cplx<R>* W;          // [nc] raw direction read by neighbours
  double* partial;     // [2][grid][2 * (m + 2)], alternating per reduction
  BarrierState* bar;
  int* iters;
  double rtol;
  int m;
  int maxiter;
  int spc;             // coarse sites per CTA
  int op_in_smem;      // 1: this CTA's operator slice is staged in shared memory once
};

// out[i] = sum over this CTA's rows of conj(X_i[r]) w[r] for i < cnt (X_i = X + i * xstride),
// accumulated in the vectors' precision R (FP64 arithmetic is scarce on this GPU), then
// widened to FP64 for the per-warp partials.  Results in out[0..cnt) (shared memory).
template <typename R>
__device__ void cta_dots(const cplx<R>* X, size_t xstride, int cnt, const cplx<R> w[RPT],
                         int row0, int row1, zd* out, double* scratch) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < cnt; ++i) {
    R ar = 0, ai = 0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      int r = row0 + threadIdx.x + q * CT;
      if (r < row1) {
        cplx<R> v = X ? X[(size_t)i * xstride + r] : w[q];
        ar = fma(v.re, w[q].re, ar);
        ar = fma(v.im, w[q].im, ar);
        ai = fma(v.re, w[q].im, ai);
        ai = fma(-v.im, w[q].re, ai);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_down_sync(0xffffffffu, ar, o);
      ai += __shfl_down_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) {
      scratch[(wid * cnt + i) * 2] = (double)ar;
      scratch[(wid * cnt + i) * 2 + 1] = (double)ai;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    double x = 0, y = 0;
    for (int wv = 0; wv < CT / 32; ++wv) {
      x += scratch[(wv * cnt + i) * 2];
      y += scratch[(wv * cnt + i) * 2 + 1];
    }
    out[i] = {x, y};
  }
  __syncthreads();
}

// After a barrier: total[i] = sum over CTAs of partial[cta][i] in CTA order.
__device__ void grid_total(const double* partial, int stride, int cnt, zd* total) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < cnt; i += CT / 32) {
    double a = 0, bb = 0;
    for (int c = lane; c < (int)gridDim.x; c += 32) {
      a += __ldcg(partial + (size_t)c * stride + 2 * i);
      bb += __ldcg(partial + (size_t)c * stride + 2 * i + 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      bb += __shfl_down_sync(0xffffffffu, bb, o);
    }
    if (lane == 0) total[i] = {a, bb};
  }
  __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(CT) coarse_gmres_kernel(CArgs<R> a) {
  extern __shared__ double dsm[];
  const int m = a.m;
  zd* H = reinterpret_cast<zd*>(dsm);            // [(m+1) x m] column-major
  zd* sn = H + (m + 1) * m;                      // [m]
  zd* g = sn + m;                                // [m+1]
  zd* y = g + m + 1;                             // [m]
  zd* hv = y + m;                                // [m+2] reduced values
  double* cs = reinterpret_cast<double*>(hv + m + 2);   // [m]
  double* scratch = cs + m;                             // [CT/32][m+2][2]
  const int n2k = a.n2k;
  const int spc = a.spc;
  // staged vectors and operator start on a 16-byte boundary (16-byte copies below)
  uintptr_t p_sx = reinterpret_cast<uintptr_t>(scratch + (CT / 32) * (m + 2) * 2);
  p_sx = (p_sx + 15) & ~(uintptr_t)15;   // the host reserves 16 bytes for this
  cplx<R>* sx = reinterpret_cast<cplx<R>*>(p_sx);   // [spc][9][n2k]
  // spc * 9 * 2k complex numbers: a multiple of 16 bytes, so sOp stays aligned
  cplx<R>* sOp = sx + (size_t)spc * 9 * n2k;          // [spc][9][n2k][n2k] if op_in_smem
  __shared__ double s_res;

  const int d = a.B.d;
  const size_t nc = (size_t)d * n2k;
  const int j0 = blockIdx.x * spc;
  const int j1 = min(d, j0 + spc);
  const int row0 = j0 * n2k, row1 = j1 * n2k;
  const int stride = 2 * (m + 2);
  // Reduction number `red` writes buffer red % 2.  Its readers finish before they arrive at
  // the barrier of reduction red + 1, and reduction red + 2 writes only after that barrier.
  int red = 0;

  cplx<R> w[RPT];

  // rows of this thread: row0 + threadIdx.x + q * CT
  auto row_of = [&](int q) { return row0 + threadIdx.x + q * CT; };

  const int nloc = j1 > j0 ? j1 - j0 : 0;
  const size_t blk_el = (size_t)n2k * n2k;
  if (a.op_in_smem) {
    // this CTA's coarse sites are contiguous in Op: one coalesced copy per launch, 16-byte
    // accesses with four loads in flight per thread (both ends are 16-byte aligned: the
    // slice is a multiple of 9 (2k)^2 complex numbers and the host aligns the layout)
    const float4* src = reinterpret_cast<const float4*>(a.Op + (size_t)j0 * 9 * blk_el);
    float4* dst = reinterpret_cast<float4*>(sOp);
    size_t n16 = (size_t)nloc * 9 * blk_el * sizeof(cplx<R>) / 16;
    size_t e = threadIdx.x;
    for (; e + 3 * CT < n16; e += 4 * CT) {
      float4 v0 = __ldg(src + e), v1 = __ldg(src + e + CT);
      float4 v2 = __ldg(src + e + 2 * CT), v3 = __ldg(src + e + 3 * CT);
      dst[e] = v0;
      dst[e + CT] = v1;
      dst[e + 2 * CT] = v2;
      dst[e + 3 * CT] = v3;
    }
    for (; e < n16; e += CT) dst[e] = __ldg(src + e);
  }
  __syncthreads();

  // raw direction apply: out = A src (rows of this thread).  The nine neighbour vectors of
  // every local coarse site are staged in shared memory first (all loads in flight at once).
  auto apply = [&](cplx<R> out[RPT], const cplx<R>* src, double scale) {
    for (int e = threadIdx.x; e < nloc * 9 * n2k; e += CT) {
      int jl = e / (9 * n2k), rem = e % (9 * n2k);
      int blk = rem / n2k, bb = rem % n2k;
      int j = j0 + jl;
      int s = blk == 0 ? j : a.B.coarse_nbr(j, blk - 1);
      sx[e] = ldcg_c(src + (size_t)s * n2k + bb);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      int r = row_of(q);
      cplx<R> acc = {0, 0};
      if (r < row1) {
        int jl = r / n2k - j0, aa = r % n2k;
        const cplx<R>* O = a.op_in_smem ? sOp + (size_t)jl * 9 * blk_el + aa
                                        : a.Op + ((size_t)(j0 + jl) * 9) * blk_el + aa;
        const cplx<R>* xs = sx + (size_t)jl * 9 * n2k;
        for (int blk = 0; blk < 9; ++blk) {
#pragma unroll 8
          for (int bb = 0; bb < n2k; ++bb) cfma(acc, O[(size_t)bb * n2k], xs[bb]);
          O += blk_el;
          xs += n2k;
        }
      }
      out[q] = {(R)(scale * acc.re), (R)(scale * acc.im)};
    }
    __syncthreads();
  };

  // local norm^2 of a register vector -> partial slot 0; returns after grid reduction
  auto grid_norm = [&](const cplx<R> v[RPT], double* nrm) -> bool {
    cta_dots<R>(nullptr, 0, 1, v, row0, row1, hv, scratch);
    double* buf = a.partial + (size_t)(red & 1) * gridDim.x * stride;
    if (threadIdx.x == 0) { buf[(size_t)blockIdx.x * stride] = hv[0].re; buf[(size_t)blockIdx.x * stride + 1] = 0; }
    if (!grid_barrier(a.bar, gridDim.x)) return false;
    grid_total(buf, stride, 1, hv);
    ++red;
    *nrm = sqrt(hv[0].re);
    __syncthreads();
    return true;
  };

  // ---- x = 0, r = b, beta = ||b||
  cplx<R> rr[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    int r = row_of(q);
    if (r < row1) {
      a.x[r] = {0, 0};
      rr[q] = a.b[r];
    } else {
      rr[q] = {0, 0};
    }
  }
  double bnorm;
  if (!grid_norm(rr, &bnorm)) return;
  const double target = a.rtol * bnorm;
  int its = 0;
  double beta = bnorm;
  bool converged = !(bnorm > target);
  // W = r (raw), V0 = r / beta
  while (!converged && its < a.maxiter) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      int r = row_of(q);
      if (r < row1) {
        a.W[r] = rr[q];
        double f = beta > 0 ? 1.0 / beta : 0.0;
        a.V[r] = {(R)(f * rr[q].re), (R)(f * rr[q].im)};
      }
    }
    if (threadIdx.x == 0) {
      for (int i = 0; i < (m + 1) * m; ++i) H[i] = {0, 0};
      for (int i = 0; i <= m; ++i) g[i] = {0, 0};
      g[0] = {beta, 0};
    }
    if (!grid_barrier(a.bar, gridDim.x)) return;
    double wscale = beta > 0 ? 1.0 / beta : 0.0;   // V_j = W / wscale^-1
    int steps = 0;
    for (int jj = 0; jj < m && its < a.maxiter; ++jj) {
      // w = A V_jj = (A W) * wscale
      apply(w, a.W, wscale);
      // CGS pass 1 and 2
      for (int pass = 0; pass < 2; ++pass) {
        cta_dots<R>(a.V, nc, jj + 1, w, row0, row1, hv, scratch);
        double* buf = a.partial + (size_t)(red & 1) * gridDim.x * stride;
        for (int i = threadIdx.x; i <= jj; i += CT) {
          buf[(size_t)blockIdx.x * stride + 2 * i] = hv[i].re;
          buf[(size_t)blockIdx.x * stride + 2 * i + 1] = hv[i].im;
        }
        if (!grid_barrier(a.bar, gridDim.x)) return;
        grid_total(buf, stride, jj + 1, hv);
        ++red;
        // w -= V h ; accumulate h into the Hessenberg column
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          int r = row_of(q);
          if (r < row1) {
            cplx<R> t = w[q];
            for (int i = 0; i <= jj; ++i) {
              cplx<R> v = a.V[(size_t)i * nc + r];
              cplx<R> h = {(R)hv[i].re, (R)hv[i].im};
              t -= h * v;
            }
            w[q] = t;
          }
        }
        if (threadIdx.x == 0)
          for (int i = 0; i <= jj; ++i) H[(size_t)jj * (m + 1) + i] += hv[i];
        __syncthreads();
      }
      // raw next direction for the neighbours, then its norm
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        int r = row_of(q);
        if (r < row1) a.W[r] = w[q];
      }
      double hn;
      if (!grid_norm(w, &hn)) return;
      // V_{jj+1} rows (private) and the Givens update (identical in every CTA)
      double f = hn > 0 ? 1.0 / hn : 0.0;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        int r = row_of(q);
        if (r < row1)
          a.V[(size_t)(jj + 1) * nc + r] = {(R)(f * w[q].re), (R)(f * w[q].im)};
      }
      if (threadIdx.x == 0) {
        zd* col = H + (size_t)jj * (m + 1);
        col[jj + 1] = {hn, 0};
        for (int i = 0; i < jj; ++i) {
          double c = cs[i];
          zd sv = sn[i];
          zd x0 = col[i], x1 = col[i + 1];
          col[i] = c * x0 + sv * x1;
          col[i + 1] = c * x1 - cmulc(sv, x0);
        }
        zd a0 = col[jj], b0 = col[jj + 1];
        double na = sqrt(norm2(a0)), nbv = sqrt(norm2(b0));
        double rho = hypot(na, nbv);
        double c;
        zd sv;
        if (rho == 0.0) { c = 1.0; sv = {0, 0}; }
        else if (na == 0.0) { c = 0.0; sv = {b0.re / rho, -b0.im / rho}; }
        else { c = na / rho; zd ua = {a0.re / na, a0.im / na}; sv = (1.0 / rho) * (ua * conj(b0)); }
        col[jj] = c * a0 + sv * b0;
        col[jj + 1] = {0, 0};
        cs[jj] = c;
        sn[jj] = sv;
        zd gj = g[jj];
        g[jj] = c * gj;
        g[jj + 1] = -cmulc(sv, gj);
        s_res = sqrt(norm2(g[jj + 1]));
      }
      __syncthreads();
      wscale = f;
      ++steps;
      ++its;
      if (s_res <= target) break;
    }
    // y = R^{-1} g ; x += V y
    if (threadIdx.x == 0) {
      for (int i = steps - 1; i >= 0; --i) {
        zd acc = g[i];
        for (int k = i + 1; k < steps; ++k) acc = acc - H[(size_t)k * (m + 1) + i] * y[k];
        zd dd = H[(size_t)i * (m + 1) + i];
        double n2 = norm2(dd);
        y[i] = n2 > 0 ? (1.0 / n2) * cmulc(dd, acc) : zd{0, 0};
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      int r = row_of(q);
      if (r < row1) {
        cplx<R> t = a.x[r];
        for (int i = 0; i < steps; ++i) {
          cplx<R> v = a.V[(size_t)i * nc + r];
          cplx<R> yy = {(R)y[i].re, (R)y[i].im};
          t += yy * v;
        }
        a.x[r] = t;
      }
    }
    if (!grid_barrier(a.bar, gridDim.x)) return;
    // true residual r = b - A x
    apply(rr, a.x, 1.0);
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      int r = row_of(q);
      if (r < row1) rr[q] = a.b[r] - rr[q];
    }
    if (!grid_norm(rr, &beta)) return;
    converged = !(beta > target);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.iters = its;
}

}  // namespace

template <typename R>
int CoarseSolver<R>::alloc(size_t nc_, int m_) {
  if (nc == nc_ && m >= m_) return MG_OK;
  release();
  if (m_ > MAXM) return fail(MG_EINVAL, "coarse solver: restart > 48");
  nc = nc_;
  m = m_;
  int dev = 0;
  WMG_CUDA(cudaGetDevice(&dev));
  int coop = 0;
  WMG_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return fail(MG_ECUDA, "cooperative launch unsupported");
  max_grid = num_sms();   // one CTA per SM
  WMG_TRY(dev_alloc(&V, sizeof(cplx<R>) * nc * (m + 1)));
  WMG_TRY(dev_alloc(&W, sizeof(cplx<R>) * nc));
  WMG_TRY(dev_alloc(&partial, sizeof(double) * 2 * 2 * (m + 2) * max_grid));
  WMG_TRY(dev_alloc(&state, sizeof(BarrierState) + 2 * sizeof(int)));
  WMG_CUDA(cudaMemset(state, 0, sizeof(BarrierState) + 2 * sizeof(int)));
  WMG_TRY(host_alloc(&host_state, sizeof(BarrierState) + 2 * sizeof(int)));
  return MG_OK;
}

template <typename R>
size_t CoarseSolver<R>::smem_bytes() const {
  // H, sn, g, y, hv (zd) + cs, scratch (double); staged vectors and operator added at launch
  size_t z = (size_t)(m + 1) * m + m + (m + 1) + m + (m + 2);
  return z * sizeof(zd) + sizeof(double) * (m + (CT / 32) * (m + 2) * 2) + 16;  // + alignment pad
}

template <typename R>
void CoarseSolver<R>::release() {
  dev_free(V);
  dev_free(W);
  dev_free(partial);
  dev_free(state);
  host_free(host_state);
  V = W = nullptr;
  partial = nullptr;
  state = nullptr;
  host_state = nullptr;
  nc = 0;
  m = 0;
}

template <typename R>
bool CoarseSolver<R>::fits(const Blocking& B, int k) const {
  int grid = max_grid < B.d ? max_grid : B.d;
  if (grid < 1) return false;
  int spc = (B.d + grid - 1) / grid;
  return (long long)spc * 2 * k <= (long long)CT * RPT;
}

template <typename R>
int CoarseSolver<R>::solve(const cplx<R>* Op, const Blocking& B, int k, cplx<R>* x,
                           const cplx<R>* b, double rtol, int restart, int maxiter, int* its,
                           cudaStream_t st) {
  if (restart > m) return fail(MG_EINVAL, "coarse solver: restart longer than allocated");
  int n2k = 2 * k;
  // one CTA per SM (at most one per coarse site), whole coarse sites per CTA
  int grid = max_grid < B.d ? max_grid : B.d;
  int spc = (B.d + grid - 1) / grid;
  grid = (B.d + spc - 1) / spc;
  if ((long long)spc * n2k > (long long)CT * RPT)
    return fail(MG_EINVAL, "coarse solver: coarse system too large for one cooperative grid");
  size_t sh = smem_bytes() + sizeof(cplx<R>) * (size_t)spc * 9 * n2k;
  size_t op_bytes = sizeof(cplx<R>) * (size_t)spc * 9 * n2k * n2k;
  int op_in_smem = (sh + op_bytes <= (size_t)210 * 1024) ? 1 : 0;
  if (op_in_smem) sh += op_bytes;
  WMG_CUDA(cudaFuncSetAttribute(coarse_gmres_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sh));
  int per_sm = 0;
  WMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_gmres_kernel<R>, CT, sh));
  if (per_sm < 1 || grid > per_sm * num_sms())
    return fail(MG_ECUDA, "coarse solver: grid cannot be co-resident");
  BarrierState* bs = reinterpret_cast<BarrierState*>(state);
  int* iters = reinterpret_cast<int*>(bs + 1);
  WMG_CUDA(cudaMemsetAsync(state, 0, sizeof(BarrierState) + 2 * sizeof(int), st));
  CArgs<R> args;
  args.Op = Op;
  args.B = B;
  args.n2k = n2k;
  args.x = x;
  args.b = b;
  args.V = V;
  args.W = W;
  args.partial = partial;
  args.bar = bs;
  args.iters = iters;
  args.rtol = rtol;
  args.m = restart;
  args.maxiter = maxiter;
  args.spc = spc;
  args.op_in_smem = op_in_smem;
  void* kargs[] = {&args};
  ProfScope ps("coarse_gmres", (double)sizeof(cplx<R>) * B.d * 9.0 * n2k * n2k, 0.0, st);
  WMG_CUDA(cudaLaunchCooperativeKernel((void*)coarse_gmres_kernel<R>, dim3(grid), dim3(CT), kargs,
                                       sh, st));
  count_launch();
  WMG_CUDA(cudaMemcpyAsync(host_state, state, sizeof(BarrierState) + 2 * sizeof(int),
                           cudaMemcpyDeviceToHost, st));
  WMG_CUDA(cudaStreamSynchronize(st));
  BarrierState* hb = reinterpret_cast<BarrierState*>(host_state);
  if (hb->err) return fail(MG_ETIMEOUT, "coarse solver: grid barrier wait gave up");
  if (its) *its = reinterpret_cast<int*>(hb + 1)[0];
  return MG_OK;
}

// Diagnostic: a grid barrier that waits for one more CTA than the grid has, so every wait
// runs out.  Exercises the bounded-wait error path without faulting or hanging the GPU.
__global__ void barrier_timeout_kernel(BarrierState* bs, long long limit) {
  grid_barrier(bs, gridDim.x + 1, limit);
}

int barrier_timeout_selftest(cudaStream_t st) {
  BarrierState* bs = nullptr;
  WMG_CUDA(cudaMallocAsync(&bs, sizeof(BarrierState), st));
  WMG_CUDA(cudaMemsetAsync(bs, 0, sizeof(BarrierState), st));
  long long limit = 1ll << 16;
  barrier_timeout_kernel<<<2, 32, 0, st>>>(bs, limit);
  WMG_LAUNCHED();
  BarrierState h;
  WMG_CUDA(cudaMemcpyAsync(&h, bs, sizeof(h), cudaMemcpyDeviceToHost, st));
  WMG_CUDA(cudaStreamSynchronize(st));
  WMG_CUDA(cudaFreeAsync(bs, st));
  WMG_CUDA(cudaStreamSynchronize(st));
  if (h.err) return fail(MG_ETIMEOUT, "barrier self-test: bounded wait gave up as designed");
  return fail(MG_ECUDA, "barrier self-test: the wait did not time out");
}

template class CoarseSolver<float>;
template class CoarseSolver<double>;

}  // namespace wmg

extern "C" int mg_selftest_barrier_timeout(void* stream) {
  return wmg::barrier_timeout_selftest((cudaStream_t)stream);
}
