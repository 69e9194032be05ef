// Coarse-level GMRES (the coarse solve of the K-cycle, Sec. 2.1 / Sec. 4: ||r|| <= 0.03 ||b||)
// as one persistent cooperative kernel.
//
// The coarse system (d coarse sites x 2k unknowns) is small and its solve needs hundreds of
// Arnoldi steps, each a stencil apply and a handful of global inner products.  Launching a
// kernel per operation is latency-bound, so the whole restarted GMRES runs inside a single
// cooperative grid: every CTA owns whole coarse sites (rows), keeps its rows of the Krylov
// basis (in shared memory when they fit), and holds a private copy of the small Hessenberg
// least-squares problem in shared memory.  Global quantities (dot products, norms) are
// reduced with per-CTA partials and a fixed-order sum that every CTA performs identically, so
// all CTAs take identical decisions.
//
// Per Arnoldi step: apply (reads neighbours' raw direction W), CGS2 pass 1 (barrier),
// pass 2 (barrier), norm (barrier): three grid barriers, each a few microseconds, so the
// work between them is arranged for latency: the operator slice is bulk-copied into shared
// memory once per launch, one warp per inner product, all partial loads of a grid sum in
// flight at once.  Only W is read across CTAs; V rows are private to their owner.  Every
// wait is bounded; on timeout the kernel raises the error word and all CTAs return.
#include <cmath>

#include "common.cuh"
#include "grid.cuh"
#include "internal.h"
#include "tma.cuh"

namespace wmg {

namespace {

constexpr int CT = 256;       // threads per CTA
constexpr int NW = CT / 32;   // warps per CTA
constexpr int RPT = 8;        // rows per thread (registers)
constexpr int MAXM = 48;      // restart length supported in shared memory
constexpr int MAXG = 8;       // partial loads per lane of a grid sum: grid <= 256 CTAs
constexpr int OP_WAIT = 1 << 20;
constexpr uint32_t OP_CHUNK = 32768;   // bytes per bulk copy of the operator slice

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
  cplx<R>* V;          // [(m+1)][nc] basis rows (unused when they are kept in shared memory)
  cplx<R>* W;          // [nc] raw direction read by neighbours
  R* partial;          // [2][grid][2 * (m + 2)], alternating per reduction
  BarrierState* bar;
  int* its_acc;        // iterations, accumulated over launches
  int* err;            // pinned error word: set when a bounded wait gives up
  double rtol;
  int m;
  int maxiter;
  int spc;             // coarse sites per CTA
  int op_in_smem;      // 1: this CTA's operator slice is staged in shared memory once
  int v_in_smem;       // 1: this CTA's basis rows live in shared memory
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Dynamic shared memory of one CTA, byte offsets from a 16-byte aligned base: the small
// least-squares problem (H, sn, g, y, hv complex; cs real), neighbour offsets, this CTA's rows
// of w, the staged neighbour rows, then optionally the basis rows and the operator slice.
struct CLayout {
  size_t H, sn, g, y, hv, cs, soff, sw, sx, sV, sOp, total;
  __host__ __device__ CLayout(int m, int spc, int n2k, int csz, int v_in, int op_in) {
    const size_t rsz = (size_t)csz / 2;
    const size_t rows = (size_t)spc * n2k;
    size_t o = 0;
    H = o;   o += al16((size_t)(m + 1) * m * csz);
    sn = o;  o += al16((size_t)m * csz);
    g = o;   o += al16((size_t)(m + 1) * csz);
    y = o;   o += al16((size_t)m * csz);
    hv = o;  o += al16((size_t)(m + 2) * csz);
    cs = o;  o += al16((size_t)m * rsz);
    soff = o; o += al16(rows * 9 * sizeof(int));
    sw = o;  o += al16(rows * csz);
    sx = o;  o += al16(rows * 9 * csz);
    sV = o;  if (v_in) o += al16((size_t)(m + 1) * rows * csz);
    sOp = o; if (op_in) o += al16(rows * 9 * n2k * csz);
    total = o;
  }
};

template <typename R>
__global__ void __launch_bounds__(CT) coarse_gmres_kernel(CArgs<R> a) {
  typedef cplx<R> C;
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ uint64_t obar;
  __shared__ int s_done;
  const int m = a.m;
  const int n2k = a.n2k;
  const int spc = a.spc;
  const CLayout Lo(m, spc, n2k, (int)sizeof(C), a.v_in_smem, a.op_in_smem);
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dyn) + 15) & ~(uintptr_t)15);   // the host reserves 16 bytes
  C* H = reinterpret_cast<C*>(base + Lo.H);        // [(m+1) x m] column-major
  C* sn = reinterpret_cast<C*>(base + Lo.sn);      // [m]
  C* g = reinterpret_cast<C*>(base + Lo.g);        // [m+1]
  C* y = reinterpret_cast<C*>(base + Lo.y);        // [m]
  C* hv = reinterpret_cast<C*>(base + Lo.hv);      // [m+2] reduced values
  R* cs = reinterpret_cast<R*>(base + Lo.cs);      // [m]
  int* soff = reinterpret_cast<int*>(base + Lo.soff);   // [spc][9][n2k] source row of sx
  C* sw = reinterpret_cast<C*>(base + Lo.sw);      // [rows] this CTA's rows of w
  C* sx = reinterpret_cast<C*>(base + Lo.sx);      // [spc][9][n2k] staged neighbour rows
  C* sV = reinterpret_cast<C*>(base + Lo.sV);      // [(m+1)][rows] if v_in_smem
  C* sOp = reinterpret_cast<C*>(base + Lo.sOp);    // [spc][9][n2k][n2k] if op_in_smem

  const int d = a.B.d;
  const size_t nc = (size_t)d * n2k;
  const int j0 = blockIdx.x * spc;
  const int j1 = min(d, j0 + spc);
  const int row0 = j0 * n2k, row1 = j1 * n2k;
  const int nrows = row1 > row0 ? row1 - row0 : 0;
  const int nloc = j1 > j0 ? j1 - j0 : 0;
  const int ne = nloc * 9 * n2k;
  const size_t blk_el = (size_t)n2k * n2k;
  const int stride = 2 * (m + 2);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // G threads share one row of the stencil apply (consecutive lanes)
  const int G = nrows * 8 <= CT ? 8 : nrows * 4 <= CT ? 4 : nrows * 2 <= CT ? 2 : 1;
  // basis row rl (local) of vector i
  C* const Vb = a.v_in_smem ? sV : a.V + row0;
  const size_t vs = a.v_in_smem ? (size_t)spc * n2k : nc;
  // Reduction number `red` writes buffer red % 2.  Its readers finish before they arrive at
  // the barrier of reduction red + 1, and reduction red + 2 writes only after that barrier.
  int red = 0;
  unsigned epoch = 0;

  // ---- operator slice: this CTA's coarse sites are contiguous in Op, bulk-copied once
  const uint32_t op_bytes = (uint32_t)((size_t)nloc * 9 * blk_el * sizeof(C));
  if (threadIdx.x == 0 && a.op_in_smem) {
    mbar_init(&obar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (a.op_in_smem && threadIdx.x == 0 && op_bytes > 0) {
    const char* src = reinterpret_cast<const char*>(a.Op + (size_t)j0 * 9 * blk_el);
    char* dst = reinterpret_cast<char*>(sOp);
    mbar_arrive_expect_tx(&obar, op_bytes);
    for (uint32_t o = 0; o < op_bytes; o += OP_CHUNK)
      bulk_g2s(dst + o, src + o, min(OP_CHUNK, op_bytes - o), &obar);
  }
  // source row of every staged neighbour element
  for (int e = threadIdx.x; e < ne; e += CT) {
    int jl = e / (9 * n2k), rem = e - jl * 9 * n2k;
    int blk = rem / n2k, bb = rem - blk * n2k;
    int j = j0 + jl;
    int s = blk == 0 ? j : a.B.coarse_nbr(j, blk - 1);
    soff[e] = s * n2k + bb;
  }

  auto fail_out = [&]() {
    if (threadIdx.x == 0) *(volatile int*)a.err = 1;
  };

  // Inner products of this CTA's rows: slot i < cnt gets V_i^dag w, slot cnt (if nrm) ||w||^2
  // (w staged in sw).  One warp per slot; the grid sum lands in hv[0 .. cnt + nrm).
  auto reduce = [&](int cnt, bool nrm) -> bool {
    R* buf = a.partial + (size_t)(red & 1) * gridDim.x * stride;
    const int tot = cnt + (nrm ? 1 : 0);
    for (int i = wid; i < tot; i += NW) {
      R ar = 0, ai = 0;
      if (i < cnt) {
        const C* Vi = Vb + (size_t)i * vs;
        for (int rl = lane; rl < nrows; rl += 32) {
          C v = Vi[rl], w = sw[rl];
          ar = fma(v.re, w.re, ar);
          ar = fma(v.im, w.im, ar);
          ai = fma(v.re, w.im, ai);
          ai = fma(-v.im, w.re, ai);
        }
      } else {
        for (int rl = lane; rl < nrows; rl += 32) {
          C w = sw[rl];
          ar = fma(w.re, w.re, ar);
          ar = fma(w.im, w.im, ar);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ar += __shfl_down_sync(0xffffffffu, ar, o);
        ai += __shfl_down_sync(0xffffffffu, ai, o);
      }
      if (lane == 0) {
        buf[(size_t)blockIdx.x * stride + 2 * i] = ar;
        buf[(size_t)blockIdx.x * stride + 2 * i + 1] = ai;
      }
    }
    if (!grid_barrier(a.bar, gridDim.x, epoch)) {
      fail_out();
      return false;
    }
    for (int i = wid; i < tot; i += NW) {
      R t0[MAXG], t1[MAXG];
#pragma unroll
      for (int u = 0; u < MAXG; ++u) {
        int c = lane + 32 * u;
        bool in = c < (int)gridDim.x;
        t0[u] = in ? __ldcg(buf + (size_t)c * stride + 2 * i) : (R)0;
        t1[u] = in ? __ldcg(buf + (size_t)c * stride + 2 * i + 1) : (R)0;
      }
      R s0 = 0, s1 = 0;
#pragma unroll
      for (int u = 0; u < MAXG; ++u) {
        s0 += t0[u];
        s1 += t1[u];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
      }
      if (lane == 0) hv[i] = {s0, s1};
    }
    __syncthreads();
    ++red;
    return true;
  };

  // stage a register vector (rows of this thread) into sw
  auto stage_w = [&](const C v[RPT]) {
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      int rl = threadIdx.x + q * CT;
      if (rl < nrows) sw[rl] = v[q];
    }
    __syncthreads();
  };

  // out = scale * A src for this thread's rows, also left in sw.  The nine neighbour rows of
  // every local coarse site are staged in shared memory first; G lanes share a row.
  auto apply = [&](C out[RPT], const C* src, R scale) {
    for (int e0 = threadIdx.x; e0 < ne; e0 += 4 * CT) {
      C v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int e = e0 + u * CT;
        if (e < ne) v[u] = ldcg_c(src + soff[e]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (e0 + u * CT < ne) sx[e0 + u * CT] = v[u];
    }
    __syncthreads();
    const int nwork = nrows * G;
    const C* Obase = a.op_in_smem ? sOp : a.Op + (size_t)j0 * 9 * blk_el;
    for (int tb = wid * 32; tb < nwork; tb += CT) {
      int t = tb + lane;
      bool act = t < nwork;
      int rl = t / G, part = t - rl * G;
      C acc0 = {0, 0}, acc1 = {0, 0};
      if (act) {
        int jl = rl / n2k, aa = rl - jl * n2k;
        const C* O = Obase + (size_t)jl * 9 * blk_el + aa;
        const C* xs = sx + (size_t)jl * 9 * n2k;
        for (int blk = 0; blk < 9; ++blk) {
          int bb = part;
          for (; bb + G < n2k; bb += 2 * G) {
            cfma(acc0, O[(size_t)bb * n2k], xs[bb]);
            cfma(acc1, O[(size_t)(bb + G) * n2k], xs[bb + G]);
          }
          if (bb < n2k) cfma(acc0, O[(size_t)bb * n2k], xs[bb]);
          O += blk_el;
          xs += n2k;
        }
      }
      R re = acc0.re + acc1.re, im = acc0.im + acc1.im;
      for (int o = G >> 1; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (act && part == 0) sw[rl] = {scale * re, scale * im};
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      int rl = threadIdx.x + q * CT;
      out[q] = rl < nrows ? sw[rl] : C{0, 0};
    }
  };

  // ---- x = 0, r = b, beta = ||b||
  C rr[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    int rl = threadIdx.x + q * CT;
    if (rl < nrows) {
      a.x[row0 + rl] = {0, 0};
      rr[q] = a.b[row0 + rl];
    } else {
      rr[q] = {0, 0};
    }
  }
  stage_w(rr);
  bool ok = reduce(0, true);
  // the operator slice must have landed before the first apply (and before any return)
  if (a.op_in_smem && op_bytes > 0) {
    bool got = mbar_wait(&obar, 0, OP_WAIT);
    if (!__syncthreads_and(got)) {
      if (threadIdx.x == 0) {
        *(volatile int*)a.err = 1;
        atomicExch(&a.bar->err, 1);   // the other CTAs' barrier waits return
        mbar_wait(&obar, 0, OP_WAIT);
      }
      return;
    }
  }
  if (!ok) return;
  const R bnorm = sqrt(hv[0].re);
  const R target = (R)a.rtol * bnorm;
  const R target2 = target * target;
  int its = 0;
  R beta = bnorm;
  bool converged = !(bnorm > target);
  C w[RPT];
  while (!converged && its < a.maxiter) {
    // W = r (raw), V0 = r / beta
    const R f0 = beta > 0 ? (R)1 / beta : (R)0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      int rl = threadIdx.x + q * CT;
      if (rl < nrows) {
        a.W[row0 + rl] = rr[q];
        Vb[rl] = f0 * rr[q];
      }
    }
    for (int i = threadIdx.x; i < (m + 1) * m; i += CT) H[i] = {0, 0};
    for (int i = threadIdx.x; i <= m; i += CT) g[i] = {0, 0};
    if (threadIdx.x == 0) g[0] = {beta, 0};
    if (!grid_barrier(a.bar, gridDim.x, epoch)) { fail_out(); return; }
    R wscale = f0;   // V_j = W * wscale
    int steps = 0;
    for (int jj = 0; jj < m && its < a.maxiter; ++jj) {
      // w = A V_jj = (A W) * wscale, already staged in sw
      apply(w, a.W, wscale);
      // CGS pass 1 and 2: h = V^dag w, w -= V h, H[:, jj] += h
      for (int pass = 0; pass < 2; ++pass) {
        if (pass) stage_w(w);
        if (!reduce(jj + 1, false)) return;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          int rl = threadIdx.x + q * CT;
          if (rl < nrows) {
            C t = w[q];
            for (int i = 0; i <= jj; ++i) t -= hv[i] * Vb[(size_t)i * vs + rl];
            w[q] = t;
          }
        }
        if (threadIdx.x <= jj) H[(size_t)jj * (m + 1) + threadIdx.x] += hv[threadIdx.x];
      }
      // raw next direction for the neighbours (visible after the norm's barrier), its norm
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        int rl = threadIdx.x + q * CT;
        if (rl < nrows) a.W[row0 + rl] = w[q];
      }
      stage_w(w);
      if (!reduce(0, true)) return;
      const R nrm2 = hv[0].re;
      const R f = nrm2 > 0 ? rsqrt(nrm2) : (R)0;   // 1 / ||w||
      // V_{jj+1} rows (private) and the Givens update (identical in every CTA)
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        int rl = threadIdx.x + q * CT;
        if (rl < nrows) Vb[(size_t)(jj + 1) * vs + rl] = f * w[q];
      }
      if (threadIdx.x == 0) {
        const R hn = nrm2 * f;
        C* col = H + (size_t)jj * (m + 1);
        for (int i = 0; i < jj; ++i) {
          R c = cs[i];
          C sv = sn[i];
          C x0 = col[i], x1 = col[i + 1];
          col[i] = c * x0 + sv * x1;
          col[i + 1] = c * x1 - cmulc(sv, x0);
        }
        // rotation zeroing H[jj+1, jj] = hn (real): c = |a| / rho, s = (a / |a|) hn / rho
        C a0 = col[jj];
        R na2 = norm2(a0);
        R rho2 = na2 + hn * hn;
        R c;
        C sv;
        if (!(rho2 > 0)) { c = 1; sv = {0, 0}; }
        else if (!(na2 > 0)) { c = 0; sv = {hn * rsqrt(rho2), 0}; }
        else {
          R ir = rsqrt(rho2), ina = rsqrt(na2);
          c = na2 * ina * ir;
          R t = hn * ir * ina;
          sv = {a0.re * t, a0.im * t};
        }
        col[jj] = c * a0 + hn * sv;
        col[jj + 1] = {0, 0};
        cs[jj] = c;
        sn[jj] = sv;
        C gj = g[jj];
        g[jj] = c * gj;
        g[jj + 1] = -cmulc(sv, gj);
        s_done = norm2(g[jj + 1]) <= target2;
      }
      __syncthreads();
      wscale = f;
      ++steps;
      ++its;
      if (s_done) break;
    }
    // y = R^{-1} g ; x += V y
    if (threadIdx.x == 0) {
      for (int i = steps - 1; i >= 0; --i) {
        C acc = g[i];
        for (int k = i + 1; k < steps; ++k) acc = acc - H[(size_t)k * (m + 1) + i] * y[k];
        C dd = H[(size_t)i * (m + 1) + i];
        R n2 = norm2(dd);
        y[i] = n2 > 0 ? ((R)1 / n2) * cmulc(dd, acc) : C{0, 0};
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      int rl = threadIdx.x + q * CT;
      if (rl < nrows) {
        C t = a.x[row0 + rl];
        for (int i = 0; i < steps; ++i) t += y[i] * Vb[(size_t)i * vs + rl];
        a.x[row0 + rl] = t;
      }
    }
    if (!grid_barrier(a.bar, gridDim.x, epoch)) { fail_out(); return; }
    // true residual r = b - A x
    apply(rr, a.x, (R)1);
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      int rl = threadIdx.x + q * CT;
      if (rl < nrows) rr[q] = a.b[row0 + rl] - rr[q];
    }
    stage_w(rr);
    if (!reduce(0, true)) return;
    beta = sqrt(hv[0].re);
    converged = !(beta > target);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.its_acc, its);
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
  if (max_grid > 32 * MAXG) max_grid = 32 * MAXG;
  WMG_TRY(dev_alloc(&V, sizeof(cplx<R>) * nc * (m + 1)));
  WMG_TRY(dev_alloc(&W, sizeof(cplx<R>) * nc));
  WMG_TRY(dev_alloc(&partial, sizeof(R) * 2 * 2 * (m + 2) * max_grid));
  // barrier state, then the iteration accumulator
  WMG_TRY(dev_alloc(&state, sizeof(BarrierState) + 2 * sizeof(int)));
  WMG_CUDA(cudaMemset(state, 0, sizeof(BarrierState) + 2 * sizeof(int)));
  WMG_TRY(host_alloc(&host_state, 2 * sizeof(int)));
  return MG_OK;
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
                           const cplx<R>* b, double rtol, int restart, int maxiter,
                           cudaStream_t st) {
  if (restart > m) return fail(MG_EINVAL, "coarse solver: restart longer than allocated");
  int* err = device_error_word();
  if (!err) return fail(MG_ECUDA, "coarse solver: no error word");
  int n2k = 2 * k;
  // one CTA per SM (at most one per coarse site), whole coarse sites per CTA
  int grid = max_grid < B.d ? max_grid : B.d;
  int spc = (B.d + grid - 1) / grid;
  grid = (B.d + spc - 1) / spc;
  if ((long long)spc * n2k > (long long)CT * RPT)
    return fail(MG_EINVAL, "coarse solver: coarse system too large for one cooperative grid");
  // the basis rows and the operator slice go to shared memory when they fit
  const size_t cap = (size_t)227 * 1024 - 64 - 16;   // per CTA, less the statics and the pad
  const int csz = (int)sizeof(cplx<R>);
  int op_in_smem = 0, v_in_smem = 0;
  if (CLayout(restart, spc, n2k, csz, 0, 1).total <= cap && reinterpret_cast<uintptr_t>(Op) % 16 == 0)
    op_in_smem = 1;
  if (CLayout(restart, spc, n2k, csz, 1, op_in_smem).total <= cap) v_in_smem = 1;
  size_t sh = CLayout(restart, spc, n2k, csz, v_in_smem, op_in_smem).total + 16;
  WMG_TRY(smem_attr(coarse_gmres_kernel<R>, sh));
  int per_sm = 0;
  WMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_gmres_kernel<R>, CT, sh));
  if (per_sm < 1 || grid > per_sm * num_sms())
    return fail(MG_ECUDA, "coarse solver: grid cannot be co-resident");
  BarrierState* bs = reinterpret_cast<BarrierState*>(state);
  int* its_acc = reinterpret_cast<int*>(bs + 1);
  WMG_CUDA(cudaMemsetAsync(state, 0, sizeof(BarrierState), st));
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
  args.its_acc = its_acc;
  args.err = err;
  args.rtol = rtol;
  args.m = restart;
  args.maxiter = maxiter;
  args.spc = spc;
  args.op_in_smem = op_in_smem;
  args.v_in_smem = v_in_smem;
  void* kargs[] = {&args};
  ProfScope ps("coarse_gmres", (double)sizeof(cplx<R>) * B.d * 9.0 * n2k * n2k, 0.0, st);
  WMG_CUDA(cudaLaunchCooperativeKernel((void*)coarse_gmres_kernel<R>, dim3(grid), dim3(CT), kargs,
                                       sh, st));
  count_launch();
  return MG_OK;
}

template <typename R>
int CoarseSolver<R>::take_iterations(long long* its, cudaStream_t st) {
  if (!state) {
    if (its) *its = 0;
    return MG_OK;
  }
  int* its_acc = reinterpret_cast<int*>(reinterpret_cast<BarrierState*>(state) + 1);
  int* h = reinterpret_cast<int*>(host_state);
  WMG_CUDA(cudaMemcpyAsync(h, its_acc, sizeof(int), cudaMemcpyDeviceToHost, st));
  WMG_CUDA(cudaMemsetAsync(its_acc, 0, sizeof(int), st));
  WMG_CUDA(cudaStreamSynchronize(st));
  if (its) *its = h[0];
  return MG_OK;
}

// Diagnostic: a grid barrier that waits for one more CTA than the grid has, so every wait
// runs out.  Exercises the bounded-wait error path without faulting or hanging the GPU.
__global__ void barrier_timeout_kernel(BarrierState* bs, long long limit) {
  unsigned epoch = 0;
  grid_barrier(bs, gridDim.x + 1, epoch, limit);
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
