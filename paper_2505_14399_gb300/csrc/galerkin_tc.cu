// Forward-hop blocks of the Galerkin coarse operator (Eq. 5) on the tensor pipe, at
// double-float accuracy.
//
// CTA (j, mu) accumulates, over the fine sites x of aggregate j, C[a][b] =
// sum_{x,r} conj(Pt[x][r][a]) Ch[x][r][b] (the staged reconstruction-folded P(x) and the
// spin-projected, colour-transported P(x + mu), as in the FP32-unit kernel of coarse.cu).
// Every staged double-float entry v satisfies |v| < 2 (|P| <= 1 entrywise for orthonormal
// columns; |U h| <= sqrt(3) for unitary U and |h| <= 1), so it is written exactly enough as
// fixed-point digits in base 256,
//     v = sum_{i < NS} s_i 2^{-6-8i},  s_i integers, |s_i| <= 129,  NS = 7
// (error at most 2^-55 (1 + 2^-16)),
// each digit exact in bfloat16.  A product of digit planes is an integer matrix product:
// bf16 x bf16 tensor-core MMAs with FP32 accumulation are exact while the partial sums stay
// below 2^24, which holds for one staging batch (<= 7 digit pairs x 96 stacked rows x 129^2).
// Digit pairs i + j = d of the same weight 2^{-12-8d} share an FP32 accumulator; pairs with
// i + j >= NS (weight below 2^-68) are dropped.  After every batch the exact FP32 sums are
// scaled by their weights (exact) and added to double-float accumulators with error-free
// two-sums, so the result carries double-float accuracy (~2^-48 relative), not bf16's.
//
// The complex product is one real GEMM per digit pair: with K = 6 NB rows (NB sites x 6 half-
// spinor rows) per batch, stacked as k' = [re rows | im rows] (12 NB),
//     A'[b'][k'] : rows b < 2k = (Ch_re | Ch_im), rows 2k + b = (Ch_im | -Ch_re),
//     B'[a][k']  : (Pt_re | Pt_im),
// C'[b'][a] = sum_k' A'[b'][k'] B'[a][k'] gives Re C[a][b] (b' = b) and Im C[a][b] (b' = 2k+b).
// mma.sync m16n8k16 (row.col) tiles: 16 rows b' x 8 columns a, one warp per tile.  The digit
// planes are stored k'-major (SA[k'][b'], SB[k'][a]) so that staging threads with consecutive
// columns write consecutive addresses, and read with ldmatrix .trans; every row stride is an
// odd number of 16-byte units, so the eight rows of an ldmatrix phase hit distinct banks.
// A batch is NB = 4 sites (one warp group, three k' steps) or, for 2k <= 24, NB = 8 sites (two
// warp groups split its six 16-row k' steps; the digit planes and the double-buffered raw
// inputs of one CTA then take ~195 KB, one CTA per SM).  At 4 sites a CTA fits its shared
// memory up to the paper's k = 24, and for 2k <= 24 two CTAs share an SM, so one CTA's staging
// overlaps the other's products; the autotuner picks between the two where both fit.
#include <cuda_bf16.h>

#include "common.cuh"
#include "df64.cuh"
#include "galerkin.cuh"
#include "internal.h"
#include "tcdigits.cuh"
#include "tma.cuh"

namespace wmg {

namespace {

constexpr int TC_MAXT4 = 6;            // 2k <= 48

// Per column-tile count T4 (2k <= 8 T4) and sites per batch NB_ (8 or 4): stacked rows, warp
// groups, warps.
template <int T4, int NB_>
struct TcCfg {
  static constexpr int NB = NB_;                       // fine sites staged per batch
  static constexpr int KB = NB * 6;                    // staged rows per batch
  static constexpr int K = 2 * KB;                     // stacked real rows (96 or 48)
  static constexpr int WG = (K / 16) % 2 == 0 ? 2 : 1; // warp groups (each takes k' steps)
  static constexpr int NTILES = T4 * T4;
  // warps per group: at most 12 (two groups) or 16 (one group), tiles spread evenly
  static constexpr int MAXW = WG == 2 ? 12 : 16;
  static constexpr int TPW = (NTILES + MAXW - 1) / MAXW;   // tiles per warp
  static constexpr int NW = (NTILES + TPW - 1) / TPW;
  // resident CTAs per SM asked of the register allocator: two for 4-site batches of 2k <= 24
  // (about 100 KB of shared memory each), whose staging and products then overlap
  static constexpr int MINB = (NB == 4 && T4 <= 3) ? 2 : 1;
};

// Row strides (bf16) of the k'-major digit planes: odd multiples of 8 (16 bytes).
__host__ __device__ constexpr int tc_lda(int t4) { return 16 * t4 + 8; }
__host__ __device__ constexpr int tc_ldb(int t4) { return 8 * t4 + ((t4 & 1) ? 0 : 8); }
__host__ __device__ constexpr size_t tc_smem(int t4, int nb) {
  return sizeof(__nv_bfloat16) * (size_t)TC_NS * 12 * nb * (tc_lda(t4) + tc_ldb(t4));
}

// Shared memory of one CTA beyond the digit planes: two raw input buffers (P(x + mu) and P(x)
// column segments of 6 double-float values, U_mu(x)) and the per-site tables.
// Raw P segments are stored [site][6 components][column slot], rows padded to 8 T4 + 1 slots
// so that the copies (consecutive components of one column) spread over the banks; column b
// sits in slot (b odd ? k : 0) + b / 2, so that the staging threads, which take the column
// pairs (2q, 2q + 1) for consecutive q, read consecutive 16-byte slots.
__host__ __device__ constexpr int tc_nrp(int t4) { return 8 * t4 + 1; }
__host__ __device__ constexpr size_t tc_raw_bytes(int t4, int nb) {
  return sizeof(zdf) * 2 * ((size_t)2 * nb * 6 * tc_nrp(t4) + nb * 9);
}
__host__ __device__ inline size_t tc_table_bytes(int nd) { return sizeof(int) * 8 * (size_t)nd + 16; }
__host__ __device__ inline size_t tc_cta_bytes(int t4, int nb, int nd) {
  return tc_smem(t4, nb) + tc_raw_bytes(t4, nb) + tc_table_bytes(nd);
}
template <int T4, int NB_>
__global__ void __launch_bounds__(32 * TcCfg<T4, NB_>::WG * TcCfg<T4, NB_>::NW,
                                  TcCfg<T4, NB_>::MINB)
galerkin_tc_kernel(zd* Op, zd* Xpart, const zdf* __restrict__ Pdf, int k,
                   const zdf* __restrict__ Ldf, HopGeom g, Blocking B, int* range_flag) {
  using C = TcCfg<T4, NB_>;
  constexpr int NR = 8 * T4;                  // columns a (>= 2k)
  constexpr int NTILES = C::NTILES;
  constexpr int NW = C::NW;
  constexpr int TPW = C::TPW;                 // tiles per warp
  constexpr int NB = C::NB, KB = C::KB, K = C::K, WG = C::WG;
  constexpr int ND = TC_NS;                   // digit-pair weights d = i + j < NS
  constexpr int LDA = tc_lda(T4), LDB = tc_ldb(T4);
  extern __shared__ __align__(16) unsigned char tc_raw[];
  __nv_bfloat16* SA = reinterpret_cast<__nv_bfloat16*>(tc_raw);   // [NS][K][LDA]
  __nv_bfloat16* SB = SA + (size_t)TC_NS * K * LDA;                // [NS][K][LDB]
  constexpr int NRP = tc_nrp(T4);
  zdf* sPy = reinterpret_cast<zdf*>(tc_raw + tc_smem(T4, NB));     // [2][NB][6][NRP]
  zdf* sPx = sPy + (size_t)2 * NB * 6 * NRP;                       // [2][NB][6][NRP]
  zdf* sU = sPx + (size_t)2 * NB * 6 * NRP;                        // [2][NB][9]
  const int nd = B.nd;
  int* tx = reinterpret_cast<int*>(tc_raw + tc_smem(T4, NB) + tc_raw_bytes(T4, NB));   // site x
  int* toy = tx + nd;      // P offset of (2 j(y)) k M, y = x + mu
  int* tox = toy + nd;     // P offset of (2 j(x)) k M
  int* tly = tox + nd;     // local site of y, x
  int* tlx = tly + nd;
  int* tng = tlx + nd;     // antiperiodic sign of the hop
  int* sel = tng + nd;     // [2][nd]: local sites of pass 0, then of pass 1
  __shared__ int nsel[2];
  const int n2k = 2 * k;
  const int j = blockIdx.x, mu = blockIdx.y, dir = 2 * mu;
  const double coef = -g.kappa * g.w[mu];
  const int ne = n2k * n2k;
  const int M = B.M;
  const size_t V = (size_t)B.nd * B.d;
  const int lane = threadIdx.x & 31;
  const int wid = (threadIdx.x >> 5) % NW, grp = (threadIdx.x >> 5) / NW;   // tile slot, k' half
  const size_t plane16 = tc_smem(T4, NB) / 16;   // 16-byte chunks of SA + SB
  bool bad = false;

  // ---- per-site tables of this aggregate, and the two passes' site lists
  for (int l = threadIdx.x; l < nd; l += blockDim.x) {
    int x = B.site(j, l);
    int c[4];
    c[0] = x % g.L[0];
    int r = x / g.L[0];
    c[1] = r % g.L[1]; r /= g.L[1];
    c[2] = r % g.L[2]; c[3] = r / g.L[2];
    bool wrap = c[mu] == g.L[mu] - 1;
    int y = wrap ? x - (g.L[mu] - 1) * g.stride[mu] : x + g.stride[mu];
    int jy, ly, jx, lx;
    B.block_of(y, &jy, &ly);
    B.block_of(x, &jx, &lx);
    tx[l] = x;
    toy[l] = 2 * jy * k * M;
    tox[l] = 2 * jx * k * M;
    tly[l] = ly;
    tlx[l] = lx;
    tng[l] = (wrap && g.bc[mu] < 0) ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // a hop crosses the aggregate when the local coordinate mu is the last one
    int n0 = 0, n1 = 0;
    const int bm = B.b[mu];
    int stride = 1;
    for (int m = 0; m < mu; ++m) stride *= B.b[m];
    for (int l = 0; l < nd; ++l) {
      bool cross = (l / stride) % bm == bm - 1;
      if (cross) sel[nd + n1++] = l;
      else sel[n0++] = l;
    }
    nsel[0] = n0;
    nsel[1] = n1;
  }
  __syncthreads();

  const int pps = 2 * n2k * 6 + 9;   // 16-byte pieces per site (one double-float complex each)
  // q / pps as a multiply-high: with m = ceil(2^32 / pps), floor(q m / 2^32) = floor(q / pps)
  // whenever q pps < 2^32 (here q < NB pps and pps <= 585)
  const unsigned pps_m = 0xffffffffu / (unsigned)pps + 1u;
  // staging assignment: thread -> column pair sq of staged rows srow0, srow0 + srows, ...
  // (threads beyond srows * k stage nothing)
  const int srows = blockDim.x / k;
  const int sq = threadIdx.x % k;
  const int srow0 = threadIdx.x < srows * k ? threadIdx.x / k : 6 * NB;
  // issue the raw inputs of batch b of pass p into buffer buf (cp.async, one group)
  auto prefetch = [&](int p, int b, int buf) {
    const int* ls = sel + p * nd;
    const int h0 = b * NB;
    const int nb = min(NB, nsel[p] - h0);
    for (int q = threadIdx.x; q < nb * pps; q += blockDim.x) {
      int h = (int)__umulhi((unsigned)q, pps_m), rem = q - h * pps;
      int l = ls[h0 + h];
      const zdf* src;
      zdf* dst;
      if (rem < n2k * 6) {
        int bcol = rem / 6, part = rem - bcol * 6;
        src = Pdf + (size_t)toy[l] + (size_t)bcol * M + tly[l] * 6 + part;
        dst = sPy + (((size_t)buf * NB + h) * 6 + part) * NRP + ((bcol & 1) ? k : 0) + (bcol >> 1);
      } else if (rem < 2 * n2k * 6) {
        rem -= n2k * 6;
        int bcol = rem / 6, part = rem - bcol * 6;
        src = Pdf + (size_t)tox[l] + (size_t)bcol * M + tlx[l] * 6 + part;
        dst = sPx + (((size_t)buf * NB + h) * 6 + part) * NRP + ((bcol & 1) ? k : 0) + (bcol >> 1);
      } else {
        int part = rem - 2 * n2k * 6;
        src = Ldf + ((size_t)mu * V + tx[l]) * 9 + part;
        dst = sU + ((size_t)buf * NB + h) * 9 + part;
      }
      cp_async16(dst, src);
    }
    cp_async_commit();
  };

  for (int pass = 0; pass < 2; ++pass) {  // 0: hops inside the aggregate, 1: crossing hops
    // zero both digit planes: padding rows and columns stay zero for the whole pass
    for (size_t e = threadIdx.x; e < plane16; e += blockDim.x)
      reinterpret_cast<uint4*>(tc_raw)[e] = make_uint4(0u, 0u, 0u, 0u);
    dfacc dacc[TPW][4];
#pragma unroll
    for (int t = 0; t < TPW; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) dacc[t][e] = {0.0f, 0.0f};
    const int nbat = (nsel[pass] + NB - 1) / NB;
    if (nbat > 0) prefetch(pass, 0, 0);
    for (int b = 0; b < nbat; ++b) {
      const int buf = b & 1;
      if (b + 1 < nbat) {
        prefetch(pass, b + 1, buf ^ 1);   // its buffer was last read by batch b - 1's staging
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();   // batch b's inputs are in; every warp finished batch b - 1's products
      const int nb = min(NB, nsel[pass] - b * NB);
      const int* ls = sel + pass * nd + b * NB;
      if (nb < NB) {
        // a short batch: its unused stacked rows k' are zero in every digit plane
        const int k0 = nb * 6, kn = KB - k0;
        for (int e = threadIdx.x; e < TC_NS * 2 * kn * (LDA + LDB); e += blockDim.x) {
          int col = e % (LDA + LDB), rr = e / (LDA + LDB);
          int i = rr / (2 * kn), q = rr % (2 * kn);
          int kk = (q < kn) ? k0 + q : KB + k0 + (q - kn);
          if (col < LDA) SA[((size_t)i * K + kk) * LDA + col] = __float2bfloat16_rn(0.0f);
          else SB[((size_t)i * K + kk) * LDB + (col - LDA)] = __float2bfloat16_rn(0.0f);
        }
      }
      // stage from shared memory: Ch (spin-projected, transported P(x + mu)) and Pt
      // (reconstruction-folded P(x)) in double-float, written as digit planes; a thread takes
      // the adjacent columns 2q and 2q + 1 of one row, so every digit goes out as a packed
      // bf16 pair (one 32-bit store)
      const zdf* py = sPy + (size_t)buf * NB * 6 * NRP;
      const zdf* px = sPx + (size_t)buf * NB * 6 * NRP;
      const zdf* pu = sU + (size_t)buf * NB * 9;
      for (int rr = srow0; rr < nb * 6; rr += srows) {
        const int h = rr / 6, r = rr - 6 * (rr / 6);
        const int q = sq;
        const int s = r / 3, cc = r - 3 * s;
        const zdf* U = pu + h * 9 + cc * 3;
        const zdf u0 = U[0], u1 = U[1], u2 = U[2];
        const bool neg = tng[ls[h]] != 0;
        float cr[2][TC_NS], ci[2][TC_NS], tr[2][TC_NS], ti[2][TC_NS];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int bcol = 2 * q + u;
          const int beta = bcol >= k;
          // component q' of this column at this site: P*[q' * NRP] (slot u k + q)
          const zdf* Py = py + (size_t)h * 6 * NRP + u * k + q;
          const zdf* Px = px + (size_t)h * 6 * NRP + u * k + q;
          zdf hv[3];
#pragma unroll
          for (int c2 = 0; c2 < 3; ++c2) {
            if (beta == 0) {
              hv[c2] = Py[(s * 3 + c2) * NRP];
            } else {
              zdf p0 = Py[c2 * NRP], p1 = Py[(3 + c2) * NRP];
              hv[c2] = mu < 3 ? isigma_df(mu, s, p0, p1) : zdf_neg(s == 0 ? p0 : p1);
            }
          }
          zdfacc t{};
          zdf_fma(t, u0, hv[0]);
          zdf_fma(t, u1, hv[1]);
          zdf_fma(t, u2, hv[2]);
          zdf ch = zdf_norm(t);
          if (neg) ch = zdf_neg(ch);
          zdf pt;
          if (beta == 0) {
            pt = Px[(s * 3 + cc) * NRP];
          } else {
            zdf p0 = Px[cc * NRP], p1 = Px[(3 + cc) * NRP];
            pt = mu < 3 ? isigma_df(mu, s, p0, p1) : zdf_neg(s == 0 ? p0 : p1);
          }
          bad |= !(tc_in_range(ch.re) && tc_in_range(ch.im) && tc_in_range(pt.re) &&
                   tc_in_range(pt.im));
          tc_digits(ch.re, cr[u]);
          tc_digits(ch.im, ci[u]);
          tc_digits(pt.re, tr[u]);
          tc_digits(pt.im, ti[u]);
        }
        const int kk = h * 6 + r;
#pragma unroll
        for (int i = 0; i < TC_NS; ++i) {
          __nv_bfloat16* a0 = SA + ((size_t)i * K + kk) * LDA;          // re rows k
          __nv_bfloat16* a1 = SA + ((size_t)i * K + KB + kk) * LDA;     // im rows k
          const unsigned pr = tc_pack(cr[0][i], cr[1][i]), pi = tc_pack(ci[0][i], ci[1][i]);
          *reinterpret_cast<unsigned*>(a0 + 2 * q) = pr;
          *reinterpret_cast<unsigned*>(a1 + 2 * q) = pi;
          *reinterpret_cast<unsigned*>(a0 + n2k + 2 * q) = pi;
          *reinterpret_cast<unsigned*>(a1 + n2k + 2 * q) = pr ^ 0x80008000u;   // -Ch_re
          *reinterpret_cast<unsigned*>(SB + ((size_t)i * K + kk) * LDB + 2 * q) =
              tc_pack(tr[0][i], tr[1][i]);
          *reinterpret_cast<unsigned*>(SB + ((size_t)i * K + KB + kk) * LDB + 2 * q) =
              tc_pack(ti[0][i], ti[1][i]);
        }
      }
      __syncthreads();
      // exact digit-plane products of this warp's output tiles, folded into double-float
#pragma unroll
      for (int tt = 0; tt < TPW; ++tt) {
        const int tile = wid + tt * NW;
        if (tile < NTILES) {
          const int mt = tile / T4, nt = tile % T4;
          float acc[ND][4];
#pragma unroll
          for (int d = 0; d < ND; ++d)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[d][e] = 0.0f;
          // ldmatrix .trans row addresses: A matrices (b' 0-7 | 8-15) x (k 0-7 | 8-15) in the
          // order of the A fragment, B matrices k 0-7 | 8-15 for columns a of this tile
          const int mq = lane >> 3, rr = lane & 7;
          const __nv_bfloat16* arow = SA + (size_t)(8 * (mq >> 1) + rr) * LDA + 16 * mt + 8 * (mq & 1);
          const __nv_bfloat16* brow = SB + (size_t)(8 * (mq & 1) + rr) * LDB + 8 * nt;
#pragma unroll 1
          for (int ks = grp * (K / 16 / WG); ks < (grp + 1) * (K / 16 / WG); ++ks) {
            unsigned bfr[TC_NS][2];
#pragma unroll
            for (int i = 0; i < TC_NS; ++i)
              ldm_x2t(bfr[i], brow + ((size_t)i * K + 16 * ks) * LDB);
#pragma unroll
            for (int i = 0; i < TC_NS; ++i) {
              unsigned af[4];
              ldm_x4t(af, arow + ((size_t)i * K + 16 * ks) * LDA);
#pragma unroll
              for (int jd = 0; jd < TC_NS; ++jd)
                if (i + jd < ND) mma_bf16(acc[i + jd], af, bfr[jd]);
            }
          }
          // weights 2^{-12-8d}: exact FP32 constants
          float wgt = 1.0f / 4096.0f;
#pragma unroll
          for (int d = 0; d < ND; ++d) {
#pragma unroll
            for (int e = 0; e < 4; ++e) acc_add(dacc[tt][e], acc[d][e] * wgt);
            wgt *= 1.0f / 256.0f;
          }
        }
      }
    }
    // this pass's blocks: tiles -> shared memory (over the digit planes) -> Op / Xpart; the
    // second warp group adds its half of the rows to the first group's
    __syncthreads();
    df* sOut = reinterpret_cast<df*>(tc_raw);   // [16 T4][NR]
    for (int g2 = 0; g2 < WG; ++g2) {
      if (grp == g2) {
#pragma unroll
        for (int tt = 0; tt < TPW; ++tt) {
          const int tile = wid + tt * NW;
          if (tile < NTILES) {
            const int mt = tile / T4, nt = tile % T4;
            const int row = 16 * mt + (lane >> 2), col = 8 * nt + 2 * (lane & 3);
            const size_t o[4] = {(size_t)row * NR + col, (size_t)row * NR + col + 1,
                                 (size_t)(row + 8) * NR + col, (size_t)(row + 8) * NR + col + 1};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              df v = df_norm(dacc[tt][e]);
              sOut[o[e]] = g2 == 0 ? v : df_add(sOut[o[e]], v);
            }
          }
        }
      }
      __syncthreads();
    }
    zd* out = pass == 1 ? Op + ((size_t)j * 9 + 1 + dir) * ne
                        : Xpart + ((size_t)mu * B.d + j) * ne;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      int b = e / n2k, a = e % n2k;
      df re = sOut[(size_t)b * NR + a], im = sOut[(size_t)(n2k + b) * NR + a];
      out[(size_t)b * n2k + a] = {coef * df_val(re), coef * df_val(im)};   // column-major
    }
    __syncthreads();
  }
  if (bad) atomicExch(range_flag, 1);
}

template <int T4, int NB>
int launch_tc(zd* Op, zd* Xpart, const zdf* Pdf, int k, const zdf* Ldf, const HopGeom& g,
              const Blocking& B, int* range_flag, cudaStream_t st) {
  constexpr int NW = TcCfg<T4, NB>::NW * TcCfg<T4, NB>::WG;
  size_t sh = tc_cta_bytes(T4, NB, B.nd);
  WMG_TRY(smem_attr(galerkin_tc_kernel<T4, NB>, sh));
  if (TcCfg<T4, NB>::MINB > 1)   // room for two CTAs: the largest shared-memory carveout
    WMG_CUDA(cudaFuncSetAttribute(galerkin_tc_kernel<T4, NB>,
                                  cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared));
  galerkin_tc_kernel<T4, NB><<<dim3(B.d, 4), 32 * NW, sh, st>>>(Op, Xpart, Pdf, k, Ldf, g, B,
                                                                range_flag);
  WMG_LAUNCHED();
  return MG_OK;
}

constexpr size_t kTcSmemMax = (size_t)227 * 1024 - 1024;

}  // namespace

bool galerkin_tc_supported(int k, const Blocking& B) {
  if (k < 1 || (k + 3) / 4 > TC_MAXT4) return false;
  // shared memory of one CTA at 4 sites per batch, and tile offsets that fit an int
  const int t4 = (k + 3) / 4;
  return tc_cta_bytes(t4, 4, B.nd) <= kTcSmemMax &&
         (size_t)B.d * 2 * k * B.M < ((size_t)1 << 31);
}

double galerkin_tc_issued_flops(int k, const Blocking& B, int nb) {
  // bf16 digit-plane products issued: 28 digit pairs of a (16 T4) x (8 T4) x (12 NB) real
  // product per batch and hop direction, about n_d / NB + 1 batches per CTA
  const int t4 = (k + 3) / 4;
  return 2.0 * (16.0 * t4) * (8.0 * t4) * (12.0 * nb) * 28.0 * 4.0 * B.d *
         ((double)B.nd / nb + 1.0);
}

int galerkin_hops_tc(zd* Op, zd* Xpart, const zdf* Pdf, int k, const zdf* Ldf, const HopGeom& g,
                     const Blocking& B, int nb, int* range_flag, cudaStream_t st) {
  if (nb == 8) {
    switch ((k + 3) / 4) {
      case 1: return launch_tc<1, 8>(Op, Xpart, Pdf, k, Ldf, g, B, range_flag, st);
      case 2: return launch_tc<2, 8>(Op, Xpart, Pdf, k, Ldf, g, B, range_flag, st);
      case 3: return launch_tc<3, 8>(Op, Xpart, Pdf, k, Ldf, g, B, range_flag, st);
      default: return fail(MG_EINVAL, "galerkin (tensor pipe): 8-site batches need 2k <= 24");
    }
  }
  if (nb != 4) return fail(MG_EINVAL, "galerkin (tensor pipe): batches of 4 or 8 sites");
  switch ((k + 3) / 4) {
    case 1: return launch_tc<1, 4>(Op, Xpart, Pdf, k, Ldf, g, B, range_flag, st);
    case 2: return launch_tc<2, 4>(Op, Xpart, Pdf, k, Ldf, g, B, range_flag, st);
    case 3: return launch_tc<3, 4>(Op, Xpart, Pdf, k, Ldf, g, B, range_flag, st);
    case 4: return launch_tc<4, 4>(Op, Xpart, Pdf, k, Ldf, g, B, range_flag, st);
    case 5: return launch_tc<5, 4>(Op, Xpart, Pdf, k, Ldf, g, B, range_flag, st);
    case 6: return launch_tc<6, 4>(Op, Xpart, Pdf, k, Ldf, g, B, range_flag, st);
    default: return fail(MG_EINVAL, "galerkin (tensor pipe): 2k > 48");
  }
}

int galerkin_tc_batch(int* nb, zd* Op, zd* Xpart, const zdf* Pdf, int k, const zdf* Ldf,
                      const HopGeom& g, const Blocking& B, int* range_flag, cudaStream_t st) {
  // 8-site batches (one CTA per SM: the staging and the products of a CTA alternate) or
  // 4-site batches (two CTAs per SM whose phases overlap, twice the per-batch folds): the
  // autotuner times both on the live arguments where both fit (2k <= 24); the kernel is
  // idempotent (it rewrites its outputs from inputs it does not modify; the range flag, which
  // the caller clears before its own launch, can only be raised)
  const int t4 = (k + 3) / 4;
  if (t4 > 3 || tc_cta_bytes(t4, 8, B.nd) > kTcSmemMax) {
    *nb = 4;
    return MG_OK;
  }
  int err = MG_OK;
  auto run = [&](int v) {
    int e = galerkin_hops_tc(Op, Xpart, Pdf, k, Ldf, g, B, v == 0 ? 8 : 4, range_flag, st);
    if (e != MG_OK) err = e;
  };
  int v = tuned_variant(2000 + t4, -3, 0, B.d * B.nd, k, st, 2, run);
  if (err != MG_OK) return err;
  if (v < 0) return fail(MG_ECUDA, "galerkin (tensor pipe): autotune failed");
  *nb = v == 0 ? 8 : 4;
  return MG_OK;
}

}  // namespace wmg
