// Multigrid hierarchy handle: iCSVD setup (Algorithms 3-4), Galerkin coarse build
// (Eq. 5) and the K-cycle preconditioned FGMRES solve of D x = b (Eq. 1; Sec. 2.1, 4).
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace wmg;

// A level below level 1 (Sec. 2.1 end; Sec. 4 uses three and four levels): built by
// mg_add_level from the coarsest operator so far, level l, with the setup of Algorithm 3 and
// the Galerkin product of Eq. 5; it holds P_l (level l -> l + 1) and the operator of level
// l + 1, and the solver state of the K-cycle of level l.
struct CLevel {
  Blocking B;              // L: level-l lattice, b: aggregate, C: level-(l+1) lattice,
                           // M = n_d k_in rows per tile
  int k_in = 0, k = 0;     // k_l and k_{l+1}
  double tol = 0.03;       // relative tolerance of the level-(l+1) solve
  zd* P64 = nullptr;       // [2 d'][k][M]
  zf* P32 = nullptr;
  double* sigma = nullptr; // [2 d'][k]
  zd* Op64 = nullptr;      // level-(l+1) stencil [d'][9][2k][2k] (column-major blocks)
  zf* Op32 = nullptr;
  size_t n_in = 0, n = 0;  // complex entries of a level-l / level-(l+1) vector
  Gmres<double> solve64, post64;   // level-(l+1) solve, level-l post-smoother
  Gmres<float> solve32, post32;
  void *vc = nullptr, *ec = nullptr, *kw = nullptr, *ke = nullptr;   // solve precision
  long long its = 0;       // level-(l+1) iterations of the current solve
  void free_solver() {
    solve64.release(); post64.release(); solve32.release(); post32.release();
    dev_free(vc); dev_free(ec); dev_free(kw); dev_free(ke);
    vc = ec = kw = ke = nullptr;
  }
  ~CLevel() {
    free_solver();
    dev_free(P64); dev_free(P32); dev_free(sigma); dev_free(Op64); dev_free(Op32);
  }
};

struct mg_handle {
  mg_params p;
  Geom g;
  Blocking B;
  int k = 0;
  size_t nf = 0;   // complex entries per fine field
  size_t nc = 0;   // complex entries per coarse field
  zd* links64 = nullptr;       // ABI layout (Galerkin, gradient)
  zd* links64L = nullptr;      // lane-contiguous [mu][9][site] copies for the stencil
  zf* links32L = nullptr;
  void* links16L = nullptr;    // half-storage solve: zh or zbf lane-contiguous links
  int llay = 1;                // layout of links32L / links16L: 1 three rows, 2 two rows
  zd* clov64 = nullptr;        // clover term C(x) [site][2][6][6] (csw != 0), FP64 and FP32
  zf* clov32 = nullptr;
  zd* P64 = nullptr;
  zf* P32 = nullptr;
  double* sigma = nullptr;   // [tile][k]
  double* hist = nullptr;    // [n_s][tile][k]
  zd* Op64 = nullptr;
  zf* Op32 = nullptr;
  zd* PtP = nullptr;           // [tile][k][k] Gram matrices of the P tiles (Galerkin diagonal)
  zdf* Pdf = nullptr;          // double-float Galerkin: P and the links as (hi, lo) pairs
  zdf* Ldf = nullptr;
  bool have_P = false, have_coarse = false;
  bool pdf_ready = false;      // Pdf holds the double-float split of P64 already
  int* tc_flag = nullptr;      // device int: range flag of the tensor-pipe Galerkin
  // solver state, sized for `nrhs`
  int nrhs = 0;
  Gmres<double> outer64, coarse64, post64;
  Gmres<float> outer32, coarse32, post32;
  CoarseSolver<double> csol64;
  CoarseSolver<float> csol32;
  GmresV<zh> posth;            // half-storage post-smoother (solve_dtype MG_F16)
  GmresV<zbf> postb;           // (solve_dtype MG_BF16)
  Gmres<double> posts64;       // Schur-form post-smoother on even half-lattice fields
  Gmres<float> posts32;
  void* sbuf[5] = {};          // its half-lattice fields: r_e, r_o, r_hat, x_e, odd temporary
  void *kwh = nullptr, *keh = nullptr;
  zd *x64 = nullptr, *r64 = nullptr, *t64 = nullptr;
  zf *e32 = nullptr, *r32 = nullptr;
  zd *vc64 = nullptr, *ec64 = nullptr, *kw64 = nullptr, *ke64 = nullptr;
  zf *vc32 = nullptr, *ec32 = nullptr, *kw32 = nullptr, *ke32 = nullptr;
  double* dscal = nullptr;     // device scalars [4][nrhs]
  double* hscal = nullptr;     // pinned
  ReduceWork rw;
  std::vector<std::unique_ptr<CLevel>> lv;   // levels 2, 3, ... (mg_add_level)
  // counters of the last solve
  long long coarse_its = 0;
  int kcycles = 0;
  ~mg_handle();
  void free_solver();
};

namespace {

template <typename T>
void dfree(T*& p) {
  dev_free(p);
  p = nullptr;
}

// Galerkin sums of products in double-float (explicit, or by default in the mixed forms)
bool galerkin_df(const mg_params& p) {
  return p.fp64_emulation > 0 || (p.fp64_emulation < 0 && p.solve_dtype != MG_C128);
}

int validate(const mg_params* p, bool need_svd) {
  if (!p) return fail(MG_EINVAL, "NULL params");
  for (int m = 0; m < 4; ++m) {
    if (p->dims[m] < 2 || (p->dims[m] & 1)) return fail(MG_EINVAL, "lattice extents must be even and >= 2");
    if (p->block[m] < 1 || p->dims[m] % p->block[m]) return fail(MG_EINVAL, "block must divide dims");
  }
  int nd = p->block[0] * p->block[1] * p->block[2] * p->block[3];
  if (p->k < 1 || p->k > 6 * nd) return fail(MG_EINVAL, "k must be in [1, 6 n_d]");
  if (p->k > 32) return fail(MG_EINVAL, "k > 32 not supported");
  if (need_svd) {
    if (p->r < 1 || p->n_s < 1) return fail(MG_EINVAL, "r and n_s must be >= 1");
    if (p->k + p->r > 64) return fail(MG_EINVAL, "k + r must be <= 64");
    if ((long long)p->r * p->n_s < p->k) return fail(MG_EINVAL, "n_s * r must be >= k");
    if (p->sweeps < 0 || p->sweeps > 64) return fail(MG_EINVAL, "sweeps must be in [0, 64]");
    if (p->setup_dtype != MG_C128 && p->setup_dtype != MG_C64)
      return fail(MG_EINVAL, "setup_dtype must be MG_C128 or MG_C64");
  }
  if (p->solve_dtype != MG_C128 && p->solve_dtype != MG_C64 && p->solve_dtype != MG_F16 &&
      p->solve_dtype != MG_BF16)
    return fail(MG_EINVAL, "solve_dtype must be MG_C128, MG_C64, MG_F16 or MG_BF16");
  if (p->post_smooth < 0 || p->post_smooth > 64) return fail(MG_EINVAL, "post_smooth in [0, 64]");
  if (p->schur_smoother && p->solve_dtype != MG_C128 && p->solve_dtype != MG_C64)
    return fail(MG_EINVAL, "schur_smoother needs solve_dtype MG_C128 or MG_C64");
  if (p->csw != 0 && (p->schur_smoother || p->solve_dtype == MG_F16 || p->solve_dtype == MG_BF16))
    return fail(MG_EINVAL, "csw != 0: the clover term is applied in FP64 / FP32 without the "
                           "Schur-form smoother (schur_smoother = 0, solve_dtype MG_C128 / MG_C64)");
  if (!std::isfinite(p->csw)) return fail(MG_EINVAL, "csw must be finite");
  if (p->coarse_restart < 1 || p->coarse_restart > 128) return fail(MG_EINVAL, "coarse_restart in [1, 128]");
  if (p->outer_restart < 1 || p->outer_restart > 128) return fail(MG_EINVAL, "outer_restart in [1, 128]");
  if (!(p->coarse_tol > 0 && p->coarse_tol < 1)) return fail(MG_EINVAL, "coarse_tol in (0, 1)");
  if (p->coarse_persistent && p->coarse_restart > 48)
    return fail(MG_EINVAL, "coarse_restart <= 48 with the persistent coarse solver");
  return MG_OK;
}

int create_handle(mg_handle** out, const void* links, const mg_params* p, bool need_svd,
                  cudaStream_t st) {
  if (!out) return fail(MG_EINVAL, "NULL handle pointer");
  if (*out) return fail(MG_EINVAL, "*h must be NULL on entry");
  if (!links) return fail(MG_EINVAL, "NULL links");
  WMG_TRY(validate(p, need_svd));
  std::unique_ptr<mg_handle> h(new mg_handle());
  h->p = *p;
  WMG_TRY(make_geom(h->g, p->dims, p->kappa, p->hop_weight, p->bc_phase, true));
  WMG_TRY(make_blocking(h->B, p->dims, p->block));
  h->k = p->k;
  h->nf = (size_t)h->g.V * 12;
  h->nc = (size_t)h->B.d * 2 * h->k;
  size_t lb = (size_t)4 * h->g.V * 9;
  WMG_TRY(dev_alloc(&h->links64, lb * sizeof(zd)));
  WMG_TRY(dev_alloc(&h->links64L, lb * sizeof(zd)));
  Staged sl;
  WMG_TRY(stage_in(sl, links, lb * sizeof(zd), st));
  WMG_CUDA(cudaMemcpyAsync(h->links64, sl.dev, lb * sizeof(zd), cudaMemcpyDeviceToDevice, st));
  WMG_TRY(link_to_lanes<double>(h->links64L, h->links64, h->g.V, st));
  // the double-float copy of the links (double-float Galerkin sums) first: the SU(3) check
  // below runs on it in double-float arithmetic instead of on the FP64 units
  if (galerkin_df(*p)) {
    WMG_TRY(dev_alloc(&h->Ldf, lb * sizeof(zdf)));
    WMG_TRY(to_df(h->Ldf, h->links64, lb, st));
  }
  // the FP32 / half stencil copies keep two rows per link when the links are SU(3)
  int rows = 3;
  if (p->link_compress != 0) {
    double dev = 0;
    if (h->Ldf) WMG_TRY(su3_deviation_df(&dev, h->Ldf, (size_t)4 * h->g.V, st));
    else WMG_TRY(su3_deviation(&dev, h->links64, (size_t)4 * h->g.V, st));
    if (dev <= 1e-9) rows = 2;
    else if (p->link_compress > 0)
      return fail(MG_EINVAL, "link_compress = 1 needs SU(3) links (deviation " +
                                 std::to_string(dev) + " > 1e-9)");
  }
  h->llay = rows == 2 ? 2 : 1;
  size_t lbc = (size_t)4 * h->g.V * 3 * rows;
  WMG_TRY(dev_alloc(&h->links32L, lbc * sizeof(zf)));
  WMG_TRY(link_to_lanes<float>(h->links32L, h->links64, h->g.V, st, rows));
  if (p->solve_dtype == MG_F16 || p->solve_dtype == MG_BF16) {
    WMG_TRY(dev_alloc(&h->links16L, lbc * 4));
    if (p->solve_dtype == MG_F16) WMG_TRY(link_to_lanes_v<zh>((zh*)h->links16L, h->links64, h->g.V, st, rows));
    else WMG_TRY(link_to_lanes_v<zbf>((zbf*)h->links16L, h->links64, h->g.V, st, rows));
  }
  if (p->csw != 0) {
    WMG_TRY(dev_alloc(&h->clov64, (size_t)h->g.V * 72 * sizeof(zd)));
    WMG_TRY(dev_alloc(&h->clov32, (size_t)h->g.V * 72 * sizeof(zf)));
    WMG_TRY(clover_field(h->clov64, h->links64, h->g, p->csw, st));
    WMG_TRY((convert<float, double>(h->clov32, h->clov64, nullptr, 0, (size_t)h->g.V * 72, 1, st)));
  }
  size_t ntile = (size_t)h->B.d * 2;
  WMG_TRY(dev_alloc(&h->P64, ntile * h->k * h->B.M * sizeof(zd)));
  WMG_TRY(dev_alloc(&h->P32, ntile * h->k * h->B.M * sizeof(zf)));
  WMG_TRY(dev_alloc(&h->sigma, ntile * h->k * sizeof(double)));
  WMG_TRY(dev_alloc(&h->PtP, ntile * h->k * h->k * sizeof(zd)));
  if (galerkin_df(*p)) {
    WMG_TRY(dev_alloc(&h->Pdf, ntile * h->k * h->B.M * sizeof(zdf)));
  }
  WMG_CUDA(cudaMemsetAsync(h->sigma, 0, ntile * h->k * sizeof(double), st));
  WMG_TRY(dev_alloc(&h->tc_flag, sizeof(int)));
  int ns = p->n_s > 0 ? p->n_s : 1;
  WMG_TRY(dev_alloc(&h->hist, (size_t)ns * ntile * h->k * sizeof(double)));
  WMG_CUDA(cudaMemsetAsync(h->hist, 0, (size_t)ns * ntile * h->k * sizeof(double), st));
  WMG_CUDA(cudaStreamSynchronize(st));
  *out = h.release();
  return MG_OK;
}

// Caller-supplied vectors of mg_setup_from_vectors: n_s r fields on the device, stream s
// using fields s r .. s r + r - 1; smooth = 1: they are the initial guesses phi of Eq. 2,
// 0: they are the test vectors psi themselves.
struct SetupSource {
  const void* fields;
  int dtype;
  int smooth;
};

// psi = phi + GMRES_sweeps(D, -D phi)   (Eq. 2) for r fields, in precision R; phi is the
// stream's Philox field, or the caller's fields when src is given.  phi goes straight into
// psi, and the sum is formed as psi -= GMRES_sweeps(D, D phi): GMRES is odd in its right-hand
// side (negating b negates every basis vector and the minimiser, exactly), so neither -D phi
// nor the sum is a pass of its own.  tmp: r fields of scratch.
template <typename R>
int smooth_stream(mg_handle* h, cplx<R>* psi, cplx<R>* tmp, Gmres<R>& gm, int s,
                  cudaStream_t st, const SetupSource* src = nullptr) {
  const mg_params& p = h->p;
  int r = p.r;
  if (src) {
    size_t off = (size_t)s * r * h->nf;
    if (src->dtype == MG_C128)
      WMG_TRY((convert<R, double>(psi, static_cast<const zd*>(src->fields) + off, nullptr, 0,
                                  h->nf * r, 1, st)));
    else
      WMG_TRY((convert<R, float>(psi, static_cast<const zf*>(src->fields) + off, nullptr, 0,
                                 h->nf * r, 1, st)));
    if (!src->smooth) return MG_OK;
  } else {
    WMG_TRY(gaussian_fill<R>(psi, p.seed, (unsigned)(s * r), r, h->g.V, st));
  }
  int dt = sizeof(R) == 8 ? MG_C128 : MG_C64;
  const void* L = sizeof(R) == 8 ? (const void*)h->links64L : (const void*)h->links32L;
  const int lay = sizeof(R) == 8 ? 1 : h->llay;
  const cplx<R>* Cl = sizeof(R) == 8 ? (const cplx<R>*)h->clov64 : (const cplx<R>*)h->clov32;
  Op<R> D = [h, dt, L, r, lay, Cl](cplx<R>* out, const cplx<R>* in, cudaStream_t s2) -> int {
    WMG_TRY(dslash_launch(dt, out, in, L, h->g, -1, 0, r, s2, h->nf, h->nf, lay));
    if (Cl) WMG_TRY(clover_add<R>(out, in, Cl, h->g.V, r, s2));
    return MG_OK;
  };
  WMG_TRY(D(tmp, psi, st));   // tmp = D phi
  WMG_TRY(gm.alloc(h->nf, r, p.sweeps > 0 ? p.sweeps : 1, false));
  FusedStencil fz{h->links32L, h->g, h->llay};   // FP32 Wilson runs fuse the stencil with the projections
  WMG_TRY(gm.fixed(D, psi, tmp, p.sweeps, st, true, sizeof(R) == 4 && !Cl ? &fz : nullptr,
                   -1.0));   // psi = phi - GMRES(D, D phi)
  return MG_OK;
}

// ls_omega (device, r weights): the final update is the least-squares interpolation of Eq. 9
// instead of U_k (one stream, one Gram pass)
template <typename R>
int run_setup(mg_handle* h, cudaStream_t st, const SetupSource* src = nullptr,
              const double* ls_omega = nullptr) {
  const mg_params& p = h->p;
  int r = p.r, k = h->k;
  int cmax = k + r;
  size_t ntile = (size_t)h->B.d * 2;
  size_t M = h->B.M;
  size_t fr = h->nf * r;
  cplx<R>*psi = nullptr, *tmp = nullptr;
  zd *T0 = nullptr, *T1 = nullptr, *G = nullptr, *Vec = nullptr;
  double* lam = nullptr;
  Gmres<R> gm;
  int status = MG_OK;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);   // the cached blocks are reused only after their work ends
    dfree(psi); dfree(tmp); dfree(T0); dfree(T1); dfree(G); dfree(Vec); dfree(lam);
  };
#define STEP(x) do { status = (x); if (status != MG_OK) { cleanup(); return status; } } while (0)
#define CSTEP(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { cleanup(); return fail(e_ == cudaErrorMemoryAllocation ? MG_ENOMEM : MG_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); } } while (0)
  STEP(dev_alloc(&psi, fr * sizeof(cplx<R>)));
  STEP(dev_alloc(&tmp, fr * sizeof(cplx<R>)));
  STEP(dev_alloc(&T0, ntile * cmax * M * sizeof(zd)));
  STEP(dev_alloc(&T1, ntile * cmax * M * sizeof(zd)));
  STEP(dev_alloc(&G, ntile * cmax * cmax * sizeof(zd)));
  STEP(dev_alloc(&Vec, ntile * cmax * cmax * sizeof(zd)));
  STEP(dev_alloc(&lam, ntile * cmax * sizeof(double)));
  zd* cur = T0;
  zd* oth = T1;
  int kk = 0;
  // sums of products in double-float when asked, or by default when the test vectors are FP32
  const bool df = p.fp64_emulation > 0 || (p.fp64_emulation < 0 && sizeof(R) == 4);
  // rotate only above the accuracy of the Gram sums (FP64 ~1e-16, double-float ~1e-14)
  const double eig_tol = df ? 1e-13 : 1e-15;
  const bool refine = p.svd_refine > 0 || (p.svd_refine < 0 && sizeof(R) == 8);
  int c_prev = 0;
  for (int s = 0; s < p.n_s; ++s) {
    STEP(smooth_stream<R>(h, psi, tmp, gm, s, st, src));
    STEP(chiral_gather<R>(cur, cmax, kk, psi, r, h->B, st, df));
    int c = kk + r;
    int kn = c < k ? c : k;
    bool last = s == p.n_s - 1;
    // single-pass route: the kept columns Phi_{s-1} = A_{s-1} V_k are orthogonal with squared
    // norms lam (Phi^dag Phi = V_k^dag G V_k = Lambda_k, to the Jacobi tolerance and the
    // update's c-term rounding), so only their cross products with the new vectors and the new
    // vectors' own Gram block are summed (the second pass of the refined route recomputes all)
    const int kd = refine ? 0 : kk;
    STEP(tile_gram(G, cur, cmax, c, h->B, st, df, kd, lam, c_prev));
    STEP(tile_eig(lam, Vec, G, c, (int)ntile, st, eig_tol, df));
    if (ls_omega) {
      // P = A W with W = Omega V_k B^-1 Sigma_k^-1 (Eq. 9); G is free after the eigensolver
      STEP(tile_ls_weights(G, Vec, lam, ls_omega, c, kn, (int)ntile, st));
      STEP(tile_update(oth, cmax, cur, cmax, c, G, lam, kn, 0, h->B, st, df));
      zd* t = cur; cur = oth; oth = t;
    } else if (p.svd_refine > 0 || (p.svd_refine < 0 && sizeof(R) == 8)) {
      // B = A V (all c columns), then a second Gram/eig pass on B
      STEP(tile_update(oth, cmax, cur, cmax, c, Vec, lam, c, 0, h->B, st, df));
      STEP(tile_gram(G, oth, cmax, c, h->B, st, df));
      STEP(tile_eig(lam, Vec, G, c, (int)ntile, st, eig_tol, df));
      STEP(tile_update(cur, cmax, oth, cmax, c, Vec, lam, kn, last ? 1 : 0, h->B, st, df));
    } else {
      STEP(tile_update(oth, cmax, cur, cmax, c, Vec, lam, kn, last ? 1 : 0, h->B, st, df));
      zd* t = cur; cur = oth; oth = t;
    }
    STEP(tile_sigma(h->hist + (size_t)s * ntile * k, k, lam, c, kn, (int)ntile, st));
    kk = kn;
    c_prev = c;
  }
  if (df) {
    // double-float tiles: the canonical phase, P, its FP32 copy and (for the double-float
    // Galerkin) its double-float copy in one pass
    STEP(tile_phase_outputs(h->P64, h->P32, h->Pdf, cur, cmax, k, h->B, st));
    h->pdf_ready = h->Pdf != nullptr;
  } else {
    STEP(tile_canonical_phase(cur, cmax, k, h->B, st, df));
    CSTEP(cudaMemcpy2DAsync(h->P64, (size_t)k * M * sizeof(zd), cur, (size_t)cmax * M * sizeof(zd),
                            (size_t)k * M * sizeof(zd), ntile, cudaMemcpyDeviceToDevice, st));
    STEP((convert<float, double>(h->P32, h->P64, nullptr, 0, ntile * k * M, 1, st)));
    h->pdf_ready = false;
  }
  CSTEP(cudaMemcpyAsync(h->sigma, h->hist + (size_t)(p.n_s - 1) * ntile * k,
                        ntile * k * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CSTEP(cudaStreamSynchronize(st));
  if (take_device_error()) {
    cleanup();
    return fail(MG_ETIMEOUT, "setup: a bounded wait gave up");
  }
  cleanup();
  h->have_P = true;
  h->have_coarse = false;
#undef STEP
#undef CSTEP
  return MG_OK;
}

int ensure_solver(mg_handle* h, int nrhs) {
  if (h->nrhs == nrhs) return MG_OK;
  if (h->nrhs) cudaDeviceSynchronize();   // no queued work may still use the old buffers
  h->free_solver();
  size_t f = h->nf * nrhs, c = h->nc * nrhs;
  const mg_params& p = h->p;
  WMG_TRY(dev_alloc(&h->x64, f * sizeof(zd)));
  WMG_TRY(dev_alloc(&h->r64, f * sizeof(zd)));
  WMG_TRY(dev_alloc(&h->t64, f * sizeof(zd)));
  WMG_TRY(dev_alloc(&h->dscal, 8 * nrhs * sizeof(double)));
  WMG_TRY(host_alloc(&h->hscal, 8 * nrhs * sizeof(double)));
  WMG_TRY(h->rw.alloc(h->nf, nrhs, 2));
  if (p.solve_dtype == MG_C128) {
    WMG_TRY(dev_alloc(&h->vc64, c * sizeof(zd)));
    WMG_TRY(dev_alloc(&h->ec64, c * sizeof(zd)));
    WMG_TRY(dev_alloc(&h->kw64, f * sizeof(zd)));
    WMG_TRY(dev_alloc(&h->ke64, f * sizeof(zd)));
    WMG_TRY(h->outer64.alloc(h->nf, nrhs, p.outer_restart, true));
    WMG_TRY(h->coarse64.alloc(h->nc, nrhs, p.coarse_restart, !h->lv.empty()));
    if (p.coarse_persistent) WMG_TRY(h->csol64.alloc(h->nc, p.coarse_restart));
    WMG_TRY(h->post64.alloc(h->nf, nrhs, p.post_smooth > 0 ? p.post_smooth : 1, false));
  } else {
    WMG_TRY(dev_alloc(&h->e32, f * sizeof(zf)));
    WMG_TRY(dev_alloc(&h->r32, f * sizeof(zf)));
    WMG_TRY(dev_alloc(&h->vc32, c * sizeof(zf)));
    WMG_TRY(dev_alloc(&h->ec32, c * sizeof(zf)));
    WMG_TRY(dev_alloc(&h->kw32, f * sizeof(zf)));
    WMG_TRY(dev_alloc(&h->ke32, f * sizeof(zf)));
    WMG_TRY(h->outer32.alloc(h->nf, nrhs, p.outer_restart, true));
    WMG_TRY(h->coarse32.alloc(h->nc, nrhs, p.coarse_restart, !h->lv.empty()));
    if (p.coarse_persistent) WMG_TRY(h->csol32.alloc(h->nc, p.coarse_restart));
    int ps = p.post_smooth > 0 ? p.post_smooth : 1;
    if (p.solve_dtype == MG_F16 || p.solve_dtype == MG_BF16) {
      WMG_TRY(dev_alloc(&h->kwh, f * 4));
      WMG_TRY(dev_alloc(&h->keh, f * 4));
      if (p.solve_dtype == MG_F16) WMG_TRY(h->posth.alloc(h->nf, nrhs, ps, false));
      else WMG_TRY(h->postb.alloc(h->nf, nrhs, ps, false));
    } else {
      WMG_TRY(h->post32.alloc(h->nf, nrhs, ps, false));
    }
  }
  for (auto& L : h->lv) {
    const bool d64 = p.solve_dtype == MG_C128;
    const size_t es = d64 ? sizeof(zd) : sizeof(zf);
    WMG_TRY(dev_alloc(&L->vc, L->n * nrhs * es));
    WMG_TRY(dev_alloc(&L->ec, L->n * nrhs * es));
    WMG_TRY(dev_alloc(&L->kw, L->n_in * nrhs * es));
    WMG_TRY(dev_alloc(&L->ke, L->n_in * nrhs * es));
    const bool coarsest = L.get() == h->lv.back().get();
    int ps = p.post_smooth > 0 ? p.post_smooth : 1;
    if (d64) {
      WMG_TRY(L->solve64.alloc(L->n, nrhs, p.coarse_restart, !coarsest));
      WMG_TRY(L->post64.alloc(L->n_in, nrhs, ps, false));
    } else {
      WMG_TRY(L->solve32.alloc(L->n, nrhs, p.coarse_restart, !coarsest));
      WMG_TRY(L->post32.alloc(L->n_in, nrhs, ps, false));
    }
  }
  if (p.schur_smoother) {
    size_t eh = (h->nf / 2) * nrhs * (p.solve_dtype == MG_C128 ? sizeof(zd) : sizeof(zf));
    for (auto& b : h->sbuf) WMG_TRY(dev_alloc(&b, eh));
    int ps = p.post_smooth > 0 ? p.post_smooth : 1;
    if (p.solve_dtype == MG_C128) WMG_TRY(h->posts64.alloc(h->nf / 2, nrhs, ps, false));
    else WMG_TRY(h->posts32.alloc(h->nf / 2, nrhs, ps, false));
  }
  h->nrhs = nrhs;
  return MG_OK;
}

// Typed views of the handle's precision-dependent members.
template <typename R> struct Lvl;
template <> struct Lvl<double> {
  static const void* links(mg_handle* h) { return h->links64L; }
  static int layout(mg_handle*) { return 1; }
  static const zd* P(mg_handle* h) { return h->P64; }
  static const zd* Op(mg_handle* h) { return h->Op64; }
  static Gmres<double>& coarse(mg_handle* h) { return h->coarse64; }
  static CoarseSolver<double>& csol(mg_handle* h) { return h->csol64; }
  static Gmres<double>& post(mg_handle* h) { return h->post64; }
  static Gmres<double>& posts(mg_handle* h) { return h->posts64; }
  static Gmres<double>& outer(mg_handle* h) { return h->outer64; }
  static zd* vc(mg_handle* h) { return h->vc64; }
  static zd* ec(mg_handle* h) { return h->ec64; }
  static zd* kw(mg_handle* h) { return h->kw64; }
  static zd* ke(mg_handle* h) { return h->ke64; }
  static constexpr int dtype = MG_C128;
};
template <> struct Lvl<float> {
  static const void* links(mg_handle* h) { return h->links32L; }
  static int layout(mg_handle* h) { return h->llay; }
  static const zf* P(mg_handle* h) { return h->P32; }
  static const zf* Op(mg_handle* h) { return h->Op32; }
  static Gmres<float>& coarse(mg_handle* h) { return h->coarse32; }
  static CoarseSolver<float>& csol(mg_handle* h) { return h->csol32; }
  static Gmres<float>& post(mg_handle* h) { return h->post32; }
  static Gmres<float>& posts(mg_handle* h) { return h->posts32; }
  static Gmres<float>& outer(mg_handle* h) { return h->outer32; }
  static zf* vc(mg_handle* h) { return h->vc32; }
  static zf* ec(mg_handle* h) { return h->ec32; }
  static zf* kw(mg_handle* h) { return h->kw32; }
  static zf* ke(mg_handle* h) { return h->ke32; }
  static constexpr int dtype = MG_C64;
};

template <typename R>
Op<R> fine_op(mg_handle* h, int nrhs) {
  return [h, nrhs](cplx<R>* out, const cplx<R>* in, cudaStream_t st) -> int {
    WMG_TRY(dslash_launch(Lvl<R>::dtype, out, in, Lvl<R>::links(h), h->g, -1, 0, nrhs, st, h->nf,
                          h->nf, Lvl<R>::layout(h)));
    const cplx<R>* Cl = sizeof(R) == 8 ? (const cplx<R>*)h->clov64 : (const cplx<R>*)h->clov32;
    if (Cl) WMG_TRY(clover_add<R>(out, in, Cl, h->g.V, nrhs, st));
    return MG_OK;
  };
}

// the fine operator on half-storage fields (lane-contiguous half links, FP32 arithmetic)
template <typename H>
OpV<H> fine_op_half(mg_handle* h, int nrhs) {
  int dt = std::is_same<H, zh>::value ? MG_F16 : MG_BF16;
  return [h, nrhs, dt](H* out, const H* in, cudaStream_t st) -> int {
    return dslash_launch(dt, out, in, h->links16L, h->g, -1, 0, nrhs, st, h->nf, h->nf, h->llay);
  };
}

// Post-smoother in half storage: e = GMRES_steps(D, v - D z) with the residual, the Krylov
// basis and the stencil in H, then z += e.  v is a unit-norm FGMRES column, so its entries
// are ~ n^-1/2; the residual is scaled by n^1/2 before it is stored in H and the correction
// scaled back, which keeps FP16 entries O(1).
template <typename H>
int post_smooth_half(mg_handle* h, GmresV<H>& gm, zf* z, const zf* v, zf* kw, int nrhs,
                     cudaStream_t st) {
  size_t f = h->nf * nrhs;
  double s = std::sqrt((double)h->nf);
  WMG_TRY((lincomb_v<H, zf>((H*)h->kwh, s, v, -s, kw, f, st)));   // kw holds D z
  WMG_TRY(gm.fixed(fine_op_half<H>(h, nrhs), (H*)h->keh, (const H*)h->kwh, h->p.post_smooth, st));
  WMG_TRY((axpy_mixed<zf, H>(z, 1.0 / s, (const H*)h->keh, f, st)));
  return MG_OK;
}

// Post-smoother on the even-odd Schur system (even-odd preconditioning, Sec. 1): with the
// residual r = v - D z split into r_e, r_o,
//   r_hat = r_e + kappa H_eo r_o,  e_e = GMRES_post(D_hat, r_hat),  e_o = r_o + kappa H_oe e_e,
// and z += (e_e, e_o).  (D e)_o = r_o holds exactly for any number of steps.  The residual is
// formed and split by parity in one pass after the stencil, and the accumulation of (e_e, e_o)
// into z is one pass.
template <typename R>
int post_smooth_schur(mg_handle* h, cplx<R>* z, const cplx<R>* v, int nrhs, cudaStream_t st) {
  const Geom& g = h->g;
  const size_t nh = h->nf / 2;
  cplx<R>* re = static_cast<cplx<R>*>(h->sbuf[0]);
  cplx<R>* ro = static_cast<cplx<R>*>(h->sbuf[1]);
  cplx<R>* rh = static_cast<cplx<R>*>(h->sbuf[2]);
  cplx<R>* xe = static_cast<cplx<R>*>(h->sbuf[3]);
  cplx<R>* to = static_cast<cplx<R>*>(h->sbuf[4]);
  const void* L = Lvl<R>::links(h);
  const int lay = Lvl<R>::layout(h);
  const int dt = Lvl<R>::dtype;
  // (r_e, r_o) = split(v - D z)
  cplx<R>* kw = Lvl<R>::kw(h);
  WMG_TRY(fine_op<R>(h, nrhs)(kw, z, st));
  WMG_TRY(eo_split_diff<cplx<R>>(re, ro, v, kw, g, nrhs, st));
  WMG_TRY(dslash_launch(dt, rh, ro, L, g, 0, 0, nrhs, st, nh, nh, lay, re));   // r_hat
  Op<R> Dhat = [h, to, L, lay, nrhs](cplx<R>* out, const cplx<R>* in, cudaStream_t s2) -> int {
    return schur_apply<cplx<R>>(out, in, to, L, lay, h->g, 0, nrhs, s2);
  };
  FusedStencil fz{h->links32L, h->g, h->llay, true, to};   // FP32: hops fused with projections
  WMG_TRY(Lvl<R>::posts(h).fixed(Dhat, xe, rh, h->p.post_smooth, st, false,
                                 sizeof(R) == 4 && !h->clov32 ? &fz : nullptr));
  WMG_TRY(dslash_launch(dt, to, xe, L, g, 1, 0, nrhs, st, nh, nh, lay, ro));   // e_o
  WMG_TRY(eo_join_add<cplx<R>>(z, xe, to, g, nrhs, st));                  // z += (x_e, e_o)
  return MG_OK;
}

template <typename R>
Op<R> coarse_op(mg_handle* h, int nrhs) {
  return [h, nrhs](cplx<R>* out, const cplx<R>* in, cudaStream_t st) -> int {
    return coarse_apply_launch<R>(out, in, Lvl<R>::Op(h), h->k, h->B, nrhs, st);
  };
}

// D_l on level-l vectors (l >= 1): the level-1 operator, or that of a level added by
// mg_add_level
template <typename R>
Op<R> level_op(mg_handle* h, int l, int nrhs) {
  if (l == 1) return coarse_op<R>(h, nrhs);
  CLevel* L = h->lv[l - 2].get();
  return [L, nrhs](cplx<R>* out, const cplx<R>* in, cudaStream_t st) -> int {
    const cplx<R>* Op = std::is_same<R, double>::value ? (const cplx<R>*)L->Op64
                                                        : (const cplx<R>*)L->Op32;
    return coarse_apply_launch<R>(out, in, Op, L->k, L->B, nrhs, st);
  };
}

template <typename R>
Gmres<R>& lv_solve(CLevel* L);
template <> Gmres<double>& lv_solve<double>(CLevel* L) { return L->solve64; }
template <> Gmres<float>& lv_solve<float>(CLevel* L) { return L->solve32; }
template <typename R>
Gmres<R>& lv_post(CLevel* L);
template <> Gmres<double>& lv_post<double>(CLevel* L) { return L->post64; }
template <> Gmres<float>& lv_post<float>(CLevel* L) { return L->post32; }

// K-cycle of level l >= 1 (Sec. 2.1 end): z = M_l v -- restrict with P_l, solve level l + 1
// to its tolerance (FGMRES preconditioned by the K-cycle of level l + 1, GMRES on the
// coarsest level), prolong, post_smooth GMRES steps on D_l.
template <typename R>
Op<R> kcycle_level(mg_handle* h, int l, int nrhs) {
  return [h, l, nrhs](cplx<R>* z, const cplx<R>* v, cudaStream_t st) -> int {
    const mg_params& p = h->p;
    CLevel* L = h->lv[l - 1].get();
    const cplx<R>* P = std::is_same<R, double>::value ? (const cplx<R>*)L->P64
                                                       : (const cplx<R>*)L->P32;
    cplx<R>* vc = static_cast<cplx<R>*>(L->vc);
    cplx<R>* ec = static_cast<cplx<R>*>(L->ec);
    cplx<R>* kw = static_cast<cplx<R>*>(L->kw);
    cplx<R>* ke = static_cast<cplx<R>*>(L->ke);
    WMG_TRY(coarse_restrict<R>(vc, v, P, L->B, L->k_in, L->k, nrhs, st));
    Op<R> A = level_op<R>(h, l + 1, nrhs);
    int its = 0, s;
    if (l == (int)h->lv.size()) {
      s = lv_solve<R>(L).solve(A, nullptr, ec, vc, L->tol, p.coarse_restart, p.coarse_maxiter,
                               &its, st, 8);
    } else {
      Op<R> M = kcycle_level<R>(h, l + 1, nrhs);
      s = lv_solve<R>(L).solve(A, &M, ec, vc, L->tol, p.coarse_restart, p.coarse_maxiter, &its,
                               st);
    }
    if (s != MG_OK && s != MG_ENOCONV) return s;
    L->its += (long long)its * nrhs;
    WMG_TRY(coarse_prolong<R>(z, ec, P, L->B, L->k_in, L->k, nrhs, st));
    if (p.post_smooth > 0) {
      Op<R> D = level_op<R>(h, l, nrhs);
      WMG_TRY(D(kw, z, st));
      WMG_TRY(axpby<R>(kw, 1.0, v, -1.0, L->n_in * nrhs, 1, st));   // kw = v - D_l z
      WMG_TRY(lv_post<R>(L).fixed(D, ke, kw, p.post_smooth, st));
      WMG_TRY(axpby<R>(z, 1.0, ke, 1.0, L->n_in * nrhs, 1, st));    // z += e
    }
    return MG_OK;
  };
}

// z = M v: restrict, coarse GMRES to coarse_tol, prolong, post-smooth (Sec. 2.1 K-cycle, Sec. 4)
template <typename R>
Op<R> kcycle_op(mg_handle* h, int nrhs) {
  return [h, nrhs](cplx<R>* z, const cplx<R>* v, cudaStream_t st) -> int {
    const mg_params& p = h->p;
    cplx<R>* vc = Lvl<R>::vc(h);
    cplx<R>* ec = Lvl<R>::ec(h);
    cplx<R>* kw = Lvl<R>::kw(h);
    cplx<R>* ke = Lvl<R>::ke(h);
    WMG_TRY(restrict_launch<R>(vc, v, Lvl<R>::P(h), h->k, h->B, nrhs, st));
    int its = 0;
    if (!h->lv.empty()) {
      // deeper hierarchy: FGMRES on level 1 preconditioned by the K-cycle of level 1
      Op<R> Dc = coarse_op<R>(h, nrhs);
      Op<R> M1 = kcycle_level<R>(h, 1, nrhs);
      int s = Lvl<R>::coarse(h).solve(Dc, &M1, ec, vc, p.coarse_tol, p.coarse_restart,
                                      p.coarse_maxiter, &its, st);
      if (s != MG_OK && s != MG_ENOCONV) return s;
      its *= nrhs;
    } else if (p.coarse_persistent && Lvl<R>::csol(h).fits(h->B, h->k)) {
      // one cooperative launch per system: the whole restarted coarse GMRES on the device
      // (its iteration count accumulates there and is read once per solve)
      for (int r = 0; r < nrhs; ++r)
        WMG_TRY(Lvl<R>::csol(h).solve(Lvl<R>::Op(h), h->B, h->k, ec + r * h->nc, vc + r * h->nc,
                                      p.coarse_tol, p.coarse_restart, p.coarse_maxiter, st));
    } else {
      Op<R> Dc = coarse_op<R>(h, nrhs);
      // coarse Arnoldi steps are cheap: check convergence on the host every 8 steps
      int s = Lvl<R>::coarse(h).solve(Dc, nullptr, ec, vc, p.coarse_tol, p.coarse_restart,
                                      p.coarse_maxiter, &its, st, 8);
      if (s != MG_OK && s != MG_ENOCONV) return s;
      its *= nrhs;   // every system took each lockstep step
    }
    h->coarse_its += its;
    h->kcycles += 1;
    WMG_TRY(prolong_launch<R>(z, ec, Lvl<R>::P(h), h->k, h->B, nrhs, st));
    if (p.post_smooth > 0) {
      // the Schur form (Wilson, FP64 / FP32 storage) forms its residual itself
      if (p.schur_smoother) return post_smooth_schur<R>(h, z, v, nrhs, st);
      Op<R> D = fine_op<R>(h, nrhs);
      WMG_TRY(D(kw, z, st));
      if constexpr (std::is_same<R, float>::value) {
        if (p.solve_dtype == MG_F16) return post_smooth_half<zh>(h, h->posth, z, v, kw, nrhs, st);
        if (p.solve_dtype == MG_BF16) return post_smooth_half<zbf>(h, h->postb, z, v, kw, nrhs, st);
      }
      WMG_TRY(axpby<R>(kw, 1.0, v, -1.0, h->nf * nrhs, 1, st));   // kw = v - D z
      FusedStencil fz{h->links32L, h->g, h->llay};   // FP32 Wilson runs fuse the stencil with the projections
      WMG_TRY(Lvl<R>::post(h).fixed(D, ke, kw, p.post_smooth, st, false,
                                    sizeof(R) == 4 && !h->clov32 ? &fz : nullptr));
      WMG_TRY(axpby<R>(z, 1.0, ke, 1.0, h->nf * nrhs, 1, st));    // z += e
    }
    return MG_OK;
  };
}

int host_norms(mg_handle* h, const zd* v, int nrhs, double* out, cudaStream_t st) {
  WMG_TRY(norm2<double>(h->dscal, 1, v, h->nf, nrhs, h->rw, st));
  WMG_CUDA(cudaMemcpyAsync(h->hscal, h->dscal, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
  WMG_CUDA(cudaStreamSynchronize(st));
  for (int r = 0; r < nrhs; ++r) out[r] = h->hscal[r];
  return MG_OK;
}

int solve_impl(mg_handle* h, zd* x, const zd* b, int nrhs, double tol, int maxiter,
               mg_solve_info* info, cudaStream_t st) {
  const mg_params& p = h->p;
  WMG_TRY(ensure_solver(h, nrhs));
  h->coarse_its = 0;
  h->kcycles = 0;
  for (auto& L : h->lv) L->its = 0;
  WMG_TRY(h->csol64.take_iterations(nullptr, st));   // drop counts of an unfinished solve
  WMG_TRY(h->csol32.take_iterations(nullptr, st));
  std::vector<double> bn(nrhs), rn(nrhs);
  WMG_TRY(host_norms(h, b, nrhs, bn.data(), st));
  int outer = 0, refinements = 0;
  int status = MG_OK;
  bool r_current = false;   // r64 already holds b - D x for the returned x ...
  bool rn_current = false;  // ... and rn its norms
  Op<double> D64 = fine_op<double>(h, nrhs);
  if (p.solve_dtype == MG_C128) {
    Op<double> M = kcycle_op<double>(h, nrhs);
    int its = 0;
    status = h->outer64.solve(D64, &M, x, b, tol, p.outer_restart, maxiter, &its, st);
    outer = its;
    refinements = 1;
    if (status != MG_OK && status != MG_ENOCONV) return status;
  } else {
    // FP64 iterative refinement around the FP32 inner K-cycle FGMRES
    Op<float> D32 = fine_op<float>(h, nrhs);
    Op<float> M = kcycle_op<float>(h, nrhs);
    WMG_TRY(fill_zero<double>(x, h->nf * nrhs, st));
    WMG_CUDA(cudaMemcpyAsync(h->r64, b, h->nf * nrhs * sizeof(zd), cudaMemcpyDeviceToDevice, st));
    // every pass of the loop ends with r64 = b - D x in FP64 for the x it leaves
    r_current = true;
    double inner = p.inner_tol > 0 ? p.inner_tol : 1e-5;
    status = MG_ENOCONV;
    while (outer < maxiter && refinements < 100) {
      // the first pass's residual is b (x = 0): its norms are bn, already in dscal
      if (refinements > 0) {
        WMG_TRY(norm2<double>(h->dscal, 1, h->r64, h->nf, nrhs, h->rw, st));
        WMG_CUDA(cudaMemcpyAsync(h->hscal, h->dscal, nrhs * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
        WMG_CUDA(cudaStreamSynchronize(st));
      }
      bool done = true;
      double worst = 0;
      for (int r = 0; r < nrhs; ++r) {
        rn[r] = refinements > 0 ? h->hscal[r] : bn[r];
        if (!std::isfinite(rn[r])) return fail(MG_ENAN, "mg_solve: non-finite residual");
        done &= rn[r] <= tol * bn[r];
        worst = std::fmax(worst, rn[r] / (bn[r] > 0 ? bn[r] : 1));
      }
      if (done) { status = MG_OK; rn_current = true; break; }
      // inner tolerance: reach the target in this step if FP32 allows it
      double want = inner;
      if (worst > 0 && tol / worst > want) want = std::fmin(0.5, tol / worst);
      WMG_TRY((convert<float, double>(h->r32, h->r64, h->dscal, 1, h->nf, nrhs, st)));
      int its = 0;
      int s = h->outer32.solve(D32, &M, h->e32, h->r32, want, p.outer_restart, maxiter - outer, &its, st);
      if (s != MG_OK && s != MG_ENOCONV) return s;
      outer += its;
      ++refinements;
      WMG_TRY(accumulate_scaled<float>(x, h->e32, h->dscal, h->nf, nrhs, st));
      WMG_TRY(D64(h->t64, x, st));
      WMG_CUDA(cudaMemcpyAsync(h->r64, b, h->nf * nrhs * sizeof(zd), cudaMemcpyDeviceToDevice, st));
      WMG_TRY(axpby<double>(h->r64, -1.0, h->t64, 1.0, h->nf * nrhs, 1, st));
    }
  }
  // true residual in FP64 (the refinement loop's last one when it is current)
  if (!r_current) {
    WMG_TRY(D64(h->t64, x, st));
    WMG_CUDA(cudaMemcpyAsync(h->r64, b, h->nf * nrhs * sizeof(zd), cudaMemcpyDeviceToDevice, st));
    WMG_TRY(axpby<double>(h->r64, -1.0, h->t64, 1.0, h->nf * nrhs, 1, st));
  }
  if (!(r_current && rn_current)) WMG_TRY(host_norms(h, h->r64, nrhs, rn.data(), st));
  if (take_device_error()) return fail(MG_ETIMEOUT, "mg_solve: a bounded wait gave up");
  long long c64 = 0, c32 = 0;
  WMG_TRY(h->csol64.take_iterations(&c64, st));
  WMG_TRY(h->csol32.take_iterations(&c32, st));
  h->coarse_its += c64 + c32;
  double worst = 0;
  for (int r = 0; r < nrhs; ++r) worst = std::fmax(worst, rn[r] / (bn[r] > 0 ? bn[r] : 1));
  if (info) {
    info->outer_iterations = outer;
    info->refinements = refinements;
    info->kcycles = h->kcycles;
    info->coarse_iterations = h->coarse_its;
    info->true_residual = worst;
  }
  if (!(worst <= tol)) return fail(MG_ENOCONV, "mg_solve: tolerance not reached");
  return MG_OK;
}

// Algorithm 3 on the coarsest operator so far, D_l (l >= 1): test vectors psi = phi +
// GMRES_sweeps(D_l, -D_l phi) (Eq. 2) from Philox fields with counter word 3 = l, chiral split
// (sigma_3 halves of each site's vector) into the aggregates of L->B, streaming SVD in FP64;
// P_l (canonical phase) and its last-stream singular values into L.
int setup_level(mg_handle* h, CLevel* L, int l, int r, int n_s, cudaStream_t st) {
  const mg_params& p = h->p;
  const int k = L->k, cmax = k + r;
  const size_t ntile = (size_t)L->B.d * 2, M = L->B.M;
  const size_t fr = L->n_in * r;
  const int nsites = L->B.L[0] * L->B.L[1] * L->B.L[2] * L->B.L[3];
  zd *phi = nullptr, *psi = nullptr, *tmp = nullptr, *T0 = nullptr, *T1 = nullptr, *G = nullptr,
     *Vec = nullptr;
  double* lam = nullptr;
  Gmres<double> gm;
  int status = MG_OK;
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    dfree(phi); dfree(psi); dfree(tmp); dfree(T0); dfree(T1); dfree(G); dfree(Vec); dfree(lam);
  };
#define STEP(x) do { status = (x); if (status != MG_OK) { cleanup(); return status; } } while (0)
  STEP(dev_alloc(&phi, fr * sizeof(zd)));
  STEP(dev_alloc(&psi, fr * sizeof(zd)));
  STEP(dev_alloc(&tmp, fr * sizeof(zd)));
  STEP(dev_alloc(&T0, ntile * cmax * M * sizeof(zd)));
  STEP(dev_alloc(&T1, ntile * cmax * M * sizeof(zd)));
  STEP(dev_alloc(&G, ntile * cmax * cmax * sizeof(zd)));
  STEP(dev_alloc(&Vec, ntile * cmax * cmax * sizeof(zd)));
  STEP(dev_alloc(&lam, ntile * cmax * sizeof(double)));
  Op<double> D = level_op<double>(h, l, r);
  STEP(gm.alloc(L->n_in, r, p.sweeps > 0 ? p.sweeps : 1, false));
  zd *cur = T0, *oth = T1;
  int kk = 0;
  for (int s = 0; s < n_s; ++s) {
    STEP(gaussian_fill_n<double>(phi, p.seed, (unsigned)(s * r), r, nsites, 2 * L->k_in,
                                 (unsigned)l, st));
    STEP(D(tmp, phi, st));
    STEP(axpby<double>(tmp, 0.0, tmp, -1.0, fr, 1, st));        // tmp = -D_l phi
    STEP(gm.fixed(D, psi, tmp, p.sweeps, st));
    STEP(axpby<double>(psi, 1.0, phi, 1.0, fr, 1, st));         // psi = phi + psi'
    STEP(coarse_gather<double>(cur, cmax, kk, psi, r, L->B, L->k_in, st, false));
    const int c = kk + r, kn = c < k ? c : k;
    const bool last = s == n_s - 1;
    STEP(tile_gram(G, cur, cmax, c, L->B, st, false));
    STEP(tile_eig(lam, Vec, G, c, (int)ntile, st, 1e-15, false));
    if (p.svd_refine != 0) {
      STEP(tile_update(oth, cmax, cur, cmax, c, Vec, lam, c, 0, L->B, st, false));
      STEP(tile_gram(G, oth, cmax, c, L->B, st, false));
      STEP(tile_eig(lam, Vec, G, c, (int)ntile, st, 1e-15, false));
      STEP(tile_update(cur, cmax, oth, cmax, c, Vec, lam, kn, last ? 1 : 0, L->B, st, false));
    } else {
      STEP(tile_update(oth, cmax, cur, cmax, c, Vec, lam, kn, last ? 1 : 0, L->B, st, false));
      zd* t = cur; cur = oth; oth = t;
    }
    if (last) STEP(tile_sigma(L->sigma, k, lam, c, kn, (int)ntile, st));
    kk = kn;
  }
  STEP(tile_canonical_phase(cur, cmax, k, L->B, st, false));
  {
    cudaError_t e = cudaMemcpy2DAsync(L->P64, (size_t)k * M * sizeof(zd), cur,
                                      (size_t)cmax * M * sizeof(zd), (size_t)k * M * sizeof(zd),
                                      ntile, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) { cleanup(); return fail(MG_ECUDA, cudaGetErrorString(e)); }
  }
  STEP((convert<float, double>(L->P32, L->P64, nullptr, 0, ntile * k * M, 1, st)));
  cleanup();
  if (take_device_error()) return fail(MG_ETIMEOUT, "mg_add_level: a bounded wait gave up");
#undef STEP
  return MG_OK;
}

int check_ready(mg_handle* h, bool need_coarse) {
  if (!h) return fail(MG_EINVAL, "NULL handle");
  if (!h->have_P) return fail(MG_EINVAL, "handle has no prolongator");
  if (need_coarse && !h->have_coarse) return fail(MG_EINVAL, "coarse_build has not run");
  return MG_OK;
}

}  // namespace

mg_handle::~mg_handle() {
  free_solver();
  dfree(links64); dfree(links64L); dfree(links32L); dfree(links16L); dfree(P64); dfree(P32); dfree(sigma); dfree(hist);
  dfree(Op64); dfree(Op32); dfree(PtP); dfree(Pdf); dfree(Ldf); dfree(tc_flag);
  dfree(clov64); dfree(clov32);
}

void mg_handle::free_solver() {
  outer64.release(); coarse64.release(); post64.release();
  outer32.release(); coarse32.release(); post32.release();
  csol64.release(); csol32.release();
  posth.release(); postb.release();
  posts64.release(); posts32.release();
  for (auto& b : sbuf) dfree(b);
  for (auto& L : lv) L->free_solver();
  dfree(kwh); dfree(keh);
  dfree(x64); dfree(r64); dfree(t64); dfree(e32); dfree(r32);
  dfree(vc64); dfree(ec64); dfree(kw64); dfree(ke64);
  dfree(vc32); dfree(ec32); dfree(kw32); dfree(ke32);
  dfree(dscal);
  host_free(hscal);
  hscal = nullptr;
  rw.release();
  nrhs = 0;
}

// ============================================================================ C ABI
extern "C" int mg_create(mg_handle** h, const void* links, const mg_params* p, void* stream) {
  return create_handle(h, links, p, false, (cudaStream_t)stream);
}

extern "C" int mg_setup_streaming_svd(mg_handle** h, const void* links, const mg_params* p,
                                      void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  WMG_TRY(create_handle(h, links, p, true, st));
  int s = p->setup_dtype == MG_C128 ? run_setup<double>(*h, st) : run_setup<float>(*h, st);
  if (s != MG_OK) {
    std::string msg = mg_last_error();
    delete *h;
    *h = nullptr;
    return fail(s, msg);
  }
  return MG_OK;
}

extern "C" int mg_setup_from_vectors(mg_handle** h, const void* links, const mg_params* p,
                                     const void* vectors, int vec_dtype, int smooth,
                                     void* stream) {
  if (!vectors) return fail(MG_EINVAL, "mg_setup_from_vectors: NULL vectors");
  if (vec_dtype != MG_C128 && vec_dtype != MG_C64)
    return fail(MG_EINVAL, "mg_setup_from_vectors: vec_dtype must be MG_C128 or MG_C64");
  if (smooth != 0 && smooth != 1) return fail(MG_EINVAL, "mg_setup_from_vectors: smooth is 0 or 1");
  cudaStream_t st = (cudaStream_t)stream;
  WMG_TRY(create_handle(h, links, p, true, st));
  size_t bytes = (size_t)p->n_s * p->r * (*h)->nf * dtype_bytes(vec_dtype);
  Staged sv;
  int s = stage_in(sv, vectors, bytes, st);
  if (s == MG_OK) {
    SetupSource src{sv.dev, vec_dtype, smooth};
    s = p->setup_dtype == MG_C128 ? run_setup<double>(*h, st, &src)
                                  : run_setup<float>(*h, st, &src);
  }
  if (s != MG_OK) {
    std::string msg = mg_last_error();
    delete *h;
    *h = nullptr;
    return fail(s, msg);
  }
  return MG_OK;
}

extern "C" int mg_add_level(mg_handle* h, const int block[4], int k, int r, int n_s, double tol,
                            void* stream) {
  WMG_TRY(check_ready(h, true));
  if (!block) return fail(MG_EINVAL, "mg_add_level: NULL block");
  if (h->lv.size() >= 6) return fail(MG_EINVAL, "mg_add_level: at most 8 levels");
  cudaStream_t st = (cudaStream_t)stream;
  const int l = 1 + (int)h->lv.size();      // the level the new P starts from
  const Blocking& Bp = h->lv.empty() ? h->B : h->lv.back()->B;
  const int k_in = h->lv.empty() ? h->k : h->lv.back()->k;
  const zd* Op_in = h->lv.empty() ? h->Op64 : h->lv.back()->Op64;
  std::unique_ptr<CLevel> L(new CLevel());
  WMG_TRY(make_blocking(L->B, Bp.C, block));
  const int nd = L->B.nd;
  if (k < 1 || k > 32 || k > nd * k_in) return fail(MG_EINVAL, "mg_add_level: k in [1, min(32, n_d k_l)]");
  if (r < 1 || n_s < 1 || k + r > 64 || (long long)r * n_s < k)
    return fail(MG_EINVAL, "mg_add_level: need r, n_s >= 1, k + r <= 64, n_s r >= k");
  if (!(tol > 0 && tol < 1)) return fail(MG_EINVAL, "mg_add_level: tol in (0, 1)");
  L->B.M = nd * k_in;
  L->k_in = k_in;
  L->k = k;
  L->tol = tol;
  L->n_in = (size_t)L->B.d * nd * 2 * k_in;
  L->n = (size_t)L->B.d * 2 * k;
  const size_t ntile = (size_t)L->B.d * 2;
  WMG_TRY(dev_alloc(&L->P64, ntile * k * L->B.M * sizeof(zd)));
  WMG_TRY(dev_alloc(&L->P32, ntile * k * L->B.M * sizeof(zf)));
  WMG_TRY(dev_alloc(&L->sigma, ntile * k * sizeof(double)));
  const size_t ne = (size_t)L->B.d * 9 * 4 * k * k;
  WMG_TRY(dev_alloc(&L->Op64, ne * sizeof(zd)));
  WMG_TRY(dev_alloc(&L->Op32, ne * sizeof(zf)));
  if (h->nrhs) cudaDeviceSynchronize();
  h->free_solver();                       // the solver state is rebuilt for the new depth
  WMG_TRY(setup_level(h, L.get(), l, r, n_s, st));
  WMG_TRY(coarse_galerkin(L->Op64, Op_in, L->P64, L->B, k_in, k, st));
  WMG_TRY((convert<float, double>(L->Op32, L->Op64, nullptr, 0, ne, 1, st)));
  WMG_CUDA(cudaStreamSynchronize(st));
  h->lv.push_back(std::move(L));
  return MG_OK;
}

extern "C" int mg_num_levels(const mg_handle* h) {
  if (!h) return 0;
  return h->have_coarse ? 2 + (int)h->lv.size() : 1;
}

extern "C" int mg_level_iterations(const mg_handle* h, long long* its, int nmax) {
  if (!h || !its) return fail(MG_EINVAL, "mg_level_iterations: NULL argument");
  int n = 1 + (int)h->lv.size();
  for (int i = 0; i < n && i < nmax; ++i) its[i] = i == 0 ? h->coarse_its : h->lv[i - 1]->its;
  return MG_OK;
}

extern "C" int mg_setup_ls(mg_handle** h, const void* links, const mg_params* p,
                           const double* omega, void* stream) {
  if (!p || !omega) return fail(MG_EINVAL, "mg_setup_ls: NULL argument");
  if (p->n_s != 1) return fail(MG_EINVAL, "mg_setup_ls: Eq. 9 uses every test vector at once: n_s = 1");
  if (p->r < p->k) return fail(MG_EINVAL, "mg_setup_ls: r >= k");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> w(p->r);
  {
    cudaPointerAttributes at{};
    bool dev = cudaPointerGetAttributes(&at, omega) == cudaSuccess &&
               (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev) WMG_CUDA(cudaMemcpy(w.data(), omega, p->r * sizeof(double), cudaMemcpyDeviceToHost));
    else std::memcpy(w.data(), omega, p->r * sizeof(double));
  }
  for (double x : w)
    if (!(x > 0) || !std::isfinite(x)) return fail(MG_EINVAL, "mg_setup_ls: weights must be positive");
  WMG_TRY(create_handle(h, links, p, true, st));
  double* dw = nullptr;
  int s = dev_alloc(&dw, p->r * sizeof(double));
  if (s == MG_OK) {
    cudaError_t e = cudaMemcpyAsync(dw, w.data(), p->r * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) s = fail(MG_ECUDA, cudaGetErrorString(e));
  }
  if (s == MG_OK)
    s = p->setup_dtype == MG_C128 ? run_setup<double>(*h, st, nullptr, dw)
                                  : run_setup<float>(*h, st, nullptr, dw);
  cudaStreamSynchronize(st);
  dfree(dw);
  if (s != MG_OK) {
    std::string msg = mg_last_error();
    delete *h;
    *h = nullptr;
    return fail(s, msg);
  }
  return MG_OK;
}

extern "C" int coarse_build(mg_handle* h, void* stream) {
  WMG_TRY(check_ready(h, false));
  cudaStream_t st = (cudaStream_t)stream;
  size_t ne = (size_t)4 * h->k * h->k;
  if (!h->Op64) {
    WMG_TRY(dev_alloc(&h->Op64, (size_t)h->B.d * 9 * ne * sizeof(zd)));
    WMG_TRY(dev_alloc(&h->Op32, (size_t)h->B.d * 9 * ne * sizeof(zf)));
  }
  if (!h->lv.empty()) {
    // the levels below were built from the operator this call replaces
    cudaDeviceSynchronize();
    h->free_solver();
    h->lv.clear();
  }
  zd* Xpart = nullptr;
  WMG_CUDA(cudaMallocAsync(&Xpart, (size_t)4 * h->B.d * ne * sizeof(zd), st));
  bool df = galerkin_df(h->p);
  int s = galerkin_build(h->Op64, Xpart, h->P64, h->Pdf, h->PtP, h->k, h->links64, h->Ldf, h->g,
                         h->B, st, df, h->pdf_ready, h->tc_flag);
  cudaFreeAsync(Xpart, st);
  WMG_TRY(s);
  if (h->clov64) WMG_TRY(clover_galerkin_add(h->Op64, h->P64, h->clov64, h->k, h->B, st));
  WMG_TRY((convert<float, double>(h->Op32, h->Op64, nullptr, 0, (size_t)h->B.d * 9 * ne, 1, st)));
  WMG_CUDA(cudaStreamSynchronize(st));
  h->have_coarse = true;
  return MG_OK;
}

// ---------------------------------------------------------------------------------------
// coarse_build_noalloc: the same Galerkin rebuild with the forward-hop partials kept in a
// fixed device array instead of a per-call allocation.  Nothing in the array has to start
// at zero: galerkin_hop_kernel writes every partial before galerkin_finish_kernel reads it.
static __device__ __align__(256) unsigned char g_galerkin_scratch[(size_t)24 << 20];

namespace {

constexpr size_t kGalerkinScratchBytes = sizeof(g_galerkin_scratch);
constexpr int kScratchMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kScratchMaxDevices] = {};

// Device address of the scratch array on the current device, looked up on the first call
// per device (with that device current) and cached.
int galerkin_scratch(void** out) {
  int dev = 0;
  WMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kScratchMaxDevices)
    return fail(MG_EINVAL, "coarse_build_noalloc: device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_galerkin_scratch);
    if (e != cudaSuccess || !p)
      return fail(MG_ECUDA, std::string("coarse_build_noalloc: cudaGetSymbolAddress failed: ") +
                                cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return MG_OK;
}

}  // namespace

extern "C" int coarse_build_noalloc(mg_handle* h, void* stream) {
  WMG_TRY(check_ready(h, false));
  cudaStream_t st = (cudaStream_t)stream;
  size_t ne = (size_t)4 * h->k * h->k;
  size_t need = (size_t)4 * h->B.d * ne * sizeof(zd);
  if (need > kGalerkinScratchBytes)
    return fail(MG_EINVAL, "coarse_build_noalloc: the Galerkin partials need " +
                               std::to_string(need) + " bytes but the fixed scratch holds " +
                               std::to_string(kGalerkinScratchBytes) +
                               " (coarse sites * k^2 must be <= 98304); use coarse_build");
  if (!h->Op64 || !h->Op32)
    return fail(MG_EINVAL, "coarse_build_noalloc: the handle has no coarse-operator storage "
                           "yet; call coarse_build once first (it allocates that storage)");
  if (!h->lv.empty())
    return fail(MG_EINVAL, "coarse_build_noalloc: the handle has levels below level 1 "
                           "(mg_add_level), which a new level-1 operator would leave stale; "
                           "use coarse_build, which drops them");
  void* scratch = nullptr;
  WMG_TRY(galerkin_scratch(&scratch));
  bool df = galerkin_df(h->p);
  WMG_TRY(galerkin_build(h->Op64, static_cast<zd*>(scratch), h->P64, h->Pdf, h->PtP, h->k,
                         h->links64, h->Ldf, h->g, h->B, st, df, h->pdf_ready, h->tc_flag));
  if (h->clov64) WMG_TRY(clover_galerkin_add(h->Op64, h->P64, h->clov64, h->k, h->B, st));
  WMG_TRY((convert<float, double>(h->Op32, h->Op64, nullptr, 0, (size_t)h->B.d * 9 * ne, 1, st)));
  WMG_CUDA(cudaStreamSynchronize(st));
  h->have_coarse = true;
  return MG_OK;
}

static int solve_entry(mg_handle* h, void* x, const void* b, int nrhs, double tol, int maxiter,
                       mg_solve_info* info, void* stream, bool adjoint) {
  WMG_TRY(check_ready(h, true));
  if (!x || !b) return fail(MG_EINVAL, "mg_solve: NULL field");
  if (nrhs < 1 || nrhs > 64) return fail(MG_EINVAL, "mg_solve: nrhs in [1, 64]");
  if (!(tol > 0)) return fail(MG_EINVAL, "mg_solve: tol must be > 0");
  if (maxiter < 1) return fail(MG_EINVAL, "mg_solve: maxiter < 1");
  cudaStream_t st = (cudaStream_t)stream;
  size_t fb = h->nf * nrhs * sizeof(zd);
  Staged sb, sx;
  WMG_TRY(stage_in(sb, b, fb, st));
  WMG_TRY(stage_out_alloc(sx, x, fb, st));
  const zd* bb = (const zd*)sb.dev;
  zd* gb = nullptr;
  if (adjoint) {
    WMG_CUDA(cudaMallocAsync(&gb, fb, st));
    WMG_TRY(apply_gamma5<double>(gb, bb, (size_t)h->g.V * nrhs, st));
    bb = gb;
  }
  int s = solve_impl(h, (zd*)sx.dev, bb, nrhs, tol, maxiter, info, st);
  if (adjoint) {
    if (s == MG_OK || s == MG_ENOCONV) {
      int s2 = apply_gamma5<double>((zd*)sx.dev, (const zd*)sx.dev, (size_t)h->g.V * nrhs, st);
      if (s2 != MG_OK) s = s2;
    }
    cudaFreeAsync(gb, st);
  }
  if (s != MG_OK && s != MG_ENOCONV) return s;
  std::string msg = s == MG_ENOCONV ? std::string(mg_last_error()) : std::string();
  WMG_TRY(stage_out_finish(sx, x, fb, st));
  WMG_CUDA(cudaStreamSynchronize(st));
  if (s == MG_ENOCONV) return fail(s, msg);
  return MG_OK;
}

extern "C" int mg_solve(mg_handle* h, void* x, const void* b, int nrhs, double tol, int maxiter,
                        mg_solve_info* info, void* stream) {
  return solve_entry(h, x, b, nrhs, tol, maxiter, info, stream, false);
}

extern "C" int mg_solve_adjoint(mg_handle* h, void* x, const void* b, int nrhs, double tol,
                                int maxiter, mg_solve_info* info, void* stream) {
  return solve_entry(h, x, b, nrhs, tol, maxiter, info, stream, true);
}

extern "C" int mg_destroy(mg_handle* h) {
  if (!h) return MG_OK;
  cudaDeviceSynchronize();
  delete h;
  return MG_OK;
}

extern "C" int mg_test_vectors(void* out, const void* links, const mg_params* p, int stream_index,
                               void* stream) {
  if (!out) return fail(MG_EINVAL, "mg_test_vectors: NULL output");
  if (!p || stream_index < 0 || stream_index >= p->n_s)
    return fail(MG_EINVAL, "mg_test_vectors: stream index out of range");
  cudaStream_t st = (cudaStream_t)stream;
  mg_handle* h = nullptr;
  WMG_TRY(create_handle(&h, links, p, true, st));
  std::unique_ptr<mg_handle> guard(h);
  size_t fr = h->nf * p->r;
  Staged so;
  WMG_TRY(stage_out_alloc(so, out, fr * sizeof(zd), st));
  if (p->setup_dtype == MG_C128) {
    zd* tmp;
    WMG_CUDA(cudaMallocAsync(&tmp, fr * sizeof(zd), st));
    Gmres<double> gm;
    int s = smooth_stream<double>(h, (zd*)so.dev, tmp, gm, stream_index, st);
    cudaStreamSynchronize(st);
    cudaFreeAsync(tmp, st);
    WMG_TRY(s);
  } else {
    zf *tmp, *psi;
    WMG_CUDA(cudaMallocAsync(&tmp, fr * sizeof(zf), st));
    WMG_CUDA(cudaMallocAsync(&psi, fr * sizeof(zf), st));
    Gmres<float> gm;
    int s = smooth_stream<float>(h, psi, tmp, gm, stream_index, st);
    if (s == MG_OK) s = convert<double, float>((zd*)so.dev, psi, nullptr, 0, fr, 1, st);
    cudaStreamSynchronize(st);
    cudaFreeAsync(tmp, st);
    cudaFreeAsync(psi, st);
    WMG_TRY(s);
  }
  WMG_TRY(stage_out_finish(so, out, fr * sizeof(zd), st));
  WMG_CUDA(cudaStreamSynchronize(st));
  return MG_OK;
}

extern "C" int mg_link_rows(const mg_handle* h) { return h ? (h->llay == 2 ? 2 : 3) : 0; }

extern "C" int mg_apply_fine(mg_handle* h, void* out, const void* in, int nrhs, int dtype,
                             int dagger, void* stream) {
  if (!h || !out || !in || nrhs < 1) return fail(MG_EINVAL, "mg_apply_fine: bad arguments");
  if (out == in) return fail(MG_EINVAL, "mg_apply_fine: out must not alias in");
  bool half = dtype == MG_F16 || dtype == MG_BF16;
  if (dtype != MG_C128 && dtype != MG_C64 && !half) return fail(MG_EINVAL, "mg_apply_fine: dtype");
  if (half && dtype != h->p.solve_dtype)
    return fail(MG_EINVAL, "mg_apply_fine: half storage needs a handle with that solve_dtype");
  cudaStream_t st = (cudaStream_t)stream;
  size_t bytes = h->nf * nrhs * dtype_bytes(dtype);
  Staged si, so;
  WMG_TRY(stage_in(si, in, bytes, st));
  WMG_TRY(stage_out_alloc(so, out, bytes, st));
  const void* L = dtype == MG_C128 ? (const void*)h->links64L
                  : dtype == MG_C64 ? (const void*)h->links32L : (const void*)h->links16L;
  WMG_TRY(dslash_launch(dtype, so.dev, si.dev, L, h->g, -1, dagger, nrhs, st, h->nf, h->nf,
                        dtype == MG_C128 ? 1 : h->llay));
  // the clover term is Hermitian: the same for D and D^dag
  if (dtype == MG_C128 && h->clov64)
    WMG_TRY(clover_add<double>((zd*)so.dev, (const zd*)si.dev, h->clov64, h->g.V, nrhs, st));
  else if (dtype == MG_C64 && h->clov32)
    WMG_TRY(clover_add<float>((zf*)so.dev, (const zf*)si.dev, h->clov32, h->g.V, nrhs, st));
  WMG_TRY(stage_out_finish(so, out, bytes, st));
  return MG_OK;
}

extern "C" int mg_get_prolongator(mg_handle* h, void* P, void* sigma, void* stream) {
  WMG_TRY(check_ready(h, false));
  cudaStream_t st = (cudaStream_t)stream;
  size_t pb = (size_t)h->B.d * 2 * h->k * h->B.M * sizeof(zd);
  if (P) WMG_CUDA(cudaMemcpyAsync(P, h->P64, pb, cudaMemcpyDefault, st));
  if (sigma)
    WMG_CUDA(cudaMemcpyAsync(sigma, h->sigma, (size_t)h->B.d * 2 * h->k * sizeof(double),
                             cudaMemcpyDefault, st));
  WMG_CUDA(cudaStreamSynchronize(st));
  return MG_OK;
}

extern "C" int mg_get_sigma_history(mg_handle* h, void* hist, void* stream) {
  WMG_TRY(check_ready(h, false));
  if (!hist) return fail(MG_EINVAL, "NULL output");
  cudaStream_t st = (cudaStream_t)stream;
  size_t n = (size_t)h->p.n_s * h->B.d * 2 * h->k * sizeof(double);
  WMG_CUDA(cudaMemcpyAsync(hist, h->hist, n, cudaMemcpyDefault, st));
  WMG_CUDA(cudaStreamSynchronize(st));
  return MG_OK;
}

extern "C" int mg_set_prolongator(mg_handle* h, const void* P, void* stream) {
  if (!h || !P) return fail(MG_EINVAL, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  size_t ne = (size_t)h->B.d * 2 * h->k * h->B.M;
  WMG_CUDA(cudaMemcpyAsync(h->P64, P, ne * sizeof(zd), cudaMemcpyDefault, st));
  WMG_TRY((convert<float, double>(h->P32, h->P64, nullptr, 0, ne, 1, st)));
  WMG_CUDA(cudaStreamSynchronize(st));
  h->have_P = true;
  h->have_coarse = false;
  h->pdf_ready = false;
  if (!h->lv.empty()) {
    cudaDeviceSynchronize();
    h->free_solver();
    h->lv.clear();
  }
  return MG_OK;
}

extern "C" int mg_restrict(mg_handle* h, void* vc, const void* v, int nrhs, void* stream) {
  WMG_TRY(check_ready(h, false));
  if (!vc || !v || nrhs < 1) return fail(MG_EINVAL, "mg_restrict: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  Staged si, so;
  WMG_TRY(stage_in(si, v, h->nf * nrhs * sizeof(zd), st));
  WMG_TRY(stage_out_alloc(so, vc, h->nc * nrhs * sizeof(zd), st));
  WMG_TRY(restrict_launch<double>((zd*)so.dev, (const zd*)si.dev, h->P64, h->k, h->B, nrhs, st));
  WMG_TRY(stage_out_finish(so, vc, h->nc * nrhs * sizeof(zd), st));
  return MG_OK;
}

extern "C" int mg_prolong(mg_handle* h, void* v, const void* vc, int nrhs, void* stream) {
  WMG_TRY(check_ready(h, false));
  if (!vc || !v || nrhs < 1) return fail(MG_EINVAL, "mg_prolong: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  Staged si, so;
  WMG_TRY(stage_in(si, vc, h->nc * nrhs * sizeof(zd), st));
  WMG_TRY(stage_out_alloc(so, v, h->nf * nrhs * sizeof(zd), st));
  WMG_TRY(prolong_launch<double>((zd*)so.dev, (const zd*)si.dev, h->P64, h->k, h->B, nrhs, st));
  WMG_TRY(stage_out_finish(so, v, h->nf * nrhs * sizeof(zd), st));
  return MG_OK;
}

namespace {
__global__ void export_coarse_kernel(zd* X, zd* Y, const zd* Op, int n2k, int d) {
  size_t ne = (size_t)n2k * n2k;
  size_t total = (size_t)d * 9 * ne;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t j = e / (9 * ne), rem = e % (9 * ne);
    int blk = (int)(rem / ne);
    size_t q = rem % ne;
    int b = (int)(q / n2k), a = (int)(q % n2k);   // Op is column-major
    zd v = Op[e];
    if (blk == 0) X[j * ne + (size_t)a * n2k + b] = v;
    else Y[((size_t)(blk - 1) * d + j) * ne + (size_t)a * n2k + b] = v;
  }
}
}  // namespace

extern "C" int mg_get_coarse_op(mg_handle* h, void* X, void* Y, void* stream) {
  WMG_TRY(check_ready(h, true));
  if (!X || !Y) return fail(MG_EINVAL, "NULL output");
  cudaStream_t st = (cudaStream_t)stream;
  size_t ne = (size_t)4 * h->k * h->k;
  Staged sx, sy;
  WMG_TRY(stage_out_alloc(sx, X, (size_t)h->B.d * ne * sizeof(zd), st));
  WMG_TRY(stage_out_alloc(sy, Y, (size_t)8 * h->B.d * ne * sizeof(zd), st));
  export_coarse_kernel<<<256, 256, 0, st>>>((zd*)sx.dev, (zd*)sy.dev, h->Op64, 2 * h->k, h->B.d);
  WMG_LAUNCHED();
  WMG_TRY(stage_out_finish(sx, X, (size_t)h->B.d * ne * sizeof(zd), st));
  WMG_TRY(stage_out_finish(sy, Y, (size_t)8 * h->B.d * ne * sizeof(zd), st));
  WMG_CUDA(cudaStreamSynchronize(st));
  return MG_OK;
}

extern "C" int mg_get_level(mg_handle* h, int level, void* P, void* sigma, void* X, void* Y,
                            void* stream) {
  if (!h) return fail(MG_EINVAL, "NULL handle");
  if (level < 2 || level - 2 >= (int)h->lv.size())
    return fail(MG_EINVAL, "mg_get_level: level must be one added by mg_add_level (>= 2)");
  CLevel* L = h->lv[level - 2].get();
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ntile = (size_t)L->B.d * 2;
  if (P) WMG_CUDA(cudaMemcpyAsync(P, L->P64, ntile * L->k * L->B.M * sizeof(zd), cudaMemcpyDefault, st));
  if (sigma) WMG_CUDA(cudaMemcpyAsync(sigma, L->sigma, ntile * L->k * sizeof(double), cudaMemcpyDefault, st));
  if (X || Y) {
    if (!X || !Y) return fail(MG_EINVAL, "mg_get_level: X and Y go together");
    size_t ne = (size_t)4 * L->k * L->k;
    Staged sx, sy;
    WMG_TRY(stage_out_alloc(sx, X, (size_t)L->B.d * ne * sizeof(zd), st));
    WMG_TRY(stage_out_alloc(sy, Y, (size_t)8 * L->B.d * ne * sizeof(zd), st));
    export_coarse_kernel<<<256, 256, 0, st>>>((zd*)sx.dev, (zd*)sy.dev, L->Op64, 2 * L->k, L->B.d);
    WMG_LAUNCHED();
    WMG_TRY(stage_out_finish(sx, X, (size_t)L->B.d * ne * sizeof(zd), st));
    WMG_TRY(stage_out_finish(sy, Y, (size_t)8 * L->B.d * ne * sizeof(zd), st));
  }
  WMG_CUDA(cudaStreamSynchronize(st));
  return MG_OK;
}

extern "C" int mg_coarse_apply(mg_handle* h, void* y, const void* x, int nrhs, int dtype,
                               void* stream) {
  WMG_TRY(check_ready(h, true));
  if (!x || !y || nrhs < 1) return fail(MG_EINVAL, "mg_coarse_apply: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  size_t n = h->nc * nrhs;
  if (dtype == MG_C128) {
    Staged si, so;
    WMG_TRY(stage_in(si, x, n * sizeof(zd), st));
    WMG_TRY(stage_out_alloc(so, y, n * sizeof(zd), st));
    WMG_TRY(coarse_apply_launch<double>((zd*)so.dev, (const zd*)si.dev, h->Op64, h->k, h->B, nrhs, st));
    WMG_TRY(stage_out_finish(so, y, n * sizeof(zd), st));
  } else if (dtype == MG_C64) {
    Staged si, so;
    WMG_TRY(stage_in(si, x, n * sizeof(zf), st));
    WMG_TRY(stage_out_alloc(so, y, n * sizeof(zf), st));
    WMG_TRY(coarse_apply_launch<float>((zf*)so.dev, (const zf*)si.dev, h->Op32, h->k, h->B, nrhs, st));
    WMG_TRY(stage_out_finish(so, y, n * sizeof(zf), st));
  } else {
    return fail(MG_EINVAL, "mg_coarse_apply: dtype must be MG_C128 or MG_C64");
  }
  return MG_OK;
}
