/*
 * wilson_mg.h -- C ABI of the GB300 streaming chiral-SVD multigrid library.
 *
 * Method: Whyte, Stathopoulos, Romero, "Accelerating multigrid with streaming chiral
 * SVD for Wilson fermions in lattice QCD" (arXiv:2505.14399).  The library solves
 * D x = b (Eq. 1) for the Wilson-Dirac operator D with a two-level multigrid
 * preconditioner whose prolongator comes from the streaming chiral SVD (iCSVD,
 * Algorithm 3) and whose coarse operator is the Galerkin product P^dag D P (Eq. 5),
 * used in a K-cycle inside flexible GMRES (Sec. 2.1, Sec. 4).
 *
 * Conventions (the paper states none of them; Eq. 3 fixes only that spins 1,2 and
 * 3,4 are the two chiralities):
 *   - dims = {Lx, Ly, Lz, Lt}; mu = 0..3 = x, y, z, t;
 *     site s = x + Lx*(y + Ly*(z + Lz*t)); parity (x+y+z+t) mod 2.
 *   - spinor fields: [site][spin 4][colour 3] complex, (re, im) interleaved;
 *     nrhs fields are stored one after another.
 *   - gauge links: [mu][site][3][3] complex row-major; U_mu(x) connects x to x+mu.
 *   - D psi(x) = psi(x) - kappa sum_mu w_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                                          + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
 *     in the chiral basis gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
 *     gamma_4 = [[0, 1], [1, 0]], gamma_5 = diag(1, 1, -1, -1); a hop that wraps
 *     around the lattice in direction mu is multiplied by bc_phase[mu] (+1 or -1).
 *   - coarse vectors: [coarse site][chirality 2][k] complex; coarse site index
 *     j = cx + Cx*(cy + Cy*(cz + Cz*ct)) with C = dims / block.
 *
 * Pointers: every field argument may be device memory or host memory (pageable
 * or pinned); host buffers are staged through device memory on the given stream.
 * `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 * asynchronous on that stream unless stated otherwise.  The caller owns every
 * buffer it passes; the library owns mg_handle and everything inside it.  Device and
 * pinned host memory the library releases (mg_destroy, a solver resized for another
 * nrhs) stays in a process-wide cache and is reused by later handles; the cache is handed
 * back to the driver when an allocation fails.
 *
 * Errors: every call returns an mg_status; no exception or device trap crosses
 * the ABI.  mg_last_error() gives a thread-local message for the last failure.
 */
#ifndef WILSON_MG_H
#define WILSON_MG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mg_status {
  MG_OK = 0,
  MG_EINVAL = 1,    /* bad dimensions, sizes, parameters or NULL pointers      */
  MG_ENOMEM = 2,    /* device allocation failed                                */
  MG_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed             */
  MG_ENOCONV = 4,   /* solver stopped at maxiter; x holds the best iterate     */
  MG_ETIMEOUT = 5,  /* a bounded device-side wait gave up                      */
  MG_ENAN = 6       /* a NaN/Inf residual was detected                         */
} mg_status;

/* storage types of complex fields */
typedef enum mg_dtype {
  MG_C128 = 0,      /* complex double                                          */
  MG_C64 = 1,       /* complex float                                           */
  MG_F16 = 2,       /* complex IEEE half storage, FP32 arithmetic              */
  MG_BF16 = 3       /* complex bfloat16 storage, FP32 arithmetic               */
} mg_dtype;

typedef struct mg_handle mg_handle;

/* Parameters of the hierarchy and of the solve.  Paper symbols: k, r, n_s
 * (Algorithm 3/4), aggregates Lambda_j of extent `block` (Sec. 2.1). */
typedef struct mg_params {
  int dims[4];               /* fine lattice extents                                    */
  int block[4];              /* aggregate extents; dims[mu] % block[mu] == 0           */
  double kappa;              /* hopping parameter                                       */
  double hop_weight[4];      /* w_mu (anisotropy), 1 for isotropic                      */
  int bc_phase[4];           /* +1 periodic, -1 antiperiodic                             */
  int k;                     /* singular vectors kept per aggregate and chirality        */
  int r;                     /* test vectors generated per stream                        */
  int n_s;                   /* number of streams                                        */
  int sweeps;                /* smoother GMRES steps per test vector (Eq. 2)             */
  unsigned long long seed;   /* Philox key of the random initial guesses                 */
  int setup_dtype;           /* MG_C128 or MG_C64: arithmetic of the setup smoother      */
  int solve_dtype;           /* MG_C128: plain FP64 solve; MG_C64: inner FGMRES +
                                K-cycle in FP32 inside FP64 iterative refinement;
                                MG_F16 / MG_BF16: the same with the K-cycle's
                                post-smoother (its residual, Krylov basis and stencil,
                                links included) in that half storage, FP32 arithmetic   */
  int post_smooth;           /* post-smoother GMRES steps in the K-cycle (8, Sec. 4)     */
  double coarse_tol;         /* coarse solve relative tolerance (0.03, Sec. 4)           */
  int coarse_restart;        /* coarse GMRES restart length                              */
  int coarse_maxiter;        /* coarse GMRES iteration cap per K-cycle                   */
  int outer_restart;         /* fine FGMRES restart length                               */
  double inner_tol;          /* inner relative tolerance of mixed-precision refinement   */
  int svd_refine;            /* 1: second Gram pass per SVD update (accuracy of the Gram
                                route restored to that of a direct SVD); 0: one pass;
                                -1: second pass only when setup_dtype is MG_C128 (FP32
                                test vectors carry 1e-7 of their own error)              */
  int coarse_persistent;     /* 1: coarse GMRES as one persistent cooperative kernel
                                (bounded grid barriers) when the coarse system fits one
                                grid (<= 2048 coarse rows per SM), else one launch per
                                operation; 0: always one launch per operation            */
  int fp64_emulation;        /* arithmetic of the SVD Gram, eigen-rotations and update
                                and of the Galerkin contraction: 1 double-float on FP32
                                units (~2^-48 relative), 0 native FP64; -1 double-float
                                only in the mixed forms (SVD: setup_dtype MG_C64;
                                Galerkin: solve_dtype other than MG_C128).  A double-float
                                Galerkin with k <= 24 runs its contraction on the tensor
                                pipe as exact bf16 digit products (same accuracy) when
                                every entry is in range (orthonormal P, unitary links),
                                else on the FP32 units                                   */
  int link_compress;         /* link copies of the FP32 / half stencils: 1 keep the first
                                two rows of each link and rebuild the third as the complex
                                conjugate of their cross product (exact for SU(3): 12 of
                                the 18 reals per link are read); 0 keep all three rows;
                                -1 two rows when every link is SU(3) to 1e-9, else three.
                                1 on links that are not SU(3) to 1e-9 gives MG_EINVAL.
                                The FP64 stencil always keeps three rows               */
  double csw;                /* clover coefficient c_sw: 0 for the Wilson operator, else
                                D = D_W + C with the clover term C of wilson_clover_field
                                in every stencil, the setup and the Galerkin diagonal
                                (Configuration B of Sec. 4); needs schur_smoother = 0 and
                                solve_dtype MG_C128 / MG_C64                             */
  int schur_smoother;        /* 1: the K-cycle post-smoother solves the even-odd Schur
                                system D_hat e_e = r_e + kappa H_eo r_o with post_smooth
                                GMRES steps and reconstructs e_o = r_o + kappa H_oe e_e
                                (even-odd preconditioning, Sec. 1); 0: GMRES on D      */
} mg_params;

typedef struct mg_solve_info {
  int outer_iterations;      /* fine-level FGMRES iterations over all refinement steps   */
  int refinements;           /* FP64 refinement steps (1 for the plain FP64 solve)       */
  int kcycles;               /* preconditioner applications                              */
  long long coarse_iterations;  /* coarse GMRES iterations, summed over K-cycles and RHS */
  double true_residual;      /* ||b - D x|| / ||b|| in FP64, per the last RHS checked    */
} mg_solve_info;

/* Defaults: k = 24, r = 24, n_s = 2, sweeps = 5, post_smooth = 8, coarse_tol = 0.03,
 * coarse_restart = 32, coarse_maxiter = 2000, outer_restart = 16, inner_tol = 1e-5,
 * setup_dtype = MG_C64, solve_dtype = MG_C64, svd_refine = -1, coarse_persistent = 1,
 * fp64_emulation = -1, link_compress = -1, schur_smoother = 0,
 * isotropic periodic. */
void mg_params_default(mg_params* p);

/* Thread-local message describing the most recent non-MG_OK return. */
const char* mg_last_error(void);

/* Number of kernels this library has launched since load (diagnostic counter). */
long long mg_kernel_launches(void);

/* JSON list of the launch shapes the autotuner has chosen so far, one object per problem key
 * ("kernel": "dslash" | "dslash_proj" | "galerkin_tc", the key fields, "variant", "ms");
 * library-owned string, valid until the next call. */
const char* mg_autotune_report(void);

/* Per-kernel timing: enable = 1 brackets every subsequent instrumented launch with CUDA
 * events on its own stream (capacity max_launches, 0 = 100000) and clears earlier records;
 * enable = 0 stops recording.  mg_profile_report() synchronises on the recorded events and
 * returns a JSON object {kernel: {launches, ms, bytes, flops}} with the algorithmic bytes
 * and flops of the recorded launches (library-owned string, valid until the next call). */
int mg_profile_enable(int enable, int max_launches);
const char* mg_profile_report(void);

/* Failure-path self-test: runs the grid barrier used by the persistent coarse solver with
 * an arrival count that is never reached, so its bounded wait expires (a few ms).  Returns
 * MG_ETIMEOUT when the timeout is reported to the host as designed; the CUDA context stays
 * usable.  No fault, trap or unbounded wait is involved. */
int mg_selftest_barrier_timeout(void* stream);

/* Arithmetic-rate probe (diagnostic; synchronises `stream`): runs independent FMA chains on
 * every SM (dtype MG_C128: FP64, MG_C64: FP32) for about 15 ms per launch and writes the
 * best of three timed launches as TFLOP/s (2 flops per FMA) to *tflops.  These are the
 * measured denominators of the ALU-bound kernels' rooflines. */
int mg_probe_fma_peak(int dtype, double* tflops, void* stream);

/* ---------------------------------------------------------------------------------
 * wilson_dslash -- the Wilson-Dirac stencil (the operator of Eq. 1).
 *   parity = -1: out = D in (or D^dag in if dagger), full-lattice fields of V sites.
 *   parity = 0 / 1: out_p = -kappa H_{p,1-p} in_{1-p}: half-lattice fields of V/2
 *     sites, ordered by checkerboard index site/2 (requires every dims[mu] even).
 *   dtype: storage of out, in and links (all the same); MG_F16 / MG_BF16 accumulate
 *   in FP32.  nrhs fields are processed in one launch sharing the links.
 * Returns MG_EINVAL for bad dims / dtype / nrhs < 1 / NULL pointers.
 * ------------------------------------------------------------------------------- */
int wilson_dslash(void* out, const void* in, const void* links, const int dims[4],
                  double kappa, const double hop_weight[4], const int bc_phase[4],
                  int parity, int dagger, int dtype, int nrhs, void* stream);

/* ---------------------------------------------------------------------------------
 * wilson_schur -- the even-odd Schur complement of D (even-odd preconditioning, Sec. 1):
 *   out_e = D_hat in_e = in_e - kappa^2 H_eo H_oe in_e   (dagger: D_hat^dag in_e),
 * where -kappa H_{p,1-p} is the single-parity hop of wilson_dslash(parity = p).  With it,
 * D x = b is solved as D_hat x_e = b_e + kappa H_eo b_o, x_o = b_o + kappa H_oe x_e.
 *   in, out: even half-lattice fields of V/2 sites (checkerboard index site / 2), nrhs of
 *   them; links: [mu][site][3][3] in the same dtype; every dims[mu] even.
 * Allocates one odd half-lattice temporary on `stream` (stream-ordered).
 * Returns MG_EINVAL for bad dims / dtype / nrhs < 1 / NULL or aliased pointers.
 * ------------------------------------------------------------------------------- */
int wilson_schur(void* out, const void* in, const void* links, const int dims[4],
                 double kappa, const double hop_weight[4], const int bc_phase[4],
                 int dagger, int dtype, int nrhs, void* stream);

/* ---------------------------------------------------------------------------------
 * wilson_clover_field -- the clover term of the Wilson-clover operator (the action of
 * Configuration B, Sec. 4; the paper writes no term, this is the textbook form):
 *   C(x) = -kappa c_sw sum_{mu<nu} sigma_mu_nu (x) F_mu_nu(x),  sigma_mu_nu = (i/2)[g_mu, g_nu],
 *   F_mu_nu(x) = traceless part of (Q - Q^dag) / (8 i), Q the four plaquettes of the mu-nu
 *   plane that start and end at x, counter-clockwise; periodic gauge field.
 * sigma_mu_nu commutes with gamma_5, so C is two 6 x 6 Hermitian blocks per site:
 *   clover: out, [site][alpha][6][6] complex double, rows/columns (spin within the
 *   chirality, colour), alpha = 0 for spins 1,2 and 1 for spins 3,4;
 *   links: complex double [mu][site][3][3].  FP64 arithmetic.
 * ------------------------------------------------------------------------------- */
int wilson_clover_field(void* clover, const void* links, const int dims[4], double kappa,
                        double csw, void* stream);

/* out = D_W in + C in (dagger: D_W^dag in + C in; C is Hermitian), full-lattice fields,
 * dtype MG_C128 or MG_C64 for out, in, links and clover (layouts as above). */
int wilson_clover_apply(void* out, const void* in, const void* links, const void* clover,
                        const int dims[4], double kappa, const double hop_weight[4],
                        const int bc_phase[4], int dagger, int dtype, int nrhs, void* stream);

/* ---------------------------------------------------------------------------------
 * mg_setup_streaming_svd -- Algorithm 4 up to P: iCSVD (Algorithm 3) on the fine
 * operator.  For s = 0..n_s-1: r Philox complex-Gaussian phi_i (vector ids s*r+i),
 * psi_i = phi_i + GMRES_sweeps(D, -D phi_i) (Eq. 2); chiral split into aggregates
 * (Eq. 3); per aggregate and chirality Phi_s = rank-k SVD([Phi_{s-1}, Psi_s]) (Eq. 8)
 * kept as U_k Sigma_k (Eq. 7); after the last stream P = U_k (Eq. 6), each column
 * with the canonical phase "sum of entries real positive".
 * links: complex double [mu][site][3][3]; copied into the handle.
 * Creates *h (must be NULL on entry).  Synchronises `stream` before returning.
 * MG_EINVAL: dims not divisible by block, k > 6*prod(block), k+r > 64,
 *            n_s*r < k, odd dims, bad dtypes.
 * ------------------------------------------------------------------------------- */
int mg_setup_streaming_svd(mg_handle** h, const void* links, const mg_params* p,
                           void* stream);

/* ---------------------------------------------------------------------------------
 * mg_setup_from_vectors -- the same iCSVD setup (Algorithm 3) on vectors the caller
 * supplies instead of the Philox fields: stream s takes fields s*r .. s*r+r-1 of
 *   vectors: n_s * r fields [field][site][4][3], complex double (vec_dtype MG_C128) or
 *            complex float (MG_C64), device or host memory, read only during the call;
 *   smooth = 1: each field is an initial guess phi, smoothed into psi = phi +
 *            GMRES_sweeps(D, -D phi) (Eq. 2) in setup_dtype arithmetic;
 *   smooth = 0: each field is used as the test vector psi itself (Eq. 3 split onward).
 * The fields are rounded to setup_dtype first (an MG_C64 field is exact in either), and
 * the SVD then runs exactly as in mg_setup_streaming_svd (same arithmetic, same kernels):
 * this is how the streaming SVD of a given set of test vectors is checked against a
 * reference, and how an application supplies its own near-null vectors.
 * MG_EINVAL: as mg_setup_streaming_svd, plus NULL vectors, vec_dtype other than MG_C128 /
 * MG_C64, smooth other than 0 / 1.  Creates *h (NULL on entry); synchronises `stream`.
 * ------------------------------------------------------------------------------- */
int mg_setup_from_vectors(mg_handle** h, const void* links, const mg_params* p,
                          const void* vectors, int vec_dtype, int smooth, void* stream);

/* ---------------------------------------------------------------------------------
 * mg_setup_ls -- the setup with the least-squares interpolation prolongator of Eq. 9
 * (Sec. 5): per aggregate and chirality, with the tile V_f of the r test vectors (Eq. 2,
 * Philox, as in mg_setup_streaming_svd), its SVD V_f = U Sigma V^dag and V_c = Sigma_k V_k^dag,
 *   P_j = V_f Omega V_c^dag (V_c Omega V_c^dag)^{-1},   Omega = diag(omega),
 * each column with the canonical phase.  omega = 1 gives U_k (the iCSVD prolongator); other
 * weights (the paper names energy norms of the test vectors) give a prolongator whose columns
 * are not orthonormal (the Galerkin product and R = P^dag handle that).
 *   omega: r positive doubles, host or device, one per test vector, the same for every
 *   aggregate.  Requires n_s = 1 and r >= k; one Gram pass (svd_refine is ignored).
 * MG_EINVAL: as mg_setup_streaming_svd, plus n_s != 1, r < k, a weight <= 0.
 * ------------------------------------------------------------------------------- */
int mg_setup_ls(mg_handle** h, const void* links, const mg_params* p, const double* omega,
                void* stream);

/* Creates a handle with links and parameters but no prolongator (for mg_set_prolongator). */
int mg_create(mg_handle** h, const void* links, const mg_params* p, void* stream);

/* ---------------------------------------------------------------------------------
 * coarse_build -- Galerkin coarse operator D_c = P^dag D P (Eq. 5; Algorithm 4) as a
 * nearest-neighbour coarse stencil: X(j) and Y_dir(j), dir = 2 mu + (0: +mu, 1: -mu),
 * each (2k) x (2k), assembled in FP64 and also kept in FP32.
 * ------------------------------------------------------------------------------- */
int coarse_build(mg_handle* h, void* stream);

/* ---------------------------------------------------------------------------------
 * coarse_build_noalloc -- coarse_build without any device memory allocation.  The
 * paper has no counterpart: this is a library service for callers that cannot let the
 * library allocate device memory while they run -- e.g. an application that has handed
 * nearly all of HBM to its own pool allocator (a library cudaMalloc would then fail or
 * fragment that pool), or one that must keep a fixed device-memory footprint after
 * start-up.  It performs the same coarse-operator rebuild as coarse_build, into the
 * handle's existing coarse-operator storage, e.g. after mg_set_prolongator.
 *   Scratch: the Galerkin forward-hop partials, 4 * d * (2k)^2 complex doubles
 *     (d = coarse sites), live in one fixed 24 MiB device array inside the library, so
 *     d * k^2 must not exceed 98304 (the 16^3x32 lattice with 4^4 aggregates fits up to
 *     k = 13); larger hierarchies return MG_EINVAL -- use coarse_build for those.
 *     Nothing in the scratch has to start at zero: every partial is written before it
 *     is read, so consecutive calls need no reset.
 *   Preconditions: the handle has a prolongator and coarse_build has run on it once
 *     (that call allocates the storage of D_c, which this call overwrites); otherwise
 *     MG_EINVAL.
 *   Set-up: the first call on each device looks up the device address of the scratch
 *     array (once, with that device current) and caches it.  Like every other device
 *     state of the library (handles, its allocation cache), the cached address belongs to
 *     the device's primary context: a cudaDeviceReset of that device while the library
 *     is loaded invalidates it.
 *   Concurrency: the scratch is shared by every handle of the process on a device, so
 *     calls on the same device must not overlap (e.g. from two host threads): two
 *     overlapping calls race on the scratch and both results are undefined.
 *   Result: the same kernels in the same order as coarse_build, so the same D_c.
 *   Synchronises `stream` before returning.
 * ------------------------------------------------------------------------------- */
int coarse_build_noalloc(mg_handle* h, void* stream);

/* ---------------------------------------------------------------------------------
 * mg_add_level -- one more level of the hierarchy (Sec. 2.1 end; Sec. 4 uses three and, near
 * the critical mass, four levels): the coarsest operator so far, D_l (l = 1 after
 * coarse_build), takes the place of D in Algorithm 3 and Eq. 5 --
 *   test vectors psi = phi + GMRES_sweeps(D_l, -D_l phi) (Eq. 2), phi complex-Gaussian
 *     Philox fields with counter (site, component, vector id, l), vector ids s r .. s r + r - 1;
 *   chiral split with sigma_3 as the chirality (gamma_5 P = P sigma_3): each level-l site
 *     vector [alpha][k_l] gives k_l rows of chirality alpha, rows (local site, i) inside the
 *     aggregates of extent `block` on the level-l lattice;
 *   streaming SVD over n_s streams of r vectors, k kept (FP64);
 *   D_{l+1} = P_l^dag D_l P_l as a nearest-neighbour stencil on the lattice of aggregates.
 * The K-cycle then recurses: the level-l system of the cycle is solved to its tolerance by
 * FGMRES preconditioned by the K-cycle of level l (GMRES on the coarsest level, restart
 * coarse_restart), with post_smooth GMRES steps on D_l; `tol` is the relative tolerance of the
 * new coarsest level's solve (the paper: 0.03; near the critical mass 0.06 and 0.6 on its
 * third and fourth level).  Requires coarse_build; coarse_build and mg_set_prolongator drop the
 * added levels.  sweeps, seed and svd_refine come from the handle's parameters.
 * MG_EINVAL: block not dividing the level-l lattice, k > min(32, n_d k_l), k + r > 64,
 * n_s r < k, tol outside (0, 1), more than 8 levels.  Synchronises `stream`.
 * ------------------------------------------------------------------------------- */
int mg_add_level(mg_handle* h, const int block[4], int k, int r, int n_s, double tol,
                 void* stream);

/* Number of levels: 1 before coarse_build, 2 after it, + 1 per mg_add_level. */
int mg_num_levels(const mg_handle* h);

/* Iterations of the last solve on levels 1 .. L-1 (its[l - 1], summed over K-cycles and
 * right-hand sides), at most nmax of them. */
int mg_level_iterations(const mg_handle* h, long long* its, int nmax);

/* Level l >= 2 added by mg_add_level: P_{l-1} tiles P[J][alpha][i][row] (row = local site *
 * k_{l-1} + component, complex double), their singular values sigma[J][alpha][i] (double), and
 * the level-l operator X[j][a][b], Y[dir][j][a][b] (complex double, row a, column b).  Any of P,
 * sigma may be NULL; X and Y are both given or both NULL. */
int mg_get_level(mg_handle* h, int level, void* P, void* sigma, void* X, void* Y, void* stream);

/* ---------------------------------------------------------------------------------
 * mg_solve -- x = D^{-1} b to ||b - D x|| <= tol ||b|| (checked in FP64) with FGMRES
 * preconditioned by the two-level K-cycle (restrict, coarse GMRES to coarse_tol,
 * prolong, post_smooth GMRES steps).  solve_dtype MG_C128: one FP64 FGMRES;
 * otherwise FP64 iterative refinement around an inner solve in solve_dtype.
 * x, b: complex double fields, nrhs of them.  x is overwritten (initial guess 0).
 * Synchronises `stream`.  MG_ENOCONV after maxiter outer iterations per RHS.
 * ------------------------------------------------------------------------------- */
int mg_solve(mg_handle* h, void* x, const void* b, int nrhs, double tol, int maxiter,
             mg_solve_info* info, void* stream);

/* x = D^{-dag} b = gamma_5 D^{-1} gamma_5 b on the same hierarchy (adjoint solve). */
int mg_solve_adjoint(mg_handle* h, void* x, const void* b, int nrhs, double tol,
                     int maxiter, mg_solve_info* info, void* stream);

int mg_destroy(mg_handle* h);

/* ---------------------------------------------------------------------------------
 * Step-level entry points (each step of the path callable on its own).
 * ------------------------------------------------------------------------------- */

/* The r test vectors of stream `stream_index` (Eq. 2) in setup_dtype arithmetic,
 * written as complex double fields out[r][site][4][3].  links: complex double. */
int mg_test_vectors(void* out, const void* links, const mg_params* p, int stream_index,
                    void* stream);

/* out = D in (dagger: D^dag in) with the handle's operator and its lane-contiguous link
 * copy (the stencil the solver runs); dtype MG_C128 or MG_C64 fields, nrhs of them, or
 * MG_F16 / MG_BF16 fields (half links) on a handle whose solve_dtype is that type. */
int mg_apply_fine(mg_handle* h, void* out, const void* in, int nrhs, int dtype, int dagger,
                  void* stream);

/* Rows per link kept by the handle's FP32 / half stencil copies (2 or 3; link_compress);
 * 0 for a NULL handle. */
int mg_link_rows(const mg_handle* h);

/* P tiles: P[j][alpha][i][row], row = (local site * 2 + spin in chirality) * 3 + colour,
 * local site lexicographic inside the aggregate; complex double.  sigma[j][alpha][k]
 * (double, may be NULL): singular values of the last stream. */
int mg_get_prolongator(mg_handle* h, void* P, void* sigma, void* stream);

/* Singular values of every stream: hist[s][j][alpha][k] (double; entries beyond the
 * stream's kept count are 0). */
int mg_get_sigma_history(mg_handle* h, void* hist, void* stream);

/* Replace P (same layout as mg_get_prolongator, complex double). */
int mg_set_prolongator(mg_handle* h, const void* P, void* stream);

/* e_c = P^dag v (R = P^dag, Sec. 2.1) and v = P e_c; complex double fields. */
int mg_restrict(mg_handle* h, void* vc, const void* v, int nrhs, void* stream);
int mg_prolong(mg_handle* h, void* v, const void* vc, int nrhs, void* stream);

/* Coarse operator export: X[j][a][b], Y[dir][j][a][b] complex double (row a, col b). */
int mg_get_coarse_op(mg_handle* h, void* X, void* Y, void* stream);

/* y = D_c x on the coarse lattice; dtype MG_C128 or MG_C64 (FP64 / FP32 stencil). */
int mg_coarse_apply(mg_handle* h, void* y, const void* x, int nrhs, int dtype, void* stream);

/* ---------------------------------------------------------------------------------
 * wilson_link_gradient -- link-angle gradient of a loss through x = D^{-1} b:
 * with g_b = D^{-dag} g_x (g_x = 2 dL/d conj x),
 *   out[mu][y][a] = -Re[ g_b(y)^dag dD/d omega^a_mu(y) x ]
 * for U_mu(y) -> exp(i sum_a omega^a T^a) U_mu(y), T^a = lambda^a / 2 (Gell-Mann).
 * g_b, x, links: complex double; out: double [4][V][8].
 * ------------------------------------------------------------------------------- */
int wilson_link_gradient(void* out, const void* g_b, const void* x, const void* links,
                         const int dims[4], double kappa, const double hop_weight[4],
                         const int bc_phase[4], void* stream);

#ifdef __cplusplus
}
#endif
#endif /* WILSON_MG_H */
