"""Streaming chiral SVD (Algorithm 3) on the GPU against the oracle, at the bounds that
first-order perturbation theory gives for the library's Gram route (tests/svd_bounds.py):

* the configuration the benchmark times, at full size: 16^3 x 32 lattice, 4^4 aggregates
  (1536-row tiles, up to 20 columns), k = 12, four streams of 8 complex-float test vectors,
  double-float Gram / Jacobi / update, tensor-pipe Galerkin -- the test vectors supplied through
  mg_setup_from_vectors, so both sides start from the same fields;
* end to end on the small workloads, Philox test vectors smoothed on each side (FP64 or FP32
  smoother), FP64 and double-float SVD arithmetic.
"""
import numpy as np
import pytest

from oracle import coarse, icsvd, wilson
from paper_2505_14399_gb300 import api, synthetic
import svd_bounds
from gpu_common import links_for, params_for, record, rel, to_dev

pytestmark = pytest.mark.gpu

C1 = synthetic.WORKLOADS["c1_4^4_haar"]
C2 = synthetic.WORKLOADS["c2_16^3x32_near_critical"]
C5 = synthetic.WORKLOADS["c5_8^4_autograd"]


def _check(name, P, H, stream_tiles, k, u, delta=0.0, sub=None):
    """sigma of every stream, projectors, orthonormality and the canonical phase of P (library
    layout (d, 2, k, rows)) against the oracle on `stream_tiles` (aggregates `sub` of P)."""
    if sub is not None:
        P = P[sub]
        H = H[:, sub]
    Pt, S_o, hist_o = icsvd.icsvd_tiles(stream_tiles, k)
    spectra = svd_bounds.stream_spectra(stream_tiles, k)
    b = svd_bounds.vector_bounds(spectra, delta, u, stream_tiles[0].shape[2])
    worst = 0.0
    for s, hs in enumerate(hist_o):
        kk = hs.shape[-1]
        es = np.abs(H[s][..., :kk] - hs).max(axis=-1)
        assert np.all(es <= b[s][1]), (s, (es / b[s][1]).max())
        worst = max(worst, (es / b[s][1]).max())
        record(name, stream=s, sigma_err_rel=(es / hs[..., 0]).max(), sigma_ratio=(es / b[s][1]).max())
    ep = svd_bounds.projector_errors(P, Pt)
    assert np.all(ep <= b[-1][0]), (ep / b[-1][0]).max()
    eye = np.eye(k)
    orth = max(np.abs(P[j, a].conj() @ P[j, a].T - eye).max()
               for j in range(P.shape[0]) for a in range(2))
    assert orth <= max(b[-1][0].max(), 1e-13), orth
    q = P.sum(axis=-1)
    assert np.all(np.abs(q.imag) <= 1e-10 * np.abs(q)) and np.all(q.real > 0)
    record(name, proj_err=ep.max(), proj_ratio=(ep / b[-1][0]).max(), orth_err=orth,
           proj_bound_min=b[-1][0].min())
    return Pt


def test_timed_configuration_full_size():
    """The benchmark's setup at full size on 32 supplied complex-float test vectors: sigma of
    every stream and the projectors of 64 of the 512 aggregates (both chiralities) within the
    double-float bound; then the tensor-pipe Galerkin operator, compared basis-free as
    P D_c P^dag x against the oracle's P P^dag D P P^dag x on the whole lattice."""
    cfg = dict(C2)
    cfg["kappa"] = synthetic.kappa_of(C2)
    dims, block, k, r, n_s = cfg["dims"], cfg["block"], cfg["k"], cfg["r"], cfg["n_s"]
    U = links_for(cfg)
    vec = synthetic.graded_fields(dims, r * n_s, 2.0, 4001).astype(np.complex64)
    p = params_for(cfg, setup_dtype="c64", solve_dtype="c64")
    h = api.Hierarchy(to_dev(U), p, vectors=to_dev(vec))
    P, _ = h.prolongator()
    P = P.cpu().numpy()
    H = h.sigma_history().cpu().numpy()
    v64 = vec.astype(np.complex128)
    tiles = [icsvd.chiral_split(v64[s * r:(s + 1) * r], dims, block) for s in range(n_s)]
    d = tiles[0].shape[0]
    sub = np.arange(0, d, 8)
    _check("timed_full_size", P, H, [t[sub] for t in tiles], k, svd_bounds.UDF, sub=sub)
    # Galerkin operator of the GPU's P against the definition on the oracle's P
    Pt_all, _, _ = icsvd.icsvd_tiles(tiles, k)
    spectra = svd_bounds.stream_spectra([t[sub] for t in tiles], k)
    bp = svd_bounds.arithmetic_bounds(spectra, svd_bounds.UDF, tiles[0].shape[2])[-1][0].max()
    h.coarse_build()
    rng = np.random.default_rng(17)
    V = wilson.volume(dims)
    x = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
    yg = h.prolong(h.coarse_apply(h.restrict(to_dev(x[None])))).cpu().numpy()[0]
    w, bc = cfg["hop_weight"], cfg["bc"]
    xc = coarse.restrict(Pt_all, x, dims, block)
    Dx = wilson.dslash(coarse.prolong(Pt_all, xc, dims, block), U, dims, cfg["kappa"], w, bc)
    yo = coarse.prolong(Pt_all, coarse.restrict(Pt_all, Dx, dims, block), dims, block)
    e = rel(yg, yo)
    # the subspaces of all 512 aggregates lie within 8x the worst bound of the sampled ones
    bound = 2.0 * (1 + 8 * cfg["kappa"]) * 8 * bp + 1e-11
    record("timed_full_size_galerkin", rel_err=e, bound=bound)
    assert e <= bound, (e, bound)
    h.close()


def _end_to_end(name, cfg, setup_dtype, u, delta, **kw):
    U = links_for(cfg)
    p = params_for(cfg, setup_dtype=setup_dtype, **kw)
    h = api.Hierarchy(to_dev(U), p)
    P, _ = h.prolongator()
    H = h.sigma_history().cpu().numpy()
    tiles = []
    for s in range(cfg["n_s"]):
        tv = icsvd.test_vectors(U, cfg["dims"], cfg["kappa"], cfg["hop_weight"], cfg["bc"],
                                cfg["tv_seed"], cfg["r"], s, cfg["sweeps"])
        tiles.append(icsvd.chiral_split(tv, cfg["dims"], cfg["block"]))
    _check(name, P.cpu().numpy(), H, tiles, cfg["k"], u, delta)
    h.close()


@pytest.mark.parametrize("cfg", [C1, C5], ids=["c1", "c5"])
@pytest.mark.parametrize("refine", [0, 1])
def test_fp64_setup_end_to_end(cfg, refine):
    """FP64 smoother and FP64 Gram / Jacobi / update: the FP64 bound (u = 2^-53)."""
    _end_to_end("fp64_%s_refine%d" % (cfg["link_seed"], refine), cfg, "c128", svd_bounds.U64,
                0.0, svd_refine=refine, fp64_emulation=0)


@pytest.mark.parametrize("cfg", [C1, C5], ids=["c1", "c5"])
@pytest.mark.parametrize("refine", [0, 1])
def test_double_float_setup_end_to_end(cfg, refine):
    """FP64 smoother, double-float Gram / Jacobi / update: the double-float bound (2^-48)."""
    _end_to_end("df_%s_refine%d" % (cfg["link_seed"], refine), cfg, "c128", svd_bounds.UDF,
                0.0, svd_refine=refine, fp64_emulation=1)


@pytest.mark.parametrize("cfg", [C1, C5], ids=["c1", "c5"])
def test_mixed_setup_end_to_end(cfg):
    """The mixed form as timed: FP32 smoother (test vectors within 1e-5 of the FP64 ones, the
    bound of the smoother's own parity test) and double-float SVD: the test-vector bound."""
    _end_to_end("mixed_%s" % cfg["link_seed"], cfg, "c64", svd_bounds.UDF, 1e-5)


def test_supplied_initial_guesses_are_smoothed():
    """smooth = 1: supplied fields are the phi of Eq. 2 (here the Philox fields the oracle
    draws), so the setup equals the plain setup."""
    from oracle import philox
    cfg = C5
    U = links_for(cfg)
    V = wilson.volume(cfg["dims"])
    m = cfg["r"] * cfg["n_s"]
    phi = philox.gaussian_vectors(cfg["tv_seed"], np.arange(m), V).reshape(m, V, 4, 3)
    p = params_for(cfg, setup_dtype="c128")
    h = api.Hierarchy(to_dev(U), p, vectors=to_dev(phi), smooth=True)
    P, _ = h.prolongator()
    H = h.sigma_history().cpu().numpy()
    tiles = []
    for s in range(cfg["n_s"]):
        tv = icsvd.test_vectors(U, cfg["dims"], cfg["kappa"], cfg["hop_weight"], cfg["bc"],
                                cfg["tv_seed"], cfg["r"], s, cfg["sweeps"])
        tiles.append(icsvd.chiral_split(tv, cfg["dims"], cfg["block"]))
    _check("supplied_phi_c5", P.cpu().numpy(), H, tiles, cfg["k"], svd_bounds.U64)
    h.close()


@pytest.mark.parametrize("cfg", [C1, C5], ids=["c1", "c5"])
@pytest.mark.parametrize("weights", ["ones", "graded"])
def test_least_squares_interpolation_prolongator(cfg, weights):
    """Eq. 9 on the GPU (FP64 setup, one stream of r test vectors) against the oracle's
    P_j = V_f Omega V_c^dag (V_c Omega V_c^dag)^{-1} on the same vectors.  The GPU computes V_k
    from the Gram matrix: its error is the subspace bound of a single stream times the
    condition number of V_k^dag Omega V_k; with Omega = 1 the result is U_k."""
    U = links_for(cfg)
    r = cfg["r"] * cfg["n_s"]
    k = cfg["k"]
    omega = np.ones(r) if weights == "ones" else 10.0 ** (-np.arange(r) / (r - 1))
    p = params_for(cfg, setup_dtype="c128", n_s=1, r=r, fp64_emulation=0, svd_refine=0)
    h = api.Hierarchy(to_dev(U), p, ls_omega=omega)
    P, _ = h.prolongator()
    P = P.cpu().numpy()
    tv = icsvd.test_vectors(U, cfg["dims"], cfg["kappa"], cfg["hop_weight"], cfg["bc"],
                            cfg["tv_seed"], r, 0, cfg["sweeps"])
    tiles = icsvd.chiral_split(tv, cfg["dims"], cfg["block"])
    Po, _ = icsvd.ls_prolongator_tiles(tiles, k, omega)
    spectra = svd_bounds.stream_spectra([tiles], k)
    bp = svd_bounds.arithmetic_bounds(spectra, svd_bounds.U64, tiles.shape[2])[-1][0]
    worst = 0.0
    for j in range(P.shape[0]):
        for a in range(2):
            _, s, Vh = np.linalg.svd(tiles[j, a], full_matrices=False)
            Vk = Vh[:k].conj().T
            cond = np.linalg.cond(Vk.conj().T @ np.diag(omega) @ Vk)
            e = np.abs(P[j, a].T - Po[j, a]).max() / np.abs(Po[j, a]).max()
            assert e <= 4 * cond * bp[j, a], (j, a, e, cond * bp[j, a])
            worst = max(worst, e)
    if weights == "ones":
        Pu, _, _ = icsvd.icsvd_tiles([tiles], k)
        assert np.all(svd_bounds.projector_errors(P, Pu) <= bp)
    record("ls_%s_%s" % (cfg["link_seed"], weights), rel_err=worst)
    h.close()


def test_anisotropic_configuration_full_size():
    """The anisotropic 16^3 x 64 workload at full size (2x2x2x4 aggregates: 8192 of them, tiles
    of 192 rows and up to 40 columns, k = 24, four streams of 16), on 64 supplied complex-float
    vectors with the mixed form's double-float SVD: sigma of every stream and the projectors of
    64 aggregates against the oracle within the double-float bound."""
    cfg = dict(synthetic.WORKLOADS["c3_16^3x64_aniso"])
    cfg["kappa"] = synthetic.kappa_of(cfg)
    dims, block, k, r, n_s = cfg["dims"], cfg["block"], cfg["k"], cfg["r"], cfg["n_s"]
    U = links_for(cfg)
    vec = synthetic.graded_fields(dims, r * n_s, 2.0, 4002).astype(np.complex64)
    p = params_for(cfg, setup_dtype="c64", solve_dtype="c64")
    h = api.Hierarchy(to_dev(U), p, vectors=to_dev(vec))
    P, _ = h.prolongator()
    P = P.cpu().numpy()
    H = h.sigma_history().cpu().numpy()
    h.close()
    d = P.shape[0]
    sub = np.arange(0, d, d // 64)
    tiles = [icsvd.chiral_split(vec[s * r:(s + 1) * r].astype(np.complex128), dims, block)[sub]
             for s in range(n_s)]
    del vec
    _check("aniso_full_size", P, H, tiles, k, svd_bounds.UDF, sub=sub)
