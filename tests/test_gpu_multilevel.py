"""Deeper hierarchies on the GPU (Sec. 2.1 end, Algorithm 4, Sec. 4) against the FP64 oracle:
the setup and Galerkin product on a coarse operator, and three- and four-level K-cycle solves."""
import numpy as np
import pytest

from oracle import icsvd, multilevel, wilson
from paper_2505_14399_gb300 import _lib as L, api, synthetic
import svd_bounds
from gpu_common import links_for, params_for, record, rel, to_dev

pytestmark = pytest.mark.gpu

C5 = synthetic.WORKLOADS["c5_8^4_autograd"]
B2 = (2, 2, 2, 2)


def _two_level(cfg, **kw):
    U = links_for(cfg)
    p = params_for(cfg, setup_dtype="c128", solve_dtype="c128", **kw)
    h = api.Hierarchy(to_dev(U), p)
    h.coarse_build()
    return h, U


def _level1(h, cfg):
    X, Y = h.coarse_op()
    cd = [cfg["dims"][m] // cfg["block"][m] for m in range(4)]
    return X.cpu().numpy(), Y.cpu().numpy(), cd


def test_level2_setup_on_the_gpu_level1_operator():
    """Level-2 test vectors, chiral split and streaming SVD on the GPU's own level-1 operator
    (exported), against the oracle's run of the same steps on that operator: sigma and
    projectors within the FP64 bound."""
    cfg = C5
    h, U = _two_level(cfg)
    X1, Y1, cd1 = _level1(h, cfg)
    k2, r2, ns2 = 6, 6, 2
    h.add_level(B2, k2, r2, ns2)
    assert h.num_levels() == 3
    P2, S2, _, _ = h.level(2)
    tiles = [multilevel.chiral_split(multilevel.test_vectors(X1, Y1, cd1, cfg["tv_seed"], r2, s,
                                                             cfg["sweeps"], 1), cd1, B2)
             for s in range(ns2)]
    Pt, S_o, _ = icsvd.icsvd_tiles(tiles, k2)
    spectra = svd_bounds.stream_spectra(tiles, k2)
    bp, bs = svd_bounds.arithmetic_bounds(spectra, svd_bounds.U64, tiles[0].shape[2])[-1]
    S2 = S2.cpu().numpy()
    es = np.abs(S2 - S_o).max(axis=-1)
    assert np.all(es <= bs), (es / bs).max()
    ep = svd_bounds.projector_errors(P2.cpu().numpy(), Pt)
    assert np.all(ep <= bp), (ep / bp).max()
    record("level2_setup", sigma_err_rel=(es / S_o[..., 0]).max(), proj_err=ep.max())
    h.close()


def test_level2_galerkin_matches_oracle_on_the_same_inputs():
    """D_2 = P_2^dag D_1 P_2 (Eq. 5 on a coarse stencil) from the GPU's P_2 and D_1, against
    the oracle's term-by-term product of the same arrays: FP64 to 1e-13."""
    cfg = C5
    h, U = _two_level(cfg)
    X1, Y1, cd1 = _level1(h, cfg)
    h.add_level(B2, 6, 6, 2)
    P2, _, X2, Y2 = h.level(2)
    P2 = np.ascontiguousarray(np.swapaxes(P2.cpu().numpy(), 2, 3))   # (d2, 2, rows, k)
    Ps = multilevel.site_prolongator(P2, cd1, B2, X1.shape[1])
    Xo, Yo = multilevel.galerkin(Ps, X1, Y1, cd1, B2)
    assert rel(X2.cpu().numpy(), Xo) < 1e-13
    assert rel(Y2.cpu().numpy(), Yo) < 1e-13
    h.close()


def _oracle_hierarchy(cfg, U, blocks, ks, rs, nss):
    return multilevel.Hierarchy(U, cfg["dims"], cfg["kappa"], cfg["hop_weight"], cfg["bc"],
                                blocks, ks, rs, nss, cfg["sweeps"], cfg["tv_seed"])


@pytest.mark.parametrize("depth", [3, 4])
def test_fp64_multilevel_solve_matches_oracle(depth):
    """FP64 K-cycle FGMRES on three / four levels: the solution and the outer iteration count of
    the oracle's hierarchy built from the same seeds (within one), true residual 1e-10."""
    cfg = C5
    h, U = _two_level(cfg)
    blocks, ks, rs, nss = [cfg["block"], B2], [cfg["k"], 6], [cfg["r"], 6], [cfg["n_s"], 2]
    h.add_level(B2, 6, 6, 2)
    if depth == 4:
        h.add_level(B2, 4, 4, 2)          # level-3 lattice of a single site
        blocks.append(B2), ks.append(4), rs.append(4), nss.append(2)
    assert h.num_levels() == depth
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])
    x, info = h.solve(to_dev(b), tol=1e-10)
    x = x.cpu().numpy()[0]
    its = h.level_iterations()
    assert len(its) == depth - 1 and all(v > 0 for v in its)
    H = _oracle_hierarchy(cfg, U, blocks, ks, rs, nss)
    xo, info_o = H.solve(b[0].reshape(-1), tol=1e-10)
    r = b[0].reshape(-1) - wilson.dslash(x, U, cfg["dims"], cfg["kappa"], cfg["hop_weight"],
                                         cfg["bc"]).reshape(-1)
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= 1e-10
    assert rel(x.reshape(-1), xo) < 1e-8
    assert abs(info["outer"] - info_o["outer"]) <= 1, (info, info_o)
    record("multilevel_fp64_%d" % depth, outer=info["outer"], outer_oracle=info_o["outer"])
    h.close()


def test_mixed_three_level_solve_two_rhs():
    """Mixed form (FP32 K-cycle on every level, FP64 refinement) on three levels: true residual
    1e-10 for two right-hand sides."""
    cfg = C5
    U = links_for(cfg)
    h = api.Hierarchy(to_dev(U), params_for(cfg))
    h.coarse_build()
    h.add_level(B2, 6, 6, 2)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"], 2)
    x, info = h.solve(to_dev(b), tol=1e-10)
    x = x.cpu().numpy()
    for k in range(2):
        r = b[k].reshape(-1) - wilson.dslash(x[k], U, cfg["dims"], cfg["kappa"],
                                             cfg["hop_weight"], cfg["bc"]).reshape(-1)
        assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1e-10
    h.close()


def test_rebuilding_level1_drops_deeper_levels():
    cfg = C5
    h, U = _two_level(cfg)
    h.add_level(B2, 6, 6, 2)
    assert h.num_levels() == 3
    assert L.lib().coarse_build_noalloc(h._h, None) == L.MG_EINVAL
    h.coarse_build()
    assert h.num_levels() == 2
    with pytest.raises(L.MgError):
        h.add_level((3, 2, 2, 2), 6, 6, 2)   # 3 does not divide the level-1 extent 4
    h.close()
