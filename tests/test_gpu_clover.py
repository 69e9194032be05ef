"""Wilson-clover operator on the GPU (Configuration B of Sec. 4) vs the FP64 oracle: the clover
field, the operator in FP64 / FP32, the Galerkin diagonal with the clover term, and the
clover solve."""
import numpy as np
import pytest
import torch

from oracle import clover, coarse, icsvd, mg, wilson
from paper_2505_14399_gb300 import api, synthetic
from gpu_common import links_for, orthonormal_tiles, params_for, rel, to_dev

pytestmark = pytest.mark.gpu

DIMS = (6, 4, 6, 10)      # 1440 sites: a ragged last CTA
CSW = 1.7
ANISO = (1.0, 1.0, 1.0, 1 / 3.5)
C5 = synthetic.WORKLOADS["c5_8^4_autograd"]


def _chiral_blocks(C):
    """oracle C (V, 12, 12) -> (V, 2, 6, 6) chirality blocks, and the largest off-block entry"""
    V = C.shape[0]
    B = np.zeros((V, 2, 6, 6), dtype=np.complex128)
    for a in range(2):
        B[:, a] = C[:, 6 * a:6 * a + 6, 6 * a:6 * a + 6]
    off = max(np.abs(C[:, :6, 6:]).max(), np.abs(C[:, 6:, :6]).max())
    return B, off


@pytest.mark.parametrize("links", ["haar", "smooth"])
def test_clover_field(links):
    U = synthetic.haar_links(DIMS, 90) if links == "haar" else synthetic.smooth_links(DIMS, 91)
    Cg = api.clover_field(to_dev(U), DIMS, 0.13, CSW).cpu().numpy()
    Co, off = _chiral_blocks(clover.clover_term(U, DIMS, 0.13, CSW))
    assert off == 0.0
    assert rel(Cg, Co) < 1e-13


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 1e-5)])
@pytest.mark.parametrize("dagger", [False, True])
def test_clover_operator(dtype, tol, dagger):
    U = synthetic.haar_links(DIMS, 92)
    psi = synthetic.gaussian_rhs(DIMS, 93, 2)
    C = clover.clover_term(U, DIMS, 0.13, CSW)
    Cb, _ = _chiral_blocks(C)
    out = api.clover_dslash(to_dev(psi, dtype), to_dev(U, dtype), to_dev(Cb, dtype), DIMS, 0.13,
                            ANISO, (1, 1, 1, -1), dagger).cpu().numpy()
    for r in range(2):
        ref = clover.dslash(psi[r], U, DIMS, 0.13, CSW, ANISO, (1, 1, 1, -1), dagger, C=C)
        assert rel(out[r], ref) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 1e-5)])
def test_handle_operator_with_clover(dtype, tol):
    """The solver's operator (mg_apply_fine) on a handle with c_sw: D_W + C."""
    U = synthetic.smooth_links(DIMS, 94)
    psi = synthetic.gaussian_rhs(DIMS, 95, 2)
    p = api.params(DIMS, (2, 2, 2, 2), 0.13, 4, 4, 1, hop_weight=ANISO, bc=(1, 1, 1, -1), csw=CSW)
    h = api.Hierarchy(to_dev(U), p, setup=False)
    out = h.apply_fine(to_dev(psi, dtype)).cpu().numpy()
    C = clover.clover_term(U, DIMS, 0.13, CSW)
    for r in range(2):
        ref = clover.dslash(psi[r], U, DIMS, 0.13, CSW, ANISO, (1, 1, 1, -1), C=C)
        assert rel(out[r], ref) < tol
    h.close()


@pytest.mark.parametrize("solve_dtype", ["c128", "c64"])   # FP64 and double-float Galerkin
def test_galerkin_with_clover(solve_dtype):
    """D_c = P^dag (D_W + C) P (Eq. 5 with the clover diagonal) against the oracle."""
    dims, block, k = (4, 4, 4, 4), (2, 2, 2, 2), 5
    U = synthetic.smooth_links(dims, 96)
    p = api.params(dims, block, 0.125, k, k, 1, hop_weight=ANISO, bc=(1, 1, 1, -1),
                   setup_dtype="c128", solve_dtype=solve_dtype, csw=CSW)
    h = api.Hierarchy(to_dev(U), p, setup=False)
    nd = int(np.prod(block))
    d = int(np.prod(dims)) // nd
    P = orthonormal_tiles(d, nd, k, 97)
    h.set_prolongator(to_dev(P))
    h.coarse_build()
    X, Y = h.coarse_op()
    Pt = np.ascontiguousarray(np.swapaxes(P, 2, 3))
    C = clover.clover_term(U, dims, 0.125, CSW)
    Xo, Yo = coarse.galerkin(Pt, U, dims, block, 0.125, ANISO, (1, 1, 1, -1), clover=C)
    assert rel(X.cpu().numpy(), Xo) < 1e-11
    assert rel(Y.cpu().numpy(), Yo) < 1e-11
    h.close()


def _clover_cfg():
    cfg = dict(C5)
    cfg["kappa"] = 0.115
    return cfg


def test_fp64_clover_solve_matches_oracle():
    """FP64 K-cycle FGMRES for D_W + C: solution and outer iteration count of the oracle's
    two-level solve of the clover system (within one)."""
    cfg = _clover_cfg()
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])
    p = params_for(cfg, setup_dtype="c128", solve_dtype="c128", csw=CSW)
    h = api.Hierarchy(to_dev(U), p)
    h.coarse_build()
    x, info = h.solve(to_dev(b), tol=1e-10)
    x = x.cpu().numpy()[0]
    C = clover.clover_term(U, cfg["dims"], cfg["kappa"], CSW)
    Pt, _, _ = icsvd.icsvd(U, cfg["dims"], cfg["kappa"], cfg["hop_weight"], cfg["bc"],
                           cfg["block"], cfg["k"], cfg["r"], cfg["n_s"], cfg["sweeps"],
                           cfg["tv_seed"], clover=C)
    lvl = mg.TwoLevel(U, cfg["dims"], cfg["kappa"], cfg["hop_weight"], cfg["bc"], cfg["block"],
                      Pt, clover=C)
    xo, info_o = lvl.solve(b[0].reshape(-1), tol=1e-10)
    r = b[0].reshape(-1) - clover.dslash(x, U, cfg["dims"], cfg["kappa"], CSW, cfg["hop_weight"],
                                         cfg["bc"], C=C).reshape(-1)
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= 1e-10
    assert rel(x.reshape(-1), xo) < 1e-8
    assert abs(info["outer"] - info_o["outer"]) <= 1
    h.close()


def test_mixed_clover_solve():
    """Mixed form with the clover term: true residual 1e-10 (oracle D_clover) on two RHS."""
    cfg = _clover_cfg()
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"], 2)
    h = api.Hierarchy(to_dev(U), params_for(cfg, csw=CSW))
    h.coarse_build()
    x, _ = h.solve(to_dev(b), tol=1e-10)
    x = x.cpu().numpy()
    C = clover.clover_term(U, cfg["dims"], cfg["kappa"], CSW)
    for k in range(2):
        r = b[k].reshape(-1) - clover.dslash(x[k], U, cfg["dims"], cfg["kappa"], CSW,
                                             cfg["hop_weight"], cfg["bc"], C=C).reshape(-1)
        assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1e-10
    h.close()
