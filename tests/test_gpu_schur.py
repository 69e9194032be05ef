"""Even-odd Schur form on the GPU (even-odd preconditioning, Sec. 1) vs the FP64 oracle: the
D_hat operator in every storage type, and the K-cycle solve with the Schur-form post-smoother."""
import numpy as np
import pytest
import torch

from oracle import icsvd, mg, schur, wilson
from paper_2505_14399_gb300 import api, synthetic
from gpu_common import from_half_pair, half_pair, links_for, params_for, rel, to_dev

pytestmark = pytest.mark.gpu

DIMS = (6, 4, 6, 10)    # 720 even sites: a ragged last CTA
ANISO = (1.0, 1.0, 1.0, 1 / 3.5)
C1 = synthetic.WORKLOADS["c1_4^4_haar"]
C5 = synthetic.WORKLOADS["c5_8^4_autograd"]


def _even_fields(nrhs, seed):
    rng = np.random.default_rng(seed)
    Vh = int(np.prod(DIMS)) // 2
    return rng.standard_normal((nrhs, Vh, 4, 3)) + 1j * rng.standard_normal((nrhs, Vh, 4, 3))


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 1e-5)])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("w,bc", [((1, 1, 1, 1), (1, 1, 1, 1)), (ANISO, (1, 1, 1, -1))])
def test_schur_operator(dtype, tol, dagger, w, bc):
    U = synthetic.haar_links(DIMS, 80)
    v = _even_fields(2, 81)
    out = api.schur(to_dev(v, dtype), to_dev(U, dtype), DIMS, 0.131, w, bc, dagger).cpu().numpy()
    for r in range(2):
        ref = schur.schur_op(v[r], U, DIMS, 0.131, w, bc, dagger)
        assert rel(out[r], ref) < tol


@pytest.mark.parametrize("tdt,tol", [(torch.float16, 4e-3), (torch.bfloat16, 3e-2)])
def test_schur_operator_half_storage(tdt, tol):
    U = synthetic.smooth_links(DIMS, 82)
    v = _even_fields(1, 83)
    out = from_half_pair(api.schur(half_pair(v, tdt), half_pair(U, tdt), DIMS, 0.131, ANISO,
                                   (1, 1, 1, -1)))
    assert rel(out[0], schur.schur_op(v[0], U, DIMS, 0.131, ANISO, (1, 1, 1, -1))) < tol


def _oracle_level(cfg, U, schur_smoother):
    Pt, _, _ = icsvd.icsvd(U, cfg["dims"], cfg["kappa"], cfg["hop_weight"], cfg["bc"],
                           cfg["block"], cfg["k"], cfg["r"], cfg["n_s"], cfg["sweeps"],
                           cfg["tv_seed"])
    return mg.TwoLevel(U, cfg["dims"], cfg["kappa"], cfg["hop_weight"], cfg["bc"], cfg["block"],
                       Pt, schur=schur_smoother)


@pytest.mark.parametrize("cfg", [C1, C5], ids=["c1", "c5"])
def test_fp64_schur_smoothed_solve_matches_oracle(cfg):
    """FP64 K-cycle FGMRES with the Schur-form post-smoother: the solution and the outer
    iteration count of the oracle's two-level solve with the same smoother (within one)."""
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])
    p = params_for(cfg, setup_dtype="c128", solve_dtype="c128", schur_smoother=1)
    h = api.Hierarchy(to_dev(U), p)
    h.coarse_build()
    x, info = h.solve(to_dev(b), tol=1e-10)
    x = x.cpu().numpy()[0]
    xo, info_o = _oracle_level(cfg, U, True).solve(b[0].reshape(-1), tol=1e-10)
    r = b[0].reshape(-1) - wilson.dslash(x, U, cfg["dims"], cfg["kappa"], cfg["hop_weight"],
                                         cfg["bc"]).reshape(-1)
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= 1e-10
    assert rel(x.reshape(-1), xo) < 1e-8
    assert abs(info["outer"] - info_o["outer"]) <= 1
    h.close()


@pytest.mark.parametrize("cfg", [C1, C5], ids=["c1", "c5"])
def test_mixed_schur_smoothed_solve(cfg):
    """The mixed form (FP32 inner K-cycle with the Schur-form smoother, FP64 refinement)
    reaches a true residual of 1e-10, computed with the oracle's D, on two right-hand sides."""
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"], 2)
    p = params_for(cfg, schur_smoother=1)
    h = api.Hierarchy(to_dev(U), p)
    h.coarse_build()
    x, info = h.solve(to_dev(b), tol=1e-10)
    x = x.cpu().numpy()
    for k in range(2):
        r = b[k].reshape(-1) - wilson.dslash(x[k], U, cfg["dims"], cfg["kappa"],
                                             cfg["hop_weight"], cfg["bc"]).reshape(-1)
        assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1e-10
    h.close()
