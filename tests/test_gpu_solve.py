"""GPU K-cycle preconditioned solve of D x = b (Eq. 1) vs the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import icsvd, mg, wilson
from paper_2505_14399_gb300 import api, synthetic
from gpu_common import links_for, params_for, rel, to_dev

pytestmark = pytest.mark.gpu

C1 = synthetic.WORKLOADS["c1_4^4_haar"]
C5 = synthetic.WORKLOADS["c5_8^4_autograd"]


def _true_residual(cfg, U, x, b):
    r = b.reshape(-1) - wilson.dslash(x, U, cfg["dims"], cfg["kappa"], cfg["hop_weight"],
                                      cfg["bc"]).reshape(-1)
    return np.linalg.norm(r) / np.linalg.norm(b)


def test_fp64_solve_matches_oracle_two_level():
    cfg = C1
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])
    p = params_for(cfg, setup_dtype="c128", solve_dtype="c128")
    h = api.Hierarchy(to_dev(U), p)
    h.coarse_build()
    x, info = h.solve(to_dev(b), tol=1e-10)
    x = x.cpu().numpy()[0]
    Pt, S, _ = icsvd.icsvd(U, cfg["dims"], cfg["kappa"], cfg["hop_weight"], cfg["bc"], cfg["block"],
                           cfg["k"], cfg["r"], cfg["n_s"], cfg["sweeps"], cfg["tv_seed"])
    tl = mg.TwoLevel(U, cfg["dims"], cfg["kappa"], cfg["hop_weight"], cfg["bc"], cfg["block"], Pt)
    xo, info_o = tl.solve(b[0].reshape(-1), tol=1e-10)
    assert _true_residual(cfg, U, x, b[0]) <= 1e-10
    assert rel(x.reshape(-1), xo) < 1e-8
    assert abs(info["outer"] - info_o["outer"]) <= 1
    assert abs(info["coarse"] - info_o["coarse"]) <= max(2, 0.1 * info_o["coarse"])
    h.close()


@pytest.mark.parametrize("solve_dtype", ["c128", "c64"])
def test_persistent_coarse_solver_matches_launch_per_op(solve_dtype):
    """The one-launch coarse GMRES takes the same steps as the kernel-per-operation one."""
    cfg = C5
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"], 2)
    out = {}
    for pers in (0, 1):
        p = params_for(cfg, setup_dtype="c128", solve_dtype=solve_dtype, coarse_persistent=pers)
        h = api.Hierarchy(to_dev(U), p)
        h.coarse_build()
        x, info = h.solve(to_dev(b), tol=1e-10)
        out[pers] = (x.cpu().numpy(), info)
        h.close()
    (x0, i0), (x1, i1) = out[0], out[1]
    assert i0["outer"] == i1["outer"]
    assert abs(i0["coarse"] - i1["coarse"]) <= 2 * i0["kcycles"] * (0 if solve_dtype == "c128" else 1)
    for r in range(2):
        assert _true_residual(cfg, U, x1[r], b[r]) <= 1e-10
        assert rel(x1[r], x0[r]) < 1e-8


@pytest.mark.parametrize("cfg", [C1, C5])
def test_mixed_precision_solve_reaches_1e10(cfg):
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"], 2)
    p = params_for(cfg, setup_dtype="c64", solve_dtype="c64")
    h = api.Hierarchy(to_dev(U), p)
    h.coarse_build()
    x, info = h.solve(to_dev(b), tol=1e-10)
    x = x.cpu().numpy()
    for r in range(2):
        assert _true_residual(cfg, U, x[r], b[r]) <= 1e-10
    assert info["refinements"] >= 2
    # adjoint solve: D^dag x = b
    xa, _ = h.solve(to_dev(b), tol=1e-10, adjoint=True)
    xa = xa.cpu().numpy()
    for r in range(2):
        Dd = wilson.dslash(xa[r], U, cfg["dims"], cfg["kappa"], cfg["hop_weight"], cfg["bc"],
                           dagger=True)
        assert rel(Dd, b[r]) <= 1e-10
    h.close()


def test_host_pointers_solve():
    cfg = C1
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])
    p = params_for(cfg)
    h = api.Hierarchy(torch.from_numpy(U), p)   # host links
    h.coarse_build()
    x, info = h.solve(torch.from_numpy(b), tol=1e-10)   # host b and x
    assert _true_residual(cfg, U, x.numpy()[0], b[0]) <= 1e-10
    h.close()


def test_full_size_near_critical_solve():
    cfg = synthetic.WORKLOADS["c2_16^3x32_near_critical"]
    kappa = synthetic.kappa_of(cfg)
    c = dict(cfg, kappa=kappa)
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])
    for solve_dtype in ("c64", "c128"):
        p = params_for(c, setup_dtype="c64", solve_dtype=solve_dtype)
        h = api.Hierarchy(to_dev(U), p)
        h.coarse_build()
        x, info = h.solve(to_dev(b), tol=1e-10, maxiter=2000)
        assert _true_residual(c, U, x.cpu().numpy()[0], b[0]) <= 1e-10
        h.close()
