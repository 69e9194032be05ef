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


@pytest.mark.parametrize("solve_dtype", ["f16", "bf16"])
@pytest.mark.parametrize("cfg", [C1, C5])
def test_half_storage_smoother_solve_reaches_1e10(cfg, solve_dtype):
    """K-cycle post-smoother in FP16/BF16 storage (FP32 arithmetic) inside FP64 refinement."""
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"], 2)
    p = params_for(cfg, setup_dtype="c64", solve_dtype=solve_dtype)
    h = api.Hierarchy(to_dev(U), p)
    h.coarse_build()
    x, info = h.solve(to_dev(b), tol=1e-10)
    x = x.cpu().numpy()
    for r in range(2):
        assert _true_residual(cfg, U, x[r], b[r]) <= 1e-10
    # the half smoother may cost iterations, not correctness: stay within 2x of FP32's
    p32 = params_for(cfg, setup_dtype="c64", solve_dtype="c64")
    h32 = api.Hierarchy(to_dev(U), p32)
    h32.coarse_build()
    _, info32 = h32.solve(to_dev(b), tol=1e-10)
    assert info["outer"] <= 2 * info32["outer"] + 2
    h.close()
    h32.close()


def test_full_size_anisotropic_half_storage_solve():
    """16^3 x 64, w_t = 1/3.5, 2x2x2x4 aggregates, k = 24, 64 test vectors streamed in 4:
    FP16 and BF16 smoother storage inside FP64 refinement reach 1e-10 (FP64 oracle check)."""
    cfg = synthetic.WORKLOADS["c3_16^3x64_aniso"]
    c = dict(cfg, kappa=synthetic.kappa_of(cfg))
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])
    for solve_dtype in ("f16", "bf16"):
        p = params_for(c, setup_dtype="c64", solve_dtype=solve_dtype)
        h = api.Hierarchy(to_dev(U), p)
        h.coarse_build()
        x, info = h.solve(to_dev(b), tol=1e-10, maxiter=3000)
        assert _true_residual(c, U, x.cpu().numpy()[0], b[0]) <= 1e-10
        h.close()


def test_full_size_batched_12_rhs_32c64():
    """32^3 x 64, 4^4 aggregates, k = 24, 48 test vectors in 2 streams, 12 Gaussian
    right-hand sides solved together (one batched FGMRES, every Dslash and BLAS launch over
    all 12): each reaches 1e-10.  The FP64 oracle checks one sampled right-hand side, the
    library's FP64 stencil all of them."""
    import time
    cfg = synthetic.WORKLOADS["c4_32^3x64_12rhs"]
    c = dict(cfg, kappa=synthetic.kappa_of(cfg))
    dims = cfg["dims"]
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(dims, cfg["rhs_seed"], cfg["nrhs"])
    p = params_for(c, setup_dtype="c64", solve_dtype="c64", outer_restart=8)
    Ud = to_dev(U)
    bd = to_dev(b)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = api.Hierarchy(Ud, p)
    h.coarse_build()
    x, info = h.solve(bd, tol=1e-10, maxiter=2000)
    torch.cuda.synchronize()
    print("32^3x64 x 12 rhs: setup+solve %.2f s, %s" % (time.perf_counter() - t0, info))
    r = bd - api.dslash(x, Ud, dims, c["kappa"], c["hop_weight"], c["bc"])
    rel_res = (torch.linalg.vector_norm(r.reshape(cfg["nrhs"], -1), dim=1)
               / torch.linalg.vector_norm(bd.reshape(cfg["nrhs"], -1), dim=1))
    assert float(rel_res.max()) <= 1e-10
    assert _true_residual(c, U, x[0].cpu().numpy(), b[0]) <= 1e-10
    h.close()
