"""GPU adjoint: link-angle gradient kernel vs the oracle, autograd vs finite differences."""
import numpy as np
import pytest
import torch

from oracle import adjoint, wilson
from paper_2505_14399_gb300 import api, synthetic
from gpu_common import links_for, params_for, rel, to_dev

pytestmark = pytest.mark.gpu


def test_link_gradient_kernel_matches_oracle():
    dims = (4, 6, 4, 8)
    U = synthetic.smooth_links(dims, 3)
    rng = np.random.default_rng(1)
    V = wilson.volume(dims)
    gb = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
    x = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
    w, bc = (1, 1, 1, 0.4), (1, 1, 1, -1)
    out = api.link_gradient(to_dev(gb), to_dev(x), to_dev(U), dims, 0.11, w, bc).cpu().numpy()
    ref = adjoint.grad_link_angles(gb, x, U, dims, 0.11, w, bc)
    assert rel(out, ref) < 1e-12


def test_autograd_matches_finite_differences():
    """loss |x|^2, x = D^{-1} b: gradients in b and link angles vs central FD (h = 1e-4)."""
    cfg = dict(synthetic.WORKLOADS["c5_8^4_autograd"])
    dims = cfg["dims"]
    U = links_for(cfg)
    b = synthetic.gaussian_rhs(dims, cfg["rhs_seed"])
    V = wilson.volume(dims)
    p = params_for(cfg, setup_dtype="c64", solve_dtype="c128")
    h = api.Hierarchy(to_dev(U), p)
    h.coarse_build()
    bt = to_dev(b).requires_grad_(True)
    om = torch.zeros((4, V, 8), dtype=torch.float64, device="cuda:0", requires_grad=True)
    x = api.mg_solve_autograd(bt, om, h, to_dev(U), 1e-12)
    loss = (x.abs() ** 2).sum()
    loss.backward()
    gb = bt.grad.cpu().numpy()
    gom = om.grad.cpu().numpy()

    def L(links, src):
        hh = api.Hierarchy(to_dev(links), p)
        hh.coarse_build()
        xx, _ = hh.solve(to_dev(src), tol=1e-13)
        hh.close()
        return float((xx.abs() ** 2).sum())

    rng = np.random.default_rng(11)
    eps = 1e-4
    errs = []
    for i in range(32):
        if i % 2 == 0:
            db = rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape)
            fd = (L(U, b + eps * db) - L(U, b - eps * db)) / (2 * eps)
            an = float(np.real(np.vdot(gb, db)))
        else:
            do = rng.standard_normal((4, V, 8))
            fd = (L(adjoint.perturb_links(U, eps * do), b)
                  - L(adjoint.perturb_links(U, -eps * do), b)) / (2 * eps)
            an = float((gom * do).sum())
        errs.append(abs(fd - an) / max(abs(fd), 1e-3 * abs(float(loss.detach()))))
    assert max(errs) < 1e-5, errs
    h.close()
