"""Failure paths on the GPU without faulting it: bounded waits, errors reported as statuses."""
import numpy as np
import pytest
import torch

from oracle import wilson
from paper_2505_14399_gb300 import _lib as L
from paper_2505_14399_gb300 import api, synthetic
from gpu_common import rel, to_dev

pytestmark = pytest.mark.gpu


def test_bounded_barrier_wait_reports_timeout_and_context_survives():
    st = L.lib().mg_selftest_barrier_timeout(None)
    assert st == L.MG_ETIMEOUT
    assert b"bounded wait" in L.lib().mg_last_error()
    dims = (4, 4, 4, 4)
    U = synthetic.haar_links(dims, 1)
    psi = synthetic.gaussian_rhs(dims, 2)
    out = api.dslash(to_dev(psi), to_dev(U), dims, 0.12)
    assert rel(out.cpu().numpy()[0], wilson.dslash(psi[0], U, dims, 0.12)) < 1e-12


def test_solver_hits_maxiter_with_enoconv():
    cfg = synthetic.WORKLOADS["c1_4^4_haar"]
    U = synthetic.make_links(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])
    p = api.params(cfg["dims"], cfg["block"], cfg["kappa"], cfg["k"], cfg["r"], cfg["n_s"],
                   solve_dtype="c128")
    h = api.Hierarchy(to_dev(U), p)
    h.coarse_build()
    with pytest.raises(L.MgError) as ei:
        h.solve(to_dev(b), tol=1e-14, maxiter=1)
    assert ei.value.status == L.MG_ENOCONV
    # the handle stays usable
    x, info = h.solve(to_dev(b), tol=1e-10)
    assert info["residual"] <= 1e-10
    h.close()


def test_nan_input_is_reported():
    cfg = synthetic.WORKLOADS["c1_4^4_haar"]
    U = synthetic.make_links(cfg)
    b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"])
    b[0, 3, 1, 2] = np.nan
    p = api.params(cfg["dims"], cfg["block"], cfg["kappa"], cfg["k"], cfg["r"], cfg["n_s"])
    h = api.Hierarchy(to_dev(U), p)
    h.coarse_build()
    with pytest.raises(L.MgError) as ei:
        h.solve(to_dev(b), tol=1e-10)
    assert ei.value.status in (L.MG_ENAN, L.MG_ENOCONV)
    h.close()


def test_bad_parameters_are_rejected_before_any_launch():
    cfg = synthetic.WORKLOADS["c1_4^4_haar"]
    U = synthetic.make_links(cfg)
    for kw in (dict(k=0), dict(k=200), dict(block=(3, 2, 2, 2))):
        args = dict(dims=cfg["dims"], block=cfg["block"], kappa=cfg["kappa"], k=cfg["k"],
                    r=cfg["r"], n_s=cfg["n_s"])
        args.update(kw)
        with pytest.raises(L.MgError) as ei:
            api.Hierarchy(to_dev(U), api.params(**args))
        assert ei.value.status == L.MG_EINVAL
