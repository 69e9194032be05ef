"""The solver's stencil with two stored rows per link (third row rebuilt as the conjugate cross
product, exact for SU(3)) against the FP64 oracle, and the choice between two and three rows."""
import numpy as np
import pytest
import torch

from oracle import wilson
from paper_2505_14399_gb300 import _lib as L, api, synthetic
from gpu_common import from_half_pair, half_pair, rel, to_dev

pytestmark = pytest.mark.gpu

DIMS = (6, 4, 6, 10)          # 1440 sites: a ragged last CTA
W, BC = (1.0, 1.0, 1.0, 1 / 3.5), (1, 1, 1, -1)


def _handle(U, compress, solve_dtype="c64"):
    p = api.params(DIMS, (2, 2, 2, 2), 0.127, 4, 4, 1, hop_weight=W, bc=BC,
                   solve_dtype=solve_dtype, link_compress=compress)
    return api.Hierarchy(to_dev(U), p, setup=False)


@pytest.mark.parametrize("links", ["haar", "smooth"])
@pytest.mark.parametrize("dagger", [False, True])
def test_two_rows_fp32(links, dagger):
    U = synthetic.haar_links(DIMS, 70) if links == "haar" else synthetic.smooth_links(DIMS, 71)
    psi = synthetic.gaussian_rhs(DIMS, 72, 2)
    h2, h3 = _handle(U, 1), _handle(U, 0)
    assert L.lib().mg_link_rows(h2._h) == 2 and L.lib().mg_link_rows(h3._h) == 3
    o2 = h2.apply_fine(to_dev(psi, torch.complex64), dagger=dagger).cpu().numpy()
    o3 = h3.apply_fine(to_dev(psi, torch.complex64), dagger=dagger).cpu().numpy()
    for r in range(2):
        ref = wilson.dslash(psi[r], U, DIMS, 0.127, W, BC, dagger)
        assert rel(o2[r], ref) < 1e-5
        assert rel(o2[r], o3[r]) < 1e-6      # both FP32: the rebuilt row adds ~1 ulp
    h2.close()
    h3.close()


@pytest.mark.parametrize("dt,tdt,tol", [("f16", torch.float16, 2e-3), ("bf16", torch.bfloat16, 1.5e-2)])
def test_two_rows_half(dt, tdt, tol):
    U = synthetic.smooth_links(DIMS, 73)
    psi = synthetic.gaussian_rhs(DIMS, 74, 2)
    h = _handle(U, 1, dt)
    out = from_half_pair(h.apply_fine(half_pair(psi, tdt)))
    for r in range(2):
        assert rel(out[r], wilson.dslash(psi[r], U, DIMS, 0.127, W, BC)) < tol
    h.close()


def test_auto_keeps_three_rows_for_non_su3_links():
    """link_compress = -1 keeps three rows when a link is not SU(3) (here U(3) links with a
    phase on the determinant), and the stencil still matches the oracle; link_compress = 1
    refuses such links."""
    U = synthetic.haar_links(DIMS, 75) * np.exp(0.3j)
    psi = synthetic.gaussian_rhs(DIMS, 76, 1)
    h = _handle(U, -1)
    assert L.lib().mg_link_rows(h._h) == 3
    out = h.apply_fine(to_dev(psi, torch.complex64)).cpu().numpy()
    assert rel(out[0], wilson.dslash(psi[0], U, DIMS, 0.127, W, BC)) < 1e-5
    h.close()
    with pytest.raises(L.MgError):
        _handle(U, 1)
    h = _handle(synthetic.haar_links(DIMS, 77), -1)
    assert L.lib().mg_link_rows(h._h) == 2
    h.close()


@pytest.mark.parametrize("solve_dtype", ["c64", "c128"])   # double-float check / FP64 check
def test_auto_threshold_resolves_1e9(solve_dtype):
    """The automatic choice resolves deviations from SU(3) around its 1e-9 threshold: one link
    scaled by 1 + 1e-8 (|U U^dag - 1| ~ 2e-8) keeps three rows, by 1 + 1e-11 two rows -- from
    the double-float link copy (mixed forms) and from the FP64 links (FP64 form)."""
    U = synthetic.haar_links(DIMS, 78)
    for eps, rows in ((1e-8, 3), (1e-11, 2)):
        Up = U.copy()
        Up[0, 0] *= 1.0 + eps
        h = _handle(Up, -1, solve_dtype)
        assert L.lib().mg_link_rows(h._h) == rows, (eps, solve_dtype)
        h.close()
