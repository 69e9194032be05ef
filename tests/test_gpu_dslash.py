"""GPU Wilson-Dirac stencil vs the FP64 oracle (all storage types, full and parity forms)."""
import numpy as np
import pytest
import torch

from oracle import wilson
from paper_2505_14399_gb300 import api, synthetic
from gpu_common import from_half_pair, half_pair, rel, to_dev

pytestmark = pytest.mark.gpu

# 1440 sites: 11.25 CTAs of 128 threads (ragged tail), all extents even
DIMS = (6, 4, 6, 10)
ANISO = (1.0, 1.0, 1.0, 1 / 3.5)
CASES = [((1, 1, 1, 1), (1, 1, 1, 1)), (ANISO, (1, 1, 1, -1)), ((0.7, 1.0, 1.3, 1.0), (-1, 1, 1, 1))]
TOL = {torch.complex128: 1e-12, torch.complex64: 1e-5}


def _fields(dims, nrhs, seed):
    U = synthetic.haar_links(dims, seed)
    psi = synthetic.gaussian_rhs(dims, seed + 1, nrhs)
    return U, psi


@pytest.mark.parametrize("w,bc", CASES)
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("dagger", [False, True])
def test_full_operator(w, bc, dtype, dagger):
    U, psi = _fields(DIMS, 3, 10)
    out = api.dslash(to_dev(psi, dtype), to_dev(U, dtype), DIMS, 0.137, w, bc, dagger=dagger)
    o = out.cpu().numpy()
    for r in range(3):
        ref = wilson.dslash(psi[r], U, DIMS, 0.137, w, bc, dagger)
        assert rel(o[r], ref) < TOL[dtype]


@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_parity_operator(parity, dtype):
    U, psi = _fields(DIMS, 2, 20)
    par = wilson.parity_of_sites(DIMS)
    half = np.ascontiguousarray(psi[:, par == 1 - parity])
    out = api.dslash(to_dev(half, dtype), to_dev(U, dtype), DIMS, 0.12, ANISO, (1, 1, 1, -1),
                     parity=parity)
    o = out.cpu().numpy()
    for r in range(2):
        ref = wilson.dslash_parity(half[r], U, DIMS, 0.12, parity, ANISO, (1, 1, 1, -1))
        assert rel(o[r], ref) < TOL[dtype]


@pytest.mark.parametrize("dtype,tol", [(torch.float16, 2e-3), (torch.bfloat16, 1.5e-2)])
def test_half_storage(dtype, tol):
    U, psi = _fields(DIMS, 2, 30)
    out = api.dslash(half_pair(psi, dtype), half_pair(U, dtype), DIMS, 0.12, ANISO, (1, 1, 1, -1))
    o = from_half_pair(out)
    for r in range(2):
        ref = wilson.dslash(psi[r], U, DIMS, 0.12, ANISO, (1, 1, 1, -1))
        assert rel(o[r], ref) < tol


def test_full_size_fp32_matches_oracle():
    """16^3 x 32, complex64, the launch configuration the solver uses."""
    cfg = synthetic.WORKLOADS["c2_16^3x32_near_critical"]
    dims = cfg["dims"]
    U = synthetic.make_links(cfg)
    psi = synthetic.gaussian_rhs(dims, 5)
    out = api.dslash(to_dev(psi, torch.complex64), to_dev(U, torch.complex64), dims, 0.13)
    ref = wilson.dslash(psi[0], U, dims, 0.13)
    assert rel(out.cpu().numpy()[0], ref) < 1e-5


def test_host_buffers_are_staged():
    U, psi = _fields(DIMS, 1, 40)
    out = np.zeros_like(psi)
    import ctypes
    from paper_2505_14399_gb300 import _lib as L
    st = L.lib().wilson_dslash(ctypes.c_void_p(out.ctypes.data), ctypes.c_void_p(psi.ctypes.data),
                               ctypes.c_void_p(U.ctypes.data), L.ivec(DIMS), 0.11, L.dvec((1, 1, 1, 1)),
                               L.ivec((1, 1, 1, 1)), -1, 0, L.MG_C128, 1, None)
    assert st == L.MG_OK
    assert rel(out[0], wilson.dslash(psi[0], U, DIMS, 0.11)) < 1e-12


def test_invalid_arguments_are_rejected():
    from paper_2505_14399_gb300 import _lib as L
    U, psi = _fields((4, 4, 4, 4), 1, 1)
    with pytest.raises(L.MgError):
        api.dslash(to_dev(psi[:, :-1].copy()), to_dev(U), (4, 4, 4, 3), 0.1, parity=0)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("dagger", [False, True])
def test_handle_operator_lane_contiguous_links(dtype, dagger):
    """The solver's stencil (lane-contiguous link copy) against the oracle."""
    dims = DIMS
    U, psi = _fields(dims, 2, 50)
    w, bc = ANISO, (1, 1, 1, -1)
    p = api.params(dims, (2, 2, 2, 2), 0.127, 4, 4, 1, hop_weight=w, bc=bc)
    h = api.Hierarchy(to_dev(U), p, setup=False)
    out = h.apply_fine(to_dev(psi, dtype), dagger=dagger).cpu().numpy()
    for r in range(2):
        ref = wilson.dslash(psi[r], U, dims, 0.127, w, bc, dagger)
        assert rel(out[r], ref) < TOL[dtype]
    h.close()


@pytest.mark.parametrize("dt,tdt,tol", [("f16", torch.float16, 2e-3), ("bf16", torch.bfloat16, 1.5e-2)])
def test_handle_operator_half_links(dt, tdt, tol):
    """The half-storage smoother's stencil (lane-contiguous half links) against the oracle."""
    U, psi = _fields(DIMS, 2, 60)
    w, bc = ANISO, (1, 1, 1, -1)
    p = api.params(DIMS, (2, 2, 2, 2), 0.127, 4, 4, 1, hop_weight=w, bc=bc, solve_dtype=dt)
    h = api.Hierarchy(to_dev(U), p, setup=False)
    out = from_half_pair(h.apply_fine(half_pair(psi, tdt)))
    for r in range(2):
        assert rel(out[r], wilson.dslash(psi[r], U, DIMS, 0.127, w, bc)) < tol
    h.close()
