"""coarse_build_noalloc: the Galerkin rebuild (Eq. 5) with its scratch in a fixed device
array instead of a device allocation, called through the C ABI and compared with
coarse_build on the same hierarchy."""
import ctypes

import numpy as np
import pytest

from paper_2505_14399_gb300 import _lib as L, api, synthetic
from gpu_common import params_for, random_tiles, rel, to_dev

pytestmark = pytest.mark.gpu

# both give the same kernels in the same order; the bound leaves room for nothing else
TOL = 1e-14


def _handle(dims, block, k, seed, solve_dtype="c64"):
    U = synthetic.smooth_links(dims, seed)
    p = api.params(dims, block, 0.125, k, k, 1, hop_weight=(1, 1, 1, 1 / 3.5),
                   bc=(1, 1, 1, -1), setup_dtype=solve_dtype, solve_dtype=solve_dtype)
    h = api.Hierarchy(to_dev(U), p, setup=False)
    d = int(np.prod(dims)) // int(np.prod(block))
    h.set_prolongator(to_dev(random_tiles(d, int(np.prod(block)), k, seed + 1)))
    return h, U, p


def _noalloc(h):
    st = L.lib().coarse_build_noalloc(h._h, None)
    assert st == L.MG_OK, L.lib().mg_last_error().decode()


def _op(h):
    X, Y = h.coarse_op()
    return X.cpu().numpy(), Y.cpu().numpy()


@pytest.mark.parametrize("solve_dtype", ["c64", "c128"])   # double-float and FP64 Galerkin
def test_two_calls_in_a_row_match_coarse_build(solve_dtype):
    dims, block, k = (6, 4, 4, 8), (2, 2, 2, 4), 7
    h, U, p = _handle(dims, block, k, 11, solve_dtype)
    h.coarse_build()
    X0, Y0 = _op(h)
    for _ in range(2):
        _noalloc(h)
        X1, Y1 = _op(h)
        assert rel(X1, X0) < TOL and rel(Y1, Y0) < TOL
    # a new prolongator: the rebuild must follow it (checked against a fresh handle)
    d = int(np.prod(dims)) // int(np.prod(block))
    P2 = random_tiles(d, int(np.prod(block)), k, 99)
    h.set_prolongator(to_dev(P2))
    _noalloc(h)
    X2, Y2 = _op(h)
    ref = api.Hierarchy(to_dev(U), p, setup=False)
    ref.set_prolongator(to_dev(P2))
    ref.coarse_build()
    Xr, Yr = _op(ref)
    assert rel(X2, X0) > 1e-3
    assert rel(X2, Xr) < TOL and rel(Y2, Yr) < TOL
    ref.close()
    h.close()


def test_calls_allocate_no_device_memory():
    """Around two calls in a row, neither the device's free memory (cudaMemGetInfo: the
    library's own allocations, the stream-ordered pool, lazily loaded code) nor torch's
    allocator changes.  The first call comes before the measurement: it may load the library's
    module with the fixed scratch array in it."""
    import torch
    dims, block, k = (8, 8, 8, 8), (2, 2, 2, 2), 9
    h, _, _ = _handle(dims, block, k, 61)
    h.coarse_build()
    _noalloc(h)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    _noalloc(h)
    _noalloc(h)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0
    h.close()


def test_scratch_left_by_a_larger_hierarchy_is_harmless():
    big, _, _ = _handle((8, 8, 8, 8), (2, 2, 2, 2), 12, 21)
    big.coarse_build()
    _noalloc(big)
    small, _, _ = _handle((4, 4, 4, 4), (2, 2, 2, 2), 3, 31)
    small.coarse_build()
    X0, Y0 = _op(small)
    _noalloc(small)
    _noalloc(small)
    X1, Y1 = _op(small)
    assert rel(X1, X0) < TOL and rel(Y1, Y0) < TOL
    big.close()
    small.close()


def test_full_size_near_critical_hierarchy():
    """16^3x32, k = 12, iCSVD prolongator: d k^2 = 73728 fits the fixed scratch."""
    cfg = synthetic.WORKLOADS["c2_16^3x32_near_critical"]
    U = synthetic.make_links(cfg)
    h = api.Hierarchy(to_dev(U), params_for(cfg, kappa=synthetic.kappa_of(cfg)))
    h.coarse_build()
    X0, Y0 = _op(h)
    _noalloc(h)
    _noalloc(h)
    X1, Y1 = _op(h)
    assert rel(X1, X0) < TOL and rel(Y1, Y0) < TOL
    h.close()


def test_rejects_hierarchy_beyond_scratch():
    # 4096 coarse sites, k = 5: d k^2 = 102400 > 98304
    h, _, _ = _handle((8, 8, 8, 8), (1, 1, 1, 1), 5, 41)
    st = L.lib().coarse_build_noalloc(h._h, None)
    assert st == L.MG_EINVAL
    assert b"98304" in L.lib().mg_last_error()
    h.close()


def test_requires_storage_from_coarse_build():
    h, _, _ = _handle((4, 4, 4, 4), (2, 2, 2, 2), 3, 51)
    st = L.lib().coarse_build_noalloc(h._h, None)
    assert st == L.MG_EINVAL
    assert b"coarse_build once" in L.lib().mg_last_error()
    assert L.lib().coarse_build_noalloc(ctypes.c_void_p(), None) == L.MG_EINVAL
    h.close()
