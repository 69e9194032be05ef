"""The C ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wilson_mg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char\*|long long)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_14399_gb300 import _build, _lib
    _build.build()
    return _lib.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("wilson_dslash", "mg_setup_streaming_svd", "coarse_build", "mg_solve", "mg_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_defaults_and_errors_without_gpu(lib):
    from paper_2505_14399_gb300 import _lib
    p = _lib.MgParams()
    lib.mg_params_default(ctypes.byref(p))
    assert p.post_smooth == 8 and abs(p.coarse_tol - 0.03) < 1e-15
    # argument validation happens before any device call
    dims = _lib.ivec((4, 4, 4, 4))
    st = lib.wilson_dslash(None, None, None, dims, 0.1, None, None, -1, 0, 0, 1, None)
    assert st == _lib.MG_EINVAL
    assert b"NULL" in lib.mg_last_error()
    h = ctypes.c_void_p()
    p.k = 0
    st = lib.mg_setup_streaming_svd(ctypes.byref(h), ctypes.c_void_p(1), ctypes.byref(p), None)
    assert st == _lib.MG_EINVAL


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_2505_14399_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def _set(p, field, value):
    cur = getattr(p, field)
    if hasattr(cur, "__setitem__"):
        cur[value[0]] = value[1]
    else:
        setattr(p, field, value)


# one broken field at a time, starting from the defaults (4^4 lattice, 2^4 aggregates, k = 24,
# r = 24, n_s = 2): (changes, fragment of the error message)
BAD_SETUP = [
    ([("dims", (0, 3))], "even"),
    ([("dims", (2, 0))], "even"),
    ([("block", (1, 3))], "block must divide"),
    ([("block", (2, 0))], "block must divide"),
    ([("k", 0)], "k must be in"),
    ([("block", (0, 1)), ("block", (1, 1)), ("block", (2, 1)), ("block", (3, 1)), ("k", 7),
      ("r", 8)], "k must be in"),
    ([("k", 33)], "k > 32"),
    ([("r", 0)], "r and n_s"),
    ([("n_s", 0)], "r and n_s"),
    ([("k", 32), ("r", 33)], "k + r"),
    ([("k", 12), ("r", 4), ("n_s", 2)], "n_s * r"),
    ([("sweeps", 65)], "sweeps"),
    ([("sweeps", -1)], "sweeps"),
    ([("setup_dtype", 2)], "setup_dtype"),
    ([("solve_dtype", 9)], "solve_dtype"),
    ([("post_smooth", -1)], "post_smooth"),
    ([("coarse_restart", 0)], "coarse_restart"),
    ([("outer_restart", 129)], "outer_restart"),
    ([("coarse_tol", 1.0)], "coarse_tol"),
    ([("coarse_tol", 0.0)], "coarse_tol"),
    ([("coarse_persistent", 1), ("coarse_restart", 64)], "persistent"),
    ([("bc_phase", (3, 2))], "bc_phase"),
]


@pytest.mark.parametrize("changes,msg", BAD_SETUP, ids=[m for _, m in BAD_SETUP])
def test_setup_rejects_each_bad_parameter_before_any_device_call(lib, changes, msg):
    from paper_2505_14399_gb300 import _lib
    p = _lib.MgParams()
    lib.mg_params_default(ctypes.byref(p))
    for field, value in changes:
        _set(p, field, value)
    h = ctypes.c_void_p()
    st = lib.mg_setup_streaming_svd(ctypes.byref(h), ctypes.c_void_p(16), ctypes.byref(p), None)
    assert st == _lib.MG_EINVAL
    assert msg.encode() in lib.mg_last_error()
    assert not h.value


def test_setup_rejects_bad_handle_arguments(lib):
    from paper_2505_14399_gb300 import _lib
    p = _lib.MgParams()
    lib.mg_params_default(ctypes.byref(p))
    h = ctypes.c_void_p()
    assert lib.mg_setup_streaming_svd(ctypes.byref(h), None, ctypes.byref(p), None) == _lib.MG_EINVAL
    assert b"links" in lib.mg_last_error()
    h = ctypes.c_void_p(64)                              # *h must be NULL on entry
    assert lib.mg_setup_streaming_svd(ctypes.byref(h), ctypes.c_void_p(16), ctypes.byref(p),
                                      None) == _lib.MG_EINVAL
    assert h.value == 64
    assert lib.mg_setup_streaming_svd(None, ctypes.c_void_p(16), ctypes.byref(p), None) == _lib.MG_EINVAL


# (dims, bc, parity, dtype, nrhs, aliased, fragment)
BAD_DSLASH = [
    ((4, 4, 4, 4), (1, 1, 1, 1), -1, 0, 0, False, "nrhs"),
    ((4, 4, 4, 4), (1, 1, 1, 1), 2, 0, 1, False, "parity"),
    ((4, 4, 4, 4), (1, 1, 1, 1), -1, 7, 1, False, "dtype"),
    ((0, 4, 4, 4), (1, 1, 1, 1), -1, 0, 1, False, "extent"),
    ((4, 3, 4, 4), (1, 1, 1, 1), 0, 1, 1, False, "even"),
    ((4, 4, 4, 4), (1, 1, 0, 1), -1, 1, 1, False, "bc_phase"),
    ((4, 4, 4, 4), (1, 1, 1, 1), -1, 1, 1, True, "alias"),
]


@pytest.mark.parametrize("dims,bc,parity,dtype,nrhs,aliased,msg", BAD_DSLASH,
                         ids=[c[-1] for c in BAD_DSLASH])
def test_dslash_rejects_bad_arguments_before_any_device_call(lib, dims, bc, parity, dtype, nrhs,
                                                             aliased, msg):
    from paper_2505_14399_gb300 import _lib
    a, b, u = ctypes.c_void_p(256), ctypes.c_void_p(512), ctypes.c_void_p(1024)
    st = lib.wilson_dslash(a, a if aliased else b, u, _lib.ivec(dims), 0.1, None, _lib.ivec(bc),
                           parity, 0, dtype, nrhs, None)
    assert st == _lib.MG_EINVAL
    assert msg.encode() in lib.mg_last_error()


def test_autograd_rejects_nonzero_link_angles():
    """MGSolve differentiates at the given links (omega = 0); any other omega is an error,
    raised on the host before any solve."""
    import torch
    from paper_2505_14399_gb300 import api
    b = torch.zeros((1, 16, 4, 3), dtype=torch.complex128)
    om = torch.zeros((4, 16, 8), dtype=torch.float64)
    om[1, 3, 2] = 1e-3
    with pytest.raises(ValueError, match="omega must be zero"):
        api.mg_solve_autograd(b, om, None, None)
