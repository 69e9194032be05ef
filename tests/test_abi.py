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
