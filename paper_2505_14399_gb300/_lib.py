"""ctypes declarations of the C ABI in include/wilson_mg.h (argument marshalling only).

The shared library is built in-tree by ``paper_2505_14399_gb300._build`` (or
``__graft_entry__.build()``).  Loading fails loudly when it is missing: there is no
CPU fallback for any entry point.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwilsonmg.so")

MG_OK, MG_EINVAL, MG_ENOMEM, MG_ECUDA, MG_ENOCONV, MG_ETIMEOUT, MG_ENAN = range(7)
MG_C128, MG_C64, MG_F16, MG_BF16 = range(4)
STATUS_NAMES = {0: "MG_OK", 1: "MG_EINVAL", 2: "MG_ENOMEM", 3: "MG_ECUDA", 4: "MG_ENOCONV",
                5: "MG_ETIMEOUT", 6: "MG_ENAN"}


class MgParams(C.Structure):
    _fields_ = [
        ("dims", C.c_int * 4),
        ("block", C.c_int * 4),
        ("kappa", C.c_double),
        ("hop_weight", C.c_double * 4),
        ("bc_phase", C.c_int * 4),
        ("k", C.c_int),
        ("r", C.c_int),
        ("n_s", C.c_int),
        ("sweeps", C.c_int),
        ("seed", C.c_ulonglong),
        ("setup_dtype", C.c_int),
        ("solve_dtype", C.c_int),
        ("post_smooth", C.c_int),
        ("coarse_tol", C.c_double),
        ("coarse_restart", C.c_int),
        ("coarse_maxiter", C.c_int),
        ("outer_restart", C.c_int),
        ("inner_tol", C.c_double),
        ("svd_refine", C.c_int),
        ("coarse_persistent", C.c_int),
        ("fp64_emulation", C.c_int),
        ("link_compress", C.c_int),
        ("csw", C.c_double),
        ("schur_smoother", C.c_int),
    ]


class MgSolveInfo(C.Structure):
    _fields_ = [
        ("outer_iterations", C.c_int),
        ("refinements", C.c_int),
        ("kcycles", C.c_int),
        ("coarse_iterations", C.c_longlong),
        ("true_residual", C.c_double),
    ]


# exported symbol -> (restype, argtypes)
P = C.c_void_p
I = C.c_int
D = C.c_double
SIGNATURES = {
    "mg_params_default": (None, [C.POINTER(MgParams)]),
    "mg_last_error": (C.c_char_p, []),
    "mg_kernel_launches": (C.c_longlong, []),
    "mg_autotune_report": (C.c_char_p, []),
    "mg_selftest_barrier_timeout": (I, [P]),
    "mg_probe_fma_peak": (I, [I, P, P]),
    "mg_profile_enable": (I, [I, I]),
    "mg_profile_report": (C.c_char_p, []),
    "wilson_dslash": (I, [P, P, P, C.POINTER(C.c_int), D, C.POINTER(C.c_double),
                          C.POINTER(C.c_int), I, I, I, I, P]),
    "wilson_schur": (I, [P, P, P, C.POINTER(C.c_int), D, C.POINTER(C.c_double),
                         C.POINTER(C.c_int), I, I, I, P]),
    "wilson_clover_field": (I, [P, P, C.POINTER(C.c_int), D, D, P]),
    "wilson_clover_apply": (I, [P, P, P, P, C.POINTER(C.c_int), D, C.POINTER(C.c_double),
                                C.POINTER(C.c_int), I, I, I, P]),
    "mg_setup_streaming_svd": (I, [C.POINTER(P), P, C.POINTER(MgParams), P]),
    "mg_setup_from_vectors": (I, [C.POINTER(P), P, C.POINTER(MgParams), P, I, I, P]),
    "mg_link_rows": (I, [P]),
    "mg_setup_ls": (I, [C.POINTER(P), P, C.POINTER(MgParams), P, P]),
    "mg_add_level": (I, [P, C.POINTER(C.c_int), I, I, I, D, P]),
    "mg_num_levels": (I, [P]),
    "mg_level_iterations": (I, [P, C.POINTER(C.c_longlong), I]),
    "mg_get_level": (I, [P, I, P, P, P, P, P]),
    "mg_create": (I, [C.POINTER(P), P, C.POINTER(MgParams), P]),
    "coarse_build": (I, [P, P]),
    "coarse_build_noalloc": (I, [P, P]),
    "mg_solve": (I, [P, P, P, I, D, I, C.POINTER(MgSolveInfo), P]),
    "mg_solve_adjoint": (I, [P, P, P, I, D, I, C.POINTER(MgSolveInfo), P]),
    "mg_destroy": (I, [P]),
    "mg_test_vectors": (I, [P, P, C.POINTER(MgParams), I, P]),
    "mg_get_prolongator": (I, [P, P, P, P]),
    "mg_apply_fine": (I, [P, P, P, I, I, I, P]),
    "mg_get_sigma_history": (I, [P, P, P]),
    "mg_set_prolongator": (I, [P, P, P]),
    "mg_restrict": (I, [P, P, P, I, P]),
    "mg_prolong": (I, [P, P, P, I, P]),
    "mg_get_coarse_op": (I, [P, P, P, P]),
    "mg_coarse_apply": (I, [P, P, P, I, I, P]),
    "wilson_link_gradient": (I, [P, P, P, P, C.POINTER(C.c_int), D, C.POINTER(C.c_double),
                                 C.POINTER(C.c_int), P]),
}

_lib = None


class MgError(RuntimeError):
    def __init__(self, status, where, msg):
        self.status = status
        super().__init__("%s failed with %s: %s" % (where, STATUS_NAMES.get(status, status), msg))


def lib():
    """Load libwilsonmg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libwilsonmg.so is not built (run __graft_entry__.build() or "
                               "python -m paper_2505_14399_gb300._build); no CPU fallback exists")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status, where):
    if status != MG_OK:
        raise MgError(status, where, lib().mg_last_error().decode())
    return status


def ivec(v):
    return (C.c_int * 4)(*[int(x) for x in v])


def dvec(v):
    return (C.c_double * 4)(*[float(x) for x in v])
