"""GPU test vectors (Eq. 2) vs the FP64 oracle; the streaming SVD itself is compared at its
derived bounds in test_gpu_setup_parity.py."""
import numpy as np
import pytest
import torch

from oracle import icsvd, philox, wilson
from paper_2505_14399_gb300 import api, synthetic
from gpu_common import links_for, params_for, rel, to_dev

pytestmark = pytest.mark.gpu

C1 = synthetic.WORKLOADS["c1_4^4_haar"]
C5 = synthetic.WORKLOADS["c5_8^4_autograd"]


@pytest.mark.parametrize("setup_dtype,tol", [("c128", 1e-14), ("c64", 1e-6)])
def test_gaussian_fields_match_philox(setup_dtype, tol):
    """sweeps = 0: psi = phi, the raw Philox complex-Gaussian field (FP64 / FP32 maps)."""
    U = links_for(C5)
    p = params_for(C5, sweeps=0, setup_dtype=setup_dtype)
    for s in range(2):
        tv = api.test_vectors(to_dev(U), p, s).cpu().numpy()
        ref = philox.gaussian_vectors(C5["tv_seed"], np.arange(s * C5["r"], (s + 1) * C5["r"]),
                                      wilson.volume(C5["dims"]))
        assert np.abs(tv - ref).max() < tol * np.abs(ref).max()


@pytest.mark.parametrize("setup_dtype,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_test_vectors(setup_dtype, tol):
    U = links_for(C1)
    p = params_for(C1, setup_dtype=setup_dtype)
    tv = api.test_vectors(to_dev(U), p, 1).cpu().numpy()
    ref = icsvd.test_vectors(U, C1["dims"], C1["kappa"], C1["hop_weight"], C1["bc"], C1["tv_seed"],
                             C1["r"], 1, C1["sweeps"])
    for i in range(C1["r"]):
        assert rel(tv[i], ref[i]) < tol


def test_single_stream_r_equals_k_is_regular_span():
    """n_s = 1, r = k spans the block-orthonormalised test vectors (Algorithm 1)."""
    cfg = dict(C1)
    p = params_for(cfg, n_s=1, r=4, k=4, setup_dtype="c128")
    U = links_for(cfg)
    h = api.Hierarchy(to_dev(U), p)
    P, _ = h.prolongator()
    P = P.cpu().numpy()
    tv = icsvd.test_vectors(U, cfg["dims"], cfg["kappa"], cfg["hop_weight"], cfg["bc"],
                            cfg["tv_seed"], 4, 0, cfg["sweeps"])
    T = icsvd.chiral_split(tv, cfg["dims"], cfg["block"])
    for j in range(P.shape[0]):
        for a in range(2):
            Q = np.linalg.qr(T[j, a])[0]
            Ug = P[j, a].T
            assert np.abs(Q @ Q.conj().T - Ug @ Ug.conj().T).max() < 1e-10
    h.close()
