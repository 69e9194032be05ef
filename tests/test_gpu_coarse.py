"""GPU restriction, prolongation, Galerkin coarse operator (Eq. 5) and coarse apply vs the oracle."""
import json

import numpy as np
import pytest
import torch

from oracle import coarse, icsvd
from paper_2505_14399_gb300 import _lib as L, api, synthetic
from gpu_common import orthonormal_tiles, rel, random_tiles, to_dev

pytestmark = pytest.mark.gpu

# (dims, block, k): coarse extents 2 (+mu and -mu neighbours coincide), 1 and 3, ragged k
CASES = [((4, 4, 4, 4), (2, 2, 2, 2), 4),
         ((4, 4, 2, 8), (2, 4, 2, 2), 5),
         ((6, 4, 4, 4), (2, 2, 2, 4), 12)]
# the tensor-pipe contraction's wider instances: 8 < 2k <= 48 with 4-site staging batches, on
# the aggregate shapes of the paper's k = 24 configurations (2x2x2x4 and 4^4, ragged batches)
TC_CASES = CASES + [((4, 4, 4, 4), (2, 2, 2, 2), 14),
                    ((4, 4, 2, 8), (2, 2, 2, 4), 20),
                    ((4, 4, 4, 8), (2, 2, 2, 4), 24),
                    ((8, 8, 4, 8), (4, 4, 4, 4), 24)]


def _handle(dims, block, k, seed, kappa=0.125, w=(1, 1, 1, 1 / 3.5), bc=(1, 1, 1, -1),
            fp64_emulation=0, tiles=random_tiles):
    U = synthetic.smooth_links(dims, seed)
    p = api.params(dims, block, kappa, k, k, 1, hop_weight=w, bc=bc, setup_dtype="c128",
                   solve_dtype="c128", fp64_emulation=fp64_emulation)
    h = api.Hierarchy(to_dev(U), p, setup=False)
    nd = int(np.prod(block))
    d = int(np.prod(dims)) // nd
    P = tiles(d, nd, k, seed + 1)                  # layout [j][alpha][i][row]
    h.set_prolongator(to_dev(P))
    Pt = np.ascontiguousarray(np.swapaxes(P, 2, 3))  # oracle layout [j][alpha][row][i]
    return h, U, Pt, (kappa, w, bc)


@pytest.mark.parametrize("dims,block,k", CASES)
def test_restrict_prolong(dims, block, k):
    h, U, Pt, _ = _handle(dims, block, k, 3)
    rng = np.random.default_rng(4)
    V = int(np.prod(dims))
    v = rng.standard_normal((2, V, 4, 3)) + 1j * rng.standard_normal((2, V, 4, 3))
    vc = h.restrict(to_dev(v)).cpu().numpy()
    for r in range(2):
        assert rel(vc[r].reshape(-1), coarse.restrict(Pt, v[r], dims, block).reshape(-1)) < 1e-13
    ec = rng.standard_normal(vc.shape) + 1j * rng.standard_normal(vc.shape)
    e = h.prolong(to_dev(ec)).cpu().numpy()
    for r in range(2):
        assert rel(e[r], coarse.prolong(Pt, ec[r], dims, block)) < 1e-13
    h.close()


@pytest.mark.parametrize("dims,block,k", TC_CASES)
def test_galerkin_tensor_pipe_contraction(dims, block, k):
    """Double-float Galerkin with an orthonormal prolongator and unitary links: every staged
    entry is inside the fixed-point range, so the forward hops run as exact bf16 digit-plane
    products on the tensor pipe (checked in the launch record); the operator must still match
    the FP64 oracle to double-float accuracy."""
    h, U, Pt, (kappa, w, bc) = _handle(dims, block, k, 9, fp64_emulation=1,
                                       tiles=orthonormal_tiles)
    L.check(L.lib().mg_profile_enable(1, 1000), "mg_profile_enable")
    try:
        h.coarse_build()
        torch.cuda.synchronize()
        kern = json.loads(L.lib().mg_profile_report().decode())
    finally:
        L.lib().mg_profile_enable(0, 0)
    assert kern.get("galerkin_tc", {}).get("launches", 0) == 1, sorted(kern)
    assert "galerkin_df64" not in kern and "galerkin_tc_range_fallback" not in kern
    X, Y = h.coarse_op()
    Xo, Yo = coarse.galerkin(Pt, U, dims, block, kappa, w, bc)
    assert rel(X.cpu().numpy(), Xo) < 1e-11
    assert rel(Y.cpu().numpy(), Yo) < 1e-11
    h.close()


BATCH_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, "tests")
from gpu_common import orthonormal_tiles, rel
from test_gpu_coarse import _handle, CASES
from oracle import coarse
out = []
for dims, block, k in CASES:
    h, U, Pt, (kappa, w, bc) = _handle(dims, block, k, 9, fp64_emulation=1,
                                       tiles=orthonormal_tiles)
    h.coarse_build()
    X, Y = h.coarse_op()
    Xo, Yo = coarse.galerkin(Pt, U, dims, block, kappa, w, bc)
    out.append(max(rel(X.cpu().numpy(), Xo), rel(Y.cpu().numpy(), Yo)))
    h.close()
print(json.dumps(out))
"""


@pytest.mark.parametrize("variant,nb", [(0, 8), (1, 4)])
def test_galerkin_tensor_pipe_batch_sizes(variant, nb):
    """For 2k <= 24 the tensor-pipe kernel has two staging batch sizes (8 sites, one CTA per
    SM; 4 sites, two CTAs per SM), of which the autotuner keeps the faster; each, forced in a
    child process, must match the FP64 oracle to double-float accuracy."""
    import os, subprocess, sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, WMG_DSLASH_VARIANT=str(variant), PYTHONPATH=root)
    env.pop("WMG_AUTOTUNE_CACHE", None)
    r = subprocess.run([sys.executable, "-c", BATCH_CHILD], cwd=root, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    errs = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(errs) == len(CASES) and max(errs) < 1e-11, (nb, errs)


@pytest.mark.parametrize("dims,block,k", CASES)
def test_galerkin_double_float_contraction(dims, block, k):
    """Galerkin contraction in double-float arithmetic on FP32 units vs the FP64 oracle: Gaussian
    tiles have entries beyond the tensor pipe's fixed-point range, so this runs the fallback."""
    h, U, Pt, (kappa, w, bc) = _handle(dims, block, k, 7, fp64_emulation=1)
    h.coarse_build()
    X, Y = h.coarse_op()
    Xo, Yo = coarse.galerkin(Pt, U, dims, block, kappa, w, bc)
    assert rel(X.cpu().numpy(), Xo) < 1e-11
    assert rel(Y.cpu().numpy(), Yo) < 1e-11
    h.close()


@pytest.mark.parametrize("dims,block,k", CASES)
def test_galerkin_and_coarse_apply(dims, block, k):
    h, U, Pt, (kappa, w, bc) = _handle(dims, block, k, 7)
    h.coarse_build()
    X, Y = h.coarse_op()
    Xo, Yo = coarse.galerkin(Pt, U, dims, block, kappa, w, bc)
    assert rel(X.cpu().numpy(), Xo) < 1e-12
    assert rel(Y.cpu().numpy(), Yo) < 1e-12
    cd = [dims[m] // block[m] for m in range(4)]
    rng = np.random.default_rng(8)
    d = Xo.shape[0]
    vc = rng.standard_normal((3, d, 2, k)) + 1j * rng.standard_normal((3, d, 2, k))
    ref = np.stack([coarse.coarse_apply(Xo, Yo, vc[r].reshape(d, -1), cd) for r in range(3)])
    y64 = h.coarse_apply(to_dev(vc)).cpu().numpy().reshape(ref.shape)
    assert rel(y64, ref) < 1e-12
    y32 = h.coarse_apply(to_dev(vc.astype(np.complex64))).cpu().numpy().reshape(ref.shape)
    assert rel(y32, ref) < 1e-5
    h.close()


def test_coarse_operator_symmetry_full_size():
    """sigma_3 D_c sigma_3 = D_c^dag on the SVD prolongator at 16^3 x 32 (holds at any size)."""
    cfg = synthetic.WORKLOADS["c2_16^3x32_near_critical"]
    dims, block, k = cfg["dims"], cfg["block"], cfg["k"]
    U = synthetic.make_links(cfg)
    p = api.params(dims, block, 0.13, k, cfg["r"], cfg["n_s"], cfg["sweeps"], cfg["tv_seed"])
    h = api.Hierarchy(to_dev(U), p)
    P, S = h.prolongator()
    # P^dag P = I per tile, canonical phase, singular values sorted
    Pg = P.cpu().numpy()
    for t in range(0, Pg.shape[0], 37):
        for a in range(2):
            G = Pg[t, a].conj() @ Pg[t, a].T
            assert np.abs(G - np.eye(k)).max() < 1e-10
    Sg = S.cpu().numpy()
    assert np.all(np.diff(Sg, axis=-1) <= 0)
    h.coarse_build()
    X, Y = h.coarse_op()
    X = X.cpu().numpy()
    Y = Y.cpu().numpy()
    s3 = np.diag(np.repeat([1.0, -1.0], k))
    assert np.abs(s3 @ X @ s3 - np.conj(np.swapaxes(X, 1, 2))).max() < 1e-12 * np.abs(X).max()
    nbr = coarse.coarse_neighbours([dims[m] // block[m] for m in range(4)])
    for mu in range(4):
        # Y_{+mu}(j) = sigma_3 Y_{-mu}(j + mu)^dag sigma_3
        lhs = Y[2 * mu]
        rhs = s3 @ np.conj(np.swapaxes(Y[2 * mu + 1][nbr[2 * mu]], 1, 2)) @ s3
        assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(Y).max()
    h.close()
