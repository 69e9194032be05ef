"""Every launch shape of the stencil (the autotuner's candidates, forced one at a time through
WMG_DSLASH_VARIANT in a child process) against the FP64 oracle: both link layouts, both
directions of the operator, full and single-parity, 2 and 5 right-hand sides (variants 6 and
7 take 2 and 4 per thread, so both leave a ragged last group)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
from oracle import wilson
from paper_2505_14399_gb300 import api, synthetic
dims = (6, 4, 6, 10)
w, bc = (1.0, 1.0, 1.0, 1 / 3.5), (1, 1, 1, -1)
U = synthetic.haar_links(dims, 70)
psi = synthetic.gaussian_rhs(dims, 71, 2)
par = wilson.parity_of_sites(dims)
for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
    Ud = torch.from_numpy(U).to(dt).cuda()
    for dag in (False, True):
        out = api.dslash(torch.from_numpy(psi).to(dt).cuda(), Ud, dims, 0.13, w, bc,
                         dagger=dag).cpu().numpy()
        for r in range(2):
            ref = wilson.dslash(psi[r], U, dims, 0.13, w, bc, dag)
            e = np.linalg.norm(out[r] - ref) / np.linalg.norm(ref)
            assert e < tol, ("full", dt, dag, e)
    half = np.ascontiguousarray(psi[:, par == 0])
    out = api.dslash(torch.from_numpy(half).to(dt).cuda(), Ud, dims, 0.13, w, bc,
                     parity=1).cpu().numpy()
    for r in range(2):
        ref = wilson.dslash_parity(half[r], U, dims, 0.13, 1, w, bc)
        e = np.linalg.norm(out[r] - ref) / np.linalg.norm(ref)
        assert e < tol, ("parity", dt, e)
# the solver's lane-contiguous link copy, five right-hand sides (ragged groups of 2 and 4)
psi5 = synthetic.gaussian_rhs(dims, 72, 5)
p = api.params(dims, (2, 2, 2, 2), 0.13, 4, 4, 1, 1, 1, w, bc)
h = api.Hierarchy(torch.from_numpy(U).cuda(), p, setup=False)
for dt, tol in ((torch.complex128, 1e-12), (torch.complex64, 1e-5)):
    for dag in (False, True):
        out = h.apply_fine(torch.from_numpy(psi5).to(dt).cuda(), dagger=dag).cpu().numpy()
        for r in range(5):
            ref = wilson.dslash(psi5[r], U, dims, 0.13, w, bc, dag)
            e = np.linalg.norm(out[r] - ref) / np.linalg.norm(ref)
            assert e < tol, ("lanes", dt, dag, r, e)
h.close()
print("ok")
"""


@pytest.mark.parametrize("variant", range(8))
def test_forced_launch_shape_matches_oracle(variant):
    env = dict(os.environ, WMG_DSLASH_VARIANT=str(variant), PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
