"""Every launch shape of the smoother's fused stencil + projection kernel (one thread per site
at four register caps), forced one at a time through
WMG_DSLASH_VARIANT in a child process: the mixed-precision K-cycle solve with the post-smoother
on the full system and on the even-odd Schur system reaches a true residual of 1e-10 against
the oracle's operator, with the same outer iteration count (within one) for every shape."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, numpy as np, torch
from oracle import wilson
from paper_2505_14399_gb300 import api, synthetic
cfg = dict(synthetic.WORKLOADS["c5_8^4_autograd"])
U = synthetic.make_links(cfg)
b = synthetic.gaussian_rhs(cfg["dims"], cfg["rhs_seed"], 2)
out = {}
for schur in (0, 1):
    p = api.params(cfg["dims"], cfg["block"], cfg["kappa"], cfg["k"], cfg["r"], cfg["n_s"],
                   cfg["sweeps"], cfg["tv_seed"], cfg["hop_weight"], cfg["bc"],
                   setup_dtype="c64", solve_dtype="c64", schur_smoother=schur)
    h = api.Hierarchy(torch.from_numpy(U).cuda(), p)
    h.coarse_build()
    x, info = h.solve(torch.from_numpy(b).cuda(), tol=1e-10)
    x = x.cpu().numpy()
    for r in range(2):
        res = b[r].reshape(-1) - wilson.dslash(x[r], U, cfg["dims"], cfg["kappa"],
                                               cfg["hop_weight"], cfg["bc"]).reshape(-1)
        e = np.linalg.norm(res) / np.linalg.norm(b[r])
        assert e <= 1e-10, (schur, r, e)
    out[schur] = info["outer"]
    h.close()
print(json.dumps(out))
"""


def _run(variant):
    env = dict(os.environ, WMG_DSLASH_VARIANT=str(variant), PYTHONPATH=ROOT)
    env.pop("WMG_AUTOTUNE_CACHE", None)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_every_fused_shape_solves():
    its = [_run(v) for v in range(4)]
    for schur in ("0", "1"):
        counts = [d[schur] for d in its]
        assert max(counts) - min(counts) <= 1, (schur, counts)
