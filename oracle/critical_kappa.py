"""Near-critical hopping parameter of a seeded synthetic gauge field (input generation helper).

The paper tunes the bare mass to m_crit from a pion-propagator fit on its ensemble
(Sec. 4.5), which cannot be repeated on synthetic links.  The stand-in: the rightmost
eigenvalue lambda_max of the hopping matrix H (D = 1 - kappa H) from ARPACK's Arnoldi
(scipy.sparse.linalg.eigs, which='LR') applied to this oracle's H; kappa_crit =
1 / Re lambda_max, at which D becomes singular.  The near-critical workloads use
kappa = factor * kappa_crit.

Usage: python -m oracle.critical_kappa <workload name> [tol]
Prints kappa_crit.  Test infrastructure: it calls only this oracle and scipy.
"""
import sys
import time

import numpy as np
from scipy.sparse.linalg import LinearOperator, eigs

from . import wilson


def kappa_crit(links, dims, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1), tol=1e-8, ncv=48):
    n = 12 * wilson.volume(dims)
    mv = lambda v: wilson.hopping(v, links, dims, hop_weight, bc).reshape(-1)
    op = LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    rng = np.random.default_rng(0)
    v0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    lam = eigs(op, k=2, which='LR', tol=tol, ncv=ncv, v0=v0, maxiter=5000,
               return_eigenvectors=False)
    lmax = lam[np.argmax(lam.real)]
    return 1.0 / lmax.real, lmax


if __name__ == "__main__":
    sys.path.insert(0, ".")
    from paper_2505_14399_gb300 import synthetic
    name = sys.argv[1]
    tol = float(sys.argv[2]) if len(sys.argv) > 2 else 1e-8
    cfg = synthetic.WORKLOADS[name]
    U = synthetic.make_links(cfg)
    t0 = time.time()
    kc, lmax = kappa_crit(U, cfg["dims"], cfg["hop_weight"], cfg["bc"], tol)
    print("%s kappa_crit %.12f lambda_max %s (%.0f s)" % (name, kc, lmax, time.time() - t0))
