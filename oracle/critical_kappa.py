"""Near-critical hopping parameter of a seeded synthetic gauge field (input generation helper).

The paper tunes the bare mass to m_crit from a pion-propagator fit on its ensemble
(Sec. 4.5), which cannot be repeated on synthetic links.  The stand-in uses the hopping
matrix H of D = 1 - kappa H: every eigenvalue lambda of H satisfies
Re(lambda) <= mu_max, the largest eigenvalue of the Hermitian part (H + H^dag)/2 (the
field of values of H contains its spectrum).  mu_max comes from Lanczos (ARPACK eigsh,
which='LA') applied to this oracle's H and H^dag, and kappa_crit = 1 / mu_max is a lower
bound on the kappa at which D becomes singular (equal to it on unit links, where H is
normal).  The near-critical workloads use kappa = factor * kappa_crit, so that every
eigenvalue of D has real part >= 1 - factor.

Usage: python -m oracle.critical_kappa <workload name> [tol]
Prints kappa_crit.  Test infrastructure: it calls only this oracle and scipy.
"""
import sys
import time

import numpy as np
from scipy.sparse.linalg import LinearOperator, eigsh

from . import wilson


def hermitian_part_lmax(links, dims, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1), tol=1e-7,
                        ncv=40):
    n = 12 * wilson.volume(dims)

    def mv(v):
        h = wilson.hopping(v, links, dims, hop_weight, bc).reshape(-1)
        hd = wilson.hopping(v, links, dims, hop_weight, bc, dagger=True).reshape(-1)
        return 0.5 * (h + hd)

    op = LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    rng = np.random.default_rng(0)
    v0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    lam = eigsh(op, k=1, which='LA', tol=tol, ncv=ncv, v0=v0, maxiter=5000,
                return_eigenvectors=False)
    return float(lam[0])


def kappa_crit(links, dims, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1), tol=1e-7):
    return 1.0 / hermitian_part_lmax(links, dims, hop_weight, bc, tol)


if __name__ == "__main__":
    sys.path.insert(0, ".")
    from paper_2505_14399_gb300 import synthetic
    name = sys.argv[1]
    tol = float(sys.argv[2]) if len(sys.argv) > 2 else 1e-7
    cfg = synthetic.WORKLOADS[name]
    U = synthetic.make_links(cfg)
    t0 = time.time()
    kc = kappa_crit(U, cfg["dims"], cfg["hop_weight"], cfg["bc"], tol)
    print("%s kappa_crit %.12f (%.0f s)" % (name, kc, time.time() - t0))
