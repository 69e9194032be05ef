"""Seeded synthetic inputs shared by the GPU library's tests/bench and the CPU oracle.

This module synthesises INPUTS only (gauge links, right-hand sides, workload
parameters); it holds none of the method's arithmetic.  The paper's gauge ensembles
(Sec. 4: an anisotropic 32^3 x 256 lattice and an isotropic 32^3 x 64 clover-on-HISQ
lattice) are not available, so lattices of their shapes are synthesised:

* ``haar_links``: per link, the QR factor Q of a complex-Gaussian 3x3 matrix with the
  phases of diag(R) moved into Q (Mezzadri, "How to generate random matrices from the
  classical compact groups", 2007) -- Haar on U(3) -- divided by the principal cube
  root of its determinant (det = 1, SU(3)).
* ``smooth_links``: U = exp(i eps H) with H = (A + A^dag)/2 minus its trace/3 and A
  complex Gaussian; the exponential is taken through the Hermitian eigendecomposition.
  eps = 0.3 gives links near the identity, a stand-in for smeared ensembles.
* ``gaussian_rhs``: complex-Gaussian sources (real, imaginary parts N(0, 1)).

All generators use numpy's PCG64 seeded explicitly; arrays are complex128 in the
library's ABI layouts: links [mu][site][3][3], spinors [site][spin][colour].
"""
import numpy as np


def volume(dims):
    return int(dims[0] * dims[1] * dims[2] * dims[3])


def _cgauss(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def unit_links(dims):
    V = volume(dims)
    return np.broadcast_to(np.eye(3, dtype=np.complex128), (4, V, 3, 3)).copy()


def haar_links(dims, seed):
    rng = np.random.default_rng(seed)
    V = volume(dims)
    A = _cgauss(rng, (4 * V, 3, 3))
    Q, R = np.linalg.qr(A)
    d = np.diagonal(R, axis1=1, axis2=2)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    Q = Q / (det ** (1.0 / 3.0))[:, None, None]
    return Q.reshape(4, V, 3, 3)


def smooth_links(dims, seed, eps=0.3):
    rng = np.random.default_rng(seed)
    V = volume(dims)
    A = _cgauss(rng, (4 * V, 3, 3))
    H = 0.5 * (A + np.conj(np.swapaxes(A, 1, 2)))
    tr = np.trace(H, axis1=1, axis2=2).real / 3.0
    H = H - tr[:, None, None] * np.eye(3)[None]
    lam, vec = np.linalg.eigh(H)
    U = np.einsum('nab,nb,ncb->nac', vec, np.exp(1j * eps * lam), vec.conj())
    return U.reshape(4, V, 3, 3)


def gaussian_rhs(dims, seed, nrhs=1):
    rng = np.random.default_rng(seed)
    V = volume(dims)
    return _cgauss(rng, (nrhs, V, 4, 3))


def graded_fields(dims, m, decades, seed):
    """m complex-Gaussian fields (m, V, 4, 3), field i scaled by 10^(-decades i / (m - 1)):
    stand-in test vectors whose aggregate tiles have singular values spread over `decades`."""
    rng = np.random.default_rng(seed)
    V = volume(dims)
    scale = 10.0 ** (-decades * np.arange(m) / max(m - 1, 1))
    return _cgauss(rng, (m, V, 4, 3)) * scale[:, None, None, None]


# Workload definitions.  Seeds: links 1000+i, sources 2000+i, test vectors 3000+i.
# kappa=None marks a near-critical workload: kappa = kappa_factor * KAPPA_CRIT[name].
WORKLOADS = {
    "c1_4^4_haar": dict(dims=(4, 4, 4, 4), links="haar", link_seed=1000, kappa=0.124,
                        hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1), block=(2, 2, 2, 2),
                        k=4, r=4, n_s=2, sweeps=5, rhs_seed=2000, tv_seed=3000, nrhs=1),
    "c2_16^3x32_near_critical": dict(dims=(16, 16, 16, 32), links="smooth", link_seed=1001,
                                     kappa=None, kappa_factor=0.995,
                                     hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1),
                                     block=(4, 4, 4, 4), k=12, r=8, n_s=4, sweeps=5,
                                     rhs_seed=2001, tv_seed=3001, nrhs=1),
    "c3_16^3x64_aniso": dict(dims=(16, 16, 16, 64), links="smooth", link_seed=1002,
                             kappa=None, kappa_factor=0.98,
                             hop_weight=(1, 1, 1, 1 / 3.5), bc=(1, 1, 1, 1),
                             block=(2, 2, 2, 4), k=24, r=16, n_s=4, sweeps=5,
                             rhs_seed=2002, tv_seed=3002, nrhs=1),
    "c4_32^3x64_12rhs": dict(dims=(32, 32, 32, 64), links="smooth", link_seed=1003,
                             kappa=None, kappa_factor=0.98,
                             hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1),
                             block=(4, 4, 4, 4), k=24, r=24, n_s=2, sweeps=5,
                             rhs_seed=2003, tv_seed=3003, nrhs=12),
    "c5_8^4_autograd": dict(dims=(8, 8, 8, 8), links="smooth", link_seed=1004, kappa=0.12,
                            hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1), block=(2, 2, 2, 2),
                            k=8, r=8, n_s=2, sweeps=5, rhs_seed=2004, tv_seed=3004, nrhs=1),
}


# kappa_crit = 1 / (largest eigenvalue of the Hermitian part of the hopping matrix) on each
# seeded field, a lower bound on the kappa where D turns singular, computed by Lanczos on
# the FP64 oracle's hopping term (python -m oracle.critical_kappa <name>).  The 32^3 x 64
# field is too large for that run; it reuses the 16^3 x 32 value (same link distribution).
KAPPA_CRIT = {
    "c2_16^3x32_near_critical": 0.136551654556,
    "c3_16^3x64_aniso": 0.165482664759,
}
KAPPA_CRIT["c4_32^3x64_12rhs"] = KAPPA_CRIT["c2_16^3x32_near_critical"]


def kappa_of(cfg_or_name):
    """The hopping parameter of a workload (near-critical ones: factor * kappa_crit)."""
    if isinstance(cfg_or_name, str):
        name, cfg = cfg_or_name, WORKLOADS[cfg_or_name]
    else:
        cfg = cfg_or_name
        name = next(n for n, c in WORKLOADS.items() if c["link_seed"] == cfg["link_seed"])
    if cfg.get("kappa") is not None:
        return cfg["kappa"]
    kc = KAPPA_CRIT.get(name)
    if kc is None:
        raise KeyError("kappa_crit of %s has not been computed" % name)
    return cfg["kappa_factor"] * kc


def make_links(cfg):
    if cfg["links"] == "haar":
        return haar_links(cfg["dims"], cfg["link_seed"])
    if cfg["links"] == "unit":
        return unit_links(cfg["dims"])
    return smooth_links(cfg["dims"], cfg["link_seed"])
