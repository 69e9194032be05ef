"""Wilson-clover (Sheikholeslami-Wohlert) term, FP64 oracle (test infrastructure only).

Configuration B of Sec. 4 uses a clover-improved Wilson action whose term the paper does not
write.  This module takes the textbook form, in the conventions of ``oracle.wilson``:

    D_clover = D_W - kappa c_sw sum_{mu < nu} sigma_mu_nu (x) F_mu_nu(x)     (site-local)

* sigma_mu_nu = (i/2) [gamma_mu, gamma_nu]  (Hermitian; commutes with gamma_5, so the term
  is block diagonal in the chirality: two 6 x 6 Hermitian blocks per site);
* F_mu_nu(x) = traceless part of (Q_mu_nu(x) - Q_mu_nu(x)^dag) / (8 i), with Q_mu_nu(x)
  the sum of the four plaquettes of the mu-nu plane that start and end at x, each taken
  counter-clockwise (mu first, then nu):
    U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
  + U_nu(x) U_mu(x+nu-mu)^dag U_nu(x-mu)^dag U_mu(x-mu)
  + U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
  + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag;
* the gauge field is periodic: the fermion boundary phases do not enter F.
"""
import numpy as np

from . import wilson

PAIRS = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def sigma(mu, nu):
    g = wilson.GAMMA
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def _at(field, dims, shifts):
    """field(x + sum_s sign_s e_{mu_s}) for shifts = [(mu, sign), ...] (periodic)."""
    out = field
    for mu, sgn in shifts:
        out = wilson._shift(out, dims, mu, sgn, (1, 1, 1, 1))
    return out


def field_strength(links, dims):
    """F[p] for the plane PAIRS[p], shape (6, V, 3, 3), Hermitian and traceless."""
    V = wilson.volume(dims)
    F = np.zeros((6, V, 3, 3), dtype=np.complex128)
    for p, (mu, nu) in enumerate(PAIRS):
        Um, Un = links[mu], links[nu]
        l1 = Um @ _at(Un, dims, [(mu, 1)]) @ _dag(_at(Um, dims, [(nu, 1)])) @ _dag(Un)
        l2 = (Un @ _dag(_at(Um, dims, [(nu, 1), (mu, -1)])) @ _dag(_at(Un, dims, [(mu, -1)]))
              @ _at(Um, dims, [(mu, -1)]))
        l3 = (_dag(_at(Um, dims, [(mu, -1)])) @ _dag(_at(Un, dims, [(mu, -1), (nu, -1)]))
              @ _at(Um, dims, [(mu, -1), (nu, -1)]) @ _at(Un, dims, [(nu, -1)]))
        l4 = (_dag(_at(Un, dims, [(nu, -1)])) @ _at(Um, dims, [(nu, -1)])
              @ _at(Un, dims, [(nu, -1), (mu, 1)]) @ _dag(Um))
        Q = l1 + l2 + l3 + l4
        f = (Q - _dag(Q)) / 8j
        tr = np.trace(f, axis1=1, axis2=2)
        F[p] = f - (tr / 3.0)[:, None, None] * np.eye(3)
    return F


def clover_term(links, dims, kappa, csw):
    """C(x) = -kappa c_sw sum_{mu<nu} sigma_mu_nu (x) F_mu_nu(x): (V, 12, 12), rows 3 spin + colour."""
    F = field_strength(links, dims)
    V = wilson.volume(dims)
    C = np.zeros((V, 4, 3, 4, 3), dtype=np.complex128)
    for p, (mu, nu) in enumerate(PAIRS):
        C += np.einsum('st,xab->xsatb', sigma(mu, nu), F[p])
    return (-kappa * csw) * C.reshape(V, 12, 12)


def dslash(psi, links, dims, kappa, csw, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1),
           dagger=False, C=None):
    """D_clover psi (dagger: D_clover^dag psi; the clover term is Hermitian)."""
    if C is None:
        C = clover_term(links, dims, kappa, csw)
    psi = np.asarray(psi, dtype=np.complex128).reshape(-1, 4, 3)
    out = wilson.dslash(psi, links, dims, kappa, hop_weight, bc, dagger)
    return out + np.einsum('xrc,xc->xr', C, psi.reshape(-1, 12)).reshape(-1, 4, 3)


def dense_dirac(links, dims, kappa, csw, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1)):
    """Dense 12V x 12V matrix of D_clover (tiny lattices only)."""
    C = clover_term(links, dims, kappa, csw)
    n = 12 * wilson.volume(dims)
    M = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = dslash(e, links, dims, kappa, csw, hop_weight, bc, C=C).reshape(-1)
    return M
