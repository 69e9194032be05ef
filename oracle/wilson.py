"""Wilson-Dirac operator, FP64 oracle (test infrastructure only).

The paper states the problem as D x = b (Eq. 1) with D the Wilson-Dirac operator
(abstract; Sec. 2.1) and 12 degrees of freedom per site (Sec. 3) but never writes D.
This module writes it out with the conventions the library documents:

    D psi(x) = psi(x) - kappa * sum_mu w_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                                            + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ]

* lattice dims (Lx, Ly, Lz, Lt), mu = 0..3 = x, y, z, t; site index
  s = x + Lx*(y + Ly*(z + Lz*t)); parity (x+y+z+t) mod 2;
* spinor layout [site][spin 4][colour 3] complex; links [mu][site][3][3], U_mu(x)
  connects x to x+mu;
* chiral gamma basis (required by Eq. 3, where spins 1,2 and 3,4 are the two
  chiralities): gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = 1, 2, 3),
  gamma_4 = [[0, 1], [1, 0]], gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1);
* a hop that wraps around the lattice in direction mu is multiplied by bc[mu]
  (+1 periodic, -1 antiperiodic);
* D^dag = gamma_5 D gamma_5 swaps the two projectors.

Everything is numpy complex128, computed with explicit 4x4 gamma matrices and np.roll.
"""
import numpy as np

SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]


def gamma_matrices():
    """Chiral Euclidean basis; returns (gamma[0..3] for mu = x, y, z, t, gamma5)."""
    z = np.zeros((2, 2), dtype=np.complex128)
    one = np.eye(2, dtype=np.complex128)
    g = []
    for k in range(3):
        g.append(np.block([[z, -1j * SIGMA[k]], [1j * SIGMA[k], z]]))
    g.append(np.block([[z, one], [one, z]]))
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


GAMMA, GAMMA5 = gamma_matrices()
# lattice axis of direction mu in the [t][z][y][x] array view
_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def volume(dims):
    return int(dims[0] * dims[1] * dims[2] * dims[3])


def to_grid(v, dims):
    """[site][...] -> [t][z][y][x][...] (pure reshape of the lexicographic order)."""
    Lx, Ly, Lz, Lt = dims
    return v.reshape((Lt, Lz, Ly, Lx) + v.shape[1:])


def from_grid(g, dims):
    return g.reshape((volume(dims),) + g.shape[4:])


def coords(dims):
    """Integer coordinates (V, 4) in site order."""
    Lx, Ly, Lz, Lt = dims
    s = np.arange(volume(dims))
    x = s % Lx
    y = (s // Lx) % Ly
    z = (s // (Lx * Ly)) % Lz
    t = s // (Lx * Ly * Lz)
    return np.stack([x, y, z, t], axis=1)


def parity_of_sites(dims):
    return coords(dims).sum(axis=1) % 2


def _shift(field, dims, mu, direction, bc):
    """field(x + direction*mu) on the grid, with bc[mu] on the wrapped slice."""
    g = to_grid(field, dims)
    ax = _AXIS[mu]
    out = np.roll(g, -direction, axis=ax)
    if bc[mu] != 1:
        sl = [slice(None)] * out.ndim
        # for +mu the wrapped entries land on the last slice, for -mu on the first
        sl[ax] = dims[mu] - 1 if direction > 0 else 0
        out[tuple(sl)] *= bc[mu]
    return from_grid(out, dims)


def hopping(psi, links, dims, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1), dagger=False):
    """H psi = sum_mu w_mu [ (1 -/+ gamma_mu) U_mu(x) psi(x+mu) + (1 +/- gamma_mu) U_mu(x-mu)^dag psi(x-mu) ].

    Upper signs for D, lower for D^dag.  psi: (V, 4, 3); links: (4, V, 3, 3).
    """
    psi = np.asarray(psi, dtype=np.complex128).reshape(volume(dims), 4, 3)
    out = np.zeros_like(psi)
    eye = np.eye(4, dtype=np.complex128)
    sgn = 1.0 if dagger else -1.0
    for mu in range(4):
        U = links[mu]
        fwd = _shift(psi, dims, mu, +1, bc)                       # psi(x+mu)
        up = np.einsum('xab,xsb->xsa', U, fwd)                    # U_mu(x) psi(x+mu)
        out += hop_weight[mu] * np.einsum('st,xtb->xsb', eye + sgn * GAMMA[mu], up)
        Udag_psi = np.einsum('xba,xsb->xsa', U.conj(), psi)       # U_mu(x)^dag psi(x)
        bwd = _shift(Udag_psi, dims, mu, -1, bc)                  # U_mu(x-mu)^dag psi(x-mu)
        out += hop_weight[mu] * np.einsum('st,xtb->xsb', eye - sgn * GAMMA[mu], bwd)
    return out


def dslash(psi, links, dims, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1), dagger=False):
    """D psi (or D^dag psi): psi - kappa * H psi."""
    psi = np.asarray(psi, dtype=np.complex128).reshape(volume(dims), 4, 3)
    return psi - kappa * hopping(psi, links, dims, hop_weight, bc, dagger)


def dslash_parity(psi_half, links, dims, kappa, parity, hop_weight=(1, 1, 1, 1),
                  bc=(1, 1, 1, 1), dagger=False):
    """Single-parity hop: out_p = -kappa * H_{p,1-p} in_{1-p}.

    Half-lattice vectors hold the sites of one parity in increasing full-site order
    (checkerboard index = site // 2 when Lx is even).  Written from the definition:
    embed the input on the opposite parity, apply the full hopping term, read back
    the output parity.
    """
    par = parity_of_sites(dims)
    full = np.zeros((volume(dims), 4, 3), dtype=np.complex128)
    full[par == 1 - parity] = np.asarray(psi_half).reshape(-1, 4, 3)
    h = hopping(full, links, dims, hop_weight, bc, dagger)
    return -kappa * h[par == parity]


def apply_gamma5(psi):
    psi = np.asarray(psi).reshape(-1, 4, 3)
    return np.einsum('st,xtb->xsb', GAMMA5, psi)


def dense_dirac(links, dims, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1), dagger=False):
    """Dense 12V x 12V matrix of D by applying it to unit vectors (tiny lattices only)."""
    n = 12 * volume(dims)
    M = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = dslash(e, links, dims, kappa, hop_weight, bc, dagger).reshape(-1)
    return M


def free_spectrum(dims, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1)):
    """Closed-form eigenvalues of D on unit links (each with multiplicity 6).

    With plane waves exp(i p.x), p_mu = (2 pi n_mu + theta_mu) / L_mu, theta = pi for an
    antiperiodic direction, D becomes 1 - kappa sum_mu w_mu (2 cos p_mu - 2 i gamma_mu sin p_mu)
    in spin space, so its eigenvalues are
    1 - 2 kappa sum w cos p  +/-  2 i kappa sqrt(sum w^2 sin^2 p).
    """
    ps = []
    for mu in range(4):
        th = 0.0 if bc[mu] == 1 else np.pi
        ps.append((2 * np.pi * np.arange(dims[mu]) + th) / dims[mu])
    P = np.meshgrid(*ps, indexing='ij')
    w = np.asarray(hop_weight, dtype=np.float64)
    re = 1 - 2 * kappa * sum(w[m] * np.cos(P[m]) for m in range(4))
    im = 2 * kappa * np.sqrt(sum((w[m] * np.sin(P[m])) ** 2 for m in range(4)))
    lam_p = (re + 1j * im).reshape(-1)
    lam_m = (re - 1j * im).reshape(-1)
    return np.concatenate([np.repeat(lam_p, 6), np.repeat(lam_m, 6)])
