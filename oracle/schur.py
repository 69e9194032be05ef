"""Even-odd (Schur-complement) form of the Wilson-Dirac system, FP64 oracle (test
infrastructure only).

The Wilson-Dirac operator couples only sites of opposite parity through its hopping term,
so with the sites ordered (even, odd) it has the block form

    D = [[1, -kappa H_eo], [-kappa H_oe, 1]]

(H_pq: the hops from parity q to parity p).  Eliminating the odd sites leaves the Schur
complement on the even sites

    D_hat = 1 - kappa^2 H_eo H_oe,

and D x = b is solved as  x_e = D_hat^{-1} (b_e + kappa H_eo b_o),
                          x_o = b_o + kappa H_oe x_e.

The introduction of the paper (Sec. 1) lists even-odd preconditioning among the standard
preconditioners of this system; this module writes the textbook form with the
single-parity hop of ``oracle.wilson``.  Half-lattice
vectors hold the sites of one parity in increasing site order.
"""
import numpy as np

from . import wilson
from .krylov import gmres_tol


def hop(v_half, links, dims, kappa, parity_out, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1),
        dagger=False):
    """-kappa H_{p, 1-p} v (p = parity_out) on half-lattice vectors."""
    return wilson.dslash_parity(v_half, links, dims, kappa, parity_out, hop_weight, bc, dagger)


def schur_op(v_even, links, dims, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1),
             dagger=False):
    """D_hat v = v - kappa^2 H_eo H_oe v on even-site vectors (dagger: D_hat^dag)."""
    v = np.asarray(v_even, dtype=np.complex128).reshape(-1, 4, 3)
    t = hop(v, links, dims, kappa, 1, hop_weight, bc, dagger)
    return v - hop(t, links, dims, kappa, 0, hop_weight, bc, dagger)


def split(v, dims):
    par = wilson.parity_of_sites(dims)
    v = np.asarray(v).reshape(-1, 4, 3)
    return v[par == 0], v[par == 1]


def join(ve, vo, dims):
    par = wilson.parity_of_sites(dims)
    out = np.zeros((wilson.volume(dims), 4, 3), dtype=np.complex128)
    out[par == 0] = np.asarray(ve).reshape(-1, 4, 3)
    out[par == 1] = np.asarray(vo).reshape(-1, 4, 3)
    return out


def prepare(b, links, dims, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1)):
    """Even-site right-hand side b_hat = b_e + kappa H_eo b_o."""
    be, bo = split(b, dims)
    return be - hop(bo, links, dims, kappa, 0, hop_weight, bc)


def reconstruct(x_even, b, links, dims, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1)):
    """Full solution from the even half: x_o = b_o + kappa H_oe x_e."""
    _, bo = split(b, dims)
    xo = bo - hop(x_even, links, dims, kappa, 1, hop_weight, bc)
    return join(x_even, xo, dims)


def solve(b, links, dims, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1), tol=1e-12,
          restart=64, maxiter=5000):
    """D x = b through the Schur complement, with restarted GMRES on D_hat."""
    A = lambda v: schur_op(v, links, dims, kappa, hop_weight, bc).reshape(-1)
    bh = prepare(b, links, dims, kappa, hop_weight, bc).reshape(-1)
    xe, its, _ = gmres_tol(A, bh, tol, restart, maxiter)
    return reconstruct(xe, b, links, dims, kappa, hop_weight, bc), its
