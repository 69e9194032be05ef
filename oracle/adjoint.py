"""Adjoint of the solve x = D^{-1} b, FP64 oracle (test infrastructure only).

For a real loss L(x) with x = D^{-1} b (Eq. 1) and g_x = 2 dL/d conj(x) (the complex
gradient convention of torch.autograd), the chain rule gives

    g_b = D^{-dag} g_x,    D^{-dag} = gamma_5 D^{-1} gamma_5   (gamma_5-hermiticity),
    dL  = -Re[ g_b^dag (dD) x ].

Link angles: U_mu(y) -> exp(i sum_a omega^a T^a) U_mu(y), T^a = lambda^a / 2 (Gell-Mann),
so at omega = 0, dU_mu(y) = i T^a U_mu(y) d omega^a and D changes only in the two hops
that use U_mu(y):

    dL/d omega^a_mu(y) = -Re[ g_b(y)^dag (-kappa w_mu)(1 - gamma_mu)(i T^a U_mu(y)) x(y + mu) phi
                            + g_b(y + mu)^dag (-kappa w_mu)(1 + gamma_mu)(i T^a U_mu(y))^dag x(y) phi ]

with phi = bc[mu] when the hop wraps the lattice.  Everything is written with explicit
4x4 gamma and 3x3 Gell-Mann matrices.
"""
import numpy as np

from . import wilson


def gell_mann():
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j
    l[1][1, 0] = 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j
    l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j
    l[6][2, 1] = 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return l


T_GEN = gell_mann() / 2


def grad_source(x, g_x, solve_dag):
    """g_b = D^{-dag} g_x via the supplied solver for D^dag."""
    return solve_dag(g_x)


def grad_link_angles(g_b, x, links, dims, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1)):
    """dL/d omega^a_mu(y), shape (4, V, 8), from g_b = D^{-dag} g_x and x."""
    V = wilson.volume(dims)
    g_b = np.asarray(g_b).reshape(V, 4, 3)
    x = np.asarray(x).reshape(V, 4, 3)
    eye = np.eye(4, dtype=np.complex128)
    c = wilson.coords(dims)
    strides = [1, dims[0], dims[0] * dims[1], dims[0] * dims[1] * dims[2]]
    out = np.zeros((4, V, 8))
    for mu in range(4):
        xm = c[:, mu]
        wrap = xm == dims[mu] - 1
        nb = np.where(wrap, np.arange(V) - (dims[mu] - 1) * strides[mu],
                      np.arange(V) + strides[mu])
        phase = np.where(wrap, float(bc[mu]), 1.0)
        coef = -kappa * hop_weight[mu]
        U = links[mu]
        for a in range(8):
            dU = 1j * np.einsum('ab,xbc->xac', T_GEN[a], U)             # i T^a U
            dUd = np.conj(np.swapaxes(dU, 1, 2))                        # (i T^a U)^dag
            t1 = np.einsum('xab,xsb->xsa', dU, x[nb])
            t1 = np.einsum('st,xtb->xsb', eye - wilson.GAMMA[mu], t1)
            t2 = np.einsum('xab,xsb->xsa', dUd, x)
            t2 = np.einsum('st,xtb->xsb', eye + wilson.GAMMA[mu], t2)
            val = (np.einsum('xsb,xsb->x', g_b.conj(), t1)
                   + np.einsum('xsb,xsb->x', g_b[nb].conj(), t2))
            out[mu, :, a] = -np.real(coef * phase * val)
    return out


def perturb_links(links, omega):
    """U_mu(y) -> exp(i sum_a omega^a T^a) U_mu(y); omega (4, V, 8)."""
    H = np.einsum('myA,Aab->myab', omega, T_GEN)
    lam, vec = np.linalg.eigh(H)
    E = np.einsum('myab,myb,mycb->myac', vec, np.exp(1j * lam), vec.conj())
    return np.einsum('myab,mybc->myac', E, links)
