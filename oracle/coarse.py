"""Restriction, prolongation and the Galerkin coarse operator, FP64 oracle (test infrastructure only).

* R = P^dag (Sec. 2.1, Eq. 4 and the line after it; Algorithm 4).
* Prolongation e = P e_c with P block diagonal over aggregates and chiralities (Eq. 6).
* Galerkin operator D_c = R D P = P^dag D P (Eq. 5).  Because D couples only nearest
  neighbours, D_c couples a coarse site only to itself and its 8 coarse neighbours,
  so it is stored as a stencil: X(j) (self block) and Y_{dir}(j), dir = 2 mu + (0 for +mu,
  1 for -mu), each (2k) x (2k) with rows/columns ordered (alpha, i).  Entry (a, b) of the
  block linking coarse site j to j' is sum_{x in L_j, y in L_j'} P(x)_a^dag D_{x,y} P(y)_b,
  accumulated here term by term over the nonzeros of D:
    - the diagonal 1 of D contributes P(x)^dag P(x) to X(j(x)), and a site-local clover
      term C(x) (``oracle.clover``), when given, P(x)^dag C(x) P(x);
    - the hop x -> x + mu contributes -kappa w_mu P(x)^dag (1 - gamma_mu) U_mu(x) P(x+mu)
      (with bc[mu] when it wraps the lattice) to X if x+mu stays in the aggregate of x
      and to Y_{+mu}(j(x)) otherwise; the hop x -> x - mu likewise with
      (1 + gamma_mu) U_mu(x-mu)^dag and Y_{-mu}.
* Coarse apply: y(j) = X(j) x(j) + sum_mu [Y_{+mu}(j) x(j + mu) + Y_{-mu}(j) x(j - mu)]
  with periodic coarse neighbours.
"""
import numpy as np

from . import wilson
from .icsvd import block_geometry


def site_prolongator(Pt, dims, block):
    """P restricted to each fine site: (V, 12, 2k), rows 3*spin+colour, columns (alpha, i)."""
    coarse, local, cd, nd = block_geometry(dims, block)
    d, _, rows, k = Pt.shape
    V = wilson.volume(dims)
    T = Pt.reshape(d, 2, nd, 2, 3, k)
    Ps = np.zeros((V, 4, 3, 2, k), dtype=np.complex128)
    for a in range(2):
        Ps[:, 2 * a:2 * a + 2, :, a, :] = T[coarse, a, local]
    return Ps.reshape(V, 12, 2 * k)


def restrict(Pt, v, dims, block):
    """e_c = P^dag v, returned as (d, 2k) with (alpha, i) order."""
    coarse, local, cd, nd = block_geometry(dims, block)
    d = Pt.shape[0]
    Ps = site_prolongator(Pt, dims, block)
    v = np.asarray(v).reshape(-1, 12)
    per_site = np.einsum('xra,xr->xa', Ps.conj(), v)
    out = np.zeros((d, Ps.shape[2]), dtype=np.complex128)
    np.add.at(out, coarse, per_site)
    return out


def prolong(Pt, vc, dims, block):
    """e = P e_c; vc (d, 2k) -> (V, 4, 3)."""
    coarse, local, cd, nd = block_geometry(dims, block)
    Ps = site_prolongator(Pt, dims, block)
    vc = np.asarray(vc).reshape(Pt.shape[0], -1)
    return np.einsum('xra,xa->xr', Ps, vc[coarse]).reshape(-1, 4, 3)


def galerkin(Pt, links, dims, block, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1),
             chunk=4096, clover=None):
    """Eq. 5 as a coarse stencil. Returns X (d, 2k, 2k), Y (8, d, 2k, 2k).

    clover: optional site-local term C (V, 12, 12) of D (the Wilson-clover operator)."""
    coarse, local, cd, nd = block_geometry(dims, block)
    d = Pt.shape[0]
    c = wilson.coords(dims)
    Ps = site_prolongator(Pt, dims, block)
    n2k = Ps.shape[2]
    V = wilson.volume(dims)
    X = np.zeros((d, n2k, n2k), dtype=np.complex128)
    Y = np.zeros((8, d, n2k, n2k), dtype=np.complex128)
    eye = np.eye(4, dtype=np.complex128)
    strides = [1, dims[0], dims[0] * dims[1], dims[0] * dims[1] * dims[2]]
    # diagonal of D
    np.add.at(X, coarse, np.einsum('xra,xrb->xab', Ps.conj(), Ps))
    if clover is not None:
        np.add.at(X, coarse, np.einsum('xra,xrs,xsb->xab', Ps.conj(), clover, Ps))
    for mu in range(4):
        for sgn in (+1, -1):
            xm = c[:, mu]
            if sgn > 0:
                wrap = xm == dims[mu] - 1
                nb = np.where(wrap, np.arange(V) - (dims[mu] - 1) * strides[mu],
                              np.arange(V) + strides[mu])
                cross = (xm % block[mu]) == block[mu] - 1
                spin = eye - wilson.GAMMA[mu]
                col = links[mu]                                   # U_mu(x)
            else:
                wrap = xm == 0
                nb = np.where(wrap, np.arange(V) + (dims[mu] - 1) * strides[mu],
                              np.arange(V) - strides[mu])
                cross = (xm % block[mu]) == 0
                spin = eye + wilson.GAMMA[mu]
                col = np.conj(np.swapaxes(links[mu][nb], 1, 2))   # U_mu(x-mu)^dag
            phase = np.where(wrap, float(bc[mu]), 1.0)
            coef = -kappa * hop_weight[mu]
            direction = 2 * mu + (0 if sgn > 0 else 1)
            for s0 in range(0, V, chunk):
                sl = slice(s0, min(V, s0 + chunk))
                Py = Ps[nb[sl]].reshape(-1, 4, 3, n2k)
                B = np.einsum('xab,xsbk->xsak', col[sl], Py)        # colour
                B = np.einsum('st,xtak->xsak', spin, B)             # spin
                B = B.reshape(-1, 12, n2k) * (coef * phase[sl])[:, None, None]
                C = np.einsum('xra,xrb->xab', Ps[sl].conj(), B)
                cr = cross[sl]
                np.add.at(X, coarse[sl][~cr], C[~cr])
                np.add.at(Y[direction], coarse[sl][cr], C[cr])
    return X, Y


def coarse_neighbours(cd):
    """(8, d) index of the coarse neighbour in direction dir = 2 mu + (0: +mu, 1: -mu)."""
    d = int(np.prod(cd))
    j = np.arange(d)
    cc = np.stack([j % cd[0], (j // cd[0]) % cd[1], (j // (cd[0] * cd[1])) % cd[2],
                   j // (cd[0] * cd[1] * cd[2])], axis=1)
    out = np.zeros((8, d), dtype=np.int64)
    for mu in range(4):
        for s, sgn in enumerate((+1, -1)):
            n = cc.copy()
            n[:, mu] = (n[:, mu] + sgn) % cd[mu]
            out[2 * mu + s] = n[:, 0] + cd[0] * (n[:, 1] + cd[1] * (n[:, 2] + cd[2] * n[:, 3]))
    return out


def coarse_apply(X, Y, vc, cd):
    """y(j) = X(j) x(j) + sum_dir Y_dir(j) x(neighbour_dir(j))."""
    vc = np.asarray(vc).reshape(X.shape[0], X.shape[1])
    nbr = coarse_neighbours(cd)
    y = np.einsum('jab,jb->ja', X, vc)
    for dr in range(8):
        y += np.einsum('jab,jb->ja', Y[dr], vc[nbr[dr]])
    return y


def dense_coarse(X, Y, cd):
    """The coarse stencil as a dense (2kd) x (2kd) matrix (tiny lattices only)."""
    d, n2k, _ = X.shape
    M = np.zeros((d, n2k, d, n2k), dtype=np.complex128)
    nbr = coarse_neighbours(cd)
    for j in range(d):
        M[j, :, j, :] += X[j]
        for dr in range(8):
            M[j, :, nbr[dr, j], :] += Y[dr, j]
    return M.reshape(d * n2k, d * n2k)
