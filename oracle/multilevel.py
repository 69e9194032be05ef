"""Deeper hierarchies, FP64 oracle (test infrastructure only).

Sec. 2.1 (end) and Sec. 4 build the hierarchy recursively: the Galerkin operator of
Eq. (5) takes the place of D on the next level, gamma_5 P = P sigma_3 makes sigma_3 its
chirality, and the setup of Algorithm 3 (test vectors by smoothing, chiral split,
streaming SVD) followed by the Galerkin product of Algorithm 4 gives the level below.
The solve is a K-cycle on every level: FGMRES on level l preconditioned by the K-cycle of
level l + 1, GMRES on the coarsest level, 8 post-smoothing steps (Sec. 4).

A level-l operator (l >= 1) is a nearest-neighbour stencil on its lattice cd: self blocks
X(j) and hop blocks Y_dir(j), dir = 2 mu + (0 for +mu, 1 for -mu), each n x n with
n = 2 k_l, acting on vectors (d, n) whose entries are ordered (alpha, i) with alpha the
chirality (the layout of ``oracle.coarse``).  Aggregates on a coarse lattice are blocks of
its sites, lexicographic inside and across, exactly as on the fine lattice.

Readings (the paper is silent): the random initial guesses of a coarse level are complex
Gaussian Philox fields with counter (site, component, vector id, level); the chiral split
of a coarse level takes, for aggregate J and chirality alpha, the rows (local site, i) of
the alpha half of each site's vector.
"""
import numpy as np

from . import coarse, wilson
from .icsvd import block_geometry, icsvd_tiles
from .krylov import fgmres, gmres_fixed, gmres_tol
from .philox import gaussian_field


def coarse_block_geometry(cd, block):
    """Per coarse-lattice site: (aggregate index, local index); next lattice dims; n_d."""
    return block_geometry(cd, block)


def stencil_operator(X, Y, cd):
    """v -> D_l v for a level-l stencil (flat vectors of length d * n)."""
    return lambda v: coarse.coarse_apply(X, Y, v, cd).reshape(-1)


def test_vectors(X, Y, cd, seed, r, stream, sweeps, level):
    """Eq. 2 on level l: psi = phi + GMRES_sweeps(D_l, -D_l phi, x0 = 0); shape (r, d, n)."""
    d, n = X.shape[0], X.shape[1]
    ids = np.arange(stream * r, stream * r + r)
    phis = gaussian_field(seed, ids, d, n, level)
    A = stencil_operator(X, Y, cd)
    out = []
    for i in range(r):
        phi = phis[i].reshape(-1)
        out.append((phi + gmres_fixed(A, -A(phi), sweeps)).reshape(d, n))
    return np.stack(out)


def chiral_split(vectors, cd, block):
    """Eq. 3 on a coarse level: (m, d, 2k) -> tiles (d', 2, n_d k, m), rows (local site, i)."""
    agg, local, cd2, nd = coarse_block_geometry(cd, block)
    d2 = int(np.prod(cd2))
    m, d, n = vectors.shape
    k = n // 2
    T = np.zeros((d2, 2, nd, k, m), dtype=np.complex128)
    for a in range(2):
        part = np.moveaxis(vectors[:, :, a * k:(a + 1) * k], 0, -1)     # (d, k, m)
        T[agg, a, local] = part
    return T.reshape(d2, 2, nd * k, m)


def site_prolongator(Pt, cd, block, n):
    """P of one coarse level restricted to each of its sites: (d, n, 2 k'), block diagonal in
    the chirality: rows (alpha, i), columns (alpha', i')."""
    agg, local, cd2, nd = coarse_block_geometry(cd, block)
    d = int(np.prod(cd))
    k = n // 2
    d2, _, rows, kp = Pt.shape
    T = Pt.reshape(d2, 2, nd, k, kp)
    Ps = np.zeros((d, 2, k, 2, kp), dtype=np.complex128)
    for a in range(2):
        Ps[:, a, :, a, :] = T[agg, a, local]
    return Ps.reshape(d, n, 2 * kp)


def dense_site_prolongator(Ps, cd, block):
    """The level's P as a dense (d n) x (d' 2k') matrix; columns ordered (aggregate, alpha, i')."""
    agg, local, cd2, nd = coarse_block_geometry(cd, block)
    d, n, m = Ps.shape
    d2 = int(np.prod(cd2))
    P = np.zeros((d, n, d2, m), dtype=np.complex128)
    P[np.arange(d), :, agg, :] = Ps
    return P.reshape(d * n, d2 * m)


def restrict(Ps, v, cd, block):
    """v_c = P^dag v on a coarse level: (d, n) -> (d', 2k')."""
    agg, _, cd2, _ = coarse_block_geometry(cd, block)
    v = np.asarray(v).reshape(Ps.shape[0], Ps.shape[1])
    out = np.zeros((int(np.prod(cd2)), Ps.shape[2]), dtype=np.complex128)
    np.add.at(out, agg, np.einsum('jna,jn->ja', Ps.conj(), v))
    return out


def prolong(Ps, vc, cd, block):
    """e = P e_c on a coarse level: (d', 2k') -> (d, n)."""
    agg, _, _, _ = coarse_block_geometry(cd, block)
    vc = np.asarray(vc).reshape(-1, Ps.shape[2])
    return np.einsum('jna,ja->jn', Ps, vc[agg])


def galerkin(Ps, X, Y, cd, block):
    """Eq. 5 on a coarse level: D_{l+1} = P^dag D_l P as a stencil on the next lattice.

    Term by term over the blocks of the level-l stencil: P(j)^dag X(j) P(j) goes to the
    self block of j's aggregate; P(j)^dag Y_dir(j) P(j + dir) goes to the self block if
    j + dir lies in the same aggregate (the hop does not leave it in direction dir) and to
    the hop block dir of j's aggregate otherwise.
    """
    agg, local, cd2, nd = coarse_block_geometry(cd, block)
    d2 = int(np.prod(cd2))
    m = Ps.shape[2]
    c = wilson.coords(cd)
    nbr = coarse.coarse_neighbours(cd)
    X2 = np.zeros((d2, m, m), dtype=np.complex128)
    Y2 = np.zeros((8, d2, m, m), dtype=np.complex128)
    np.add.at(X2, agg, np.einsum('jna,jnb,jbc->jac', Ps.conj(), X, Ps))
    for mu in range(4):
        for s, sgn in enumerate((+1, -1)):
            dr = 2 * mu + s
            edge = block[mu] - 1 if sgn > 0 else 0
            cross = (c[:, mu] % block[mu]) == edge
            C = np.einsum('jna,jnb,jbc->jac', Ps.conj(), Y[dr], Ps[nbr[dr]])
            np.add.at(X2, agg[~cross], C[~cross])
            np.add.at(Y2[dr], agg[cross], C[cross])
    return X2, Y2


class Hierarchy:
    """Levels 0 (Wilson-Dirac) .. L-1 built with Algorithm 3 + Eq. 5 on every level.

    blocks[l], ks[l], rs[l], n_ss[l]: aggregate shape, kept vectors, stream width and stream
    count of the setup that builds level l + 1 from level l.  P_0 comes from the fine-level
    setup of ``oracle.icsvd``; deeper P_l from this module.  ``Pts`` may supply the tiles of
    every level instead (the setup is then skipped).
    """

    def __init__(self, links, dims, kappa, hop_weight, bc, blocks, ks, rs=None, n_ss=None,
                 sweeps=5, seed=3000, Pts=None, coarse_tol=0.03, coarse_restart=32,
                 coarse_maxiter=1000, post=8, level_tols=None):
        from .icsvd import icsvd
        self.links, self.dims, self.kappa, self.w, self.bc = links, dims, kappa, hop_weight, bc
        self.blocks, self.post = blocks, post
        # relative tolerance of the solve on level l + 1 inside the K-cycle of level l: the
        # paper uses 0.03 on levels 1 and 2, and near the critical mass 0.06 on level 2 and 0.6
        # on level 3 (Sec. 4.5)
        self.level_tols = list(level_tols) if level_tols is not None else [coarse_tol] * len(blocks)
        self.coarse_tol, self.coarse_restart, self.coarse_maxiter = (coarse_tol, coarse_restart,
                                                                     coarse_maxiter)
        nl = len(blocks)
        self.Pt, self.Ps, self.XY, self.cd = [], [], [], []
        lat = list(dims)
        for l in range(nl):
            cdn = [lat[m] // blocks[l][m] for m in range(4)]
            if l == 0:
                Pt = Pts[0] if Pts is not None else icsvd(links, dims, kappa, hop_weight, bc,
                                                          blocks[0], ks[0], rs[0], n_ss[0],
                                                          sweeps, seed)[0]
                self.Pt.append(Pt)
                self.Ps.append(None)
                self.XY.append(coarse.galerkin(Pt, links, dims, blocks[0], kappa, hop_weight, bc))
            else:
                X, Y = self.XY[l - 1]
                if Pts is not None:
                    Pt = Pts[l]
                else:
                    tiles = [chiral_split(test_vectors(X, Y, lat, seed, rs[l], s, sweeps, l),
                                          lat, blocks[l]) for s in range(n_ss[l])]
                    Pt = icsvd_tiles(tiles, ks[l])[0]
                Ps = site_prolongator(Pt, lat, blocks[l], X.shape[1])
                self.Pt.append(Pt)
                self.Ps.append(Ps)
                self.XY.append(galerkin(Ps, X, Y, lat, blocks[l]))
            self.cd.append(lat)
            lat = cdn
        self.cd.append(lat)
        self.coarse_its = 0

    def op(self, l):
        """D_l as a map on flat vectors (level 0: the Wilson-Dirac operator)."""
        if l == 0:
            return lambda v: wilson.dslash(v, self.links, self.dims, self.kappa, self.w,
                                           self.bc).reshape(-1)
        X, Y = self.XY[l - 1]
        return stencil_operator(X, Y, self.cd[l])

    def restrict(self, l, v):
        if l == 0:
            return coarse.restrict(self.Pt[0], v, self.dims, self.blocks[0]).reshape(-1)
        return restrict(self.Ps[l], v, self.cd[l], self.blocks[l]).reshape(-1)

    def prolong(self, l, vc):
        if l == 0:
            return coarse.prolong(self.Pt[0], vc, self.dims, self.blocks[0]).reshape(-1)
        return prolong(self.Ps[l], vc, self.cd[l], self.blocks[l]).reshape(-1)

    def kcycle(self, l, v):
        """K-cycle of level l applied to v: restrict, solve on level l + 1 (recursively
        preconditioned), prolong, post-smooth on level l."""
        v = np.asarray(v, dtype=np.complex128).reshape(-1)
        vc = self.restrict(l, v)
        A = self.op(l + 1)
        tol = self.level_tols[l]
        if l + 1 == len(self.blocks):
            ec, its, _ = gmres_tol(A, vc, tol, self.coarse_restart, self.coarse_maxiter)
        else:
            ec, its, _ = fgmres(A, lambda u: self.kcycle(l + 1, u), vc, tol,
                                self.coarse_restart, self.coarse_maxiter)
        self.coarse_its += its
        e = self.prolong(l, ec)
        D = self.op(l)
        return e + gmres_fixed(D, v - D(e), self.post)

    def solve(self, b, tol=1e-10, restart=16, maxiter=500):
        x, its, res = fgmres(self.op(0), lambda u: self.kcycle(0, u),
                             np.asarray(b).reshape(-1), tol, restart, maxiter)
        return x, {'outer': its, 'coarse': self.coarse_its, 'residual': res}
