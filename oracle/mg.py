"""Two-level K-cycle preconditioned FGMRES solve of D x = b, FP64 oracle (test infrastructure only).

Sec. 2.1 (end) and Sec. 4: the hierarchy is used in a K-cycle as the preconditioner of
a flexible outer solver (FGMRES); FGMRES is also the smoother and the coarse solver; 8
post-smoothing iterations; the coarse system is solved to ||r|| = 0.03 ||b||.  With two
levels one application of the preconditioner to v is:

    v_c = P^dag v                                  (restrict, R = P^dag)
    e_c = GMRES(D_c, v_c) to ||v_c - D_c e_c|| <= coarse_tol ||v_c||
    e   = P e_c                                    (prolong)
    e   = e + GMRES_post(D, v - D e)               (post-smoother, from zero)

Readings the paper leaves open (restart lengths, iteration caps) are parameters.

Wilson-clover operator (``clover=C``, the site-local term of ``oracle.clover``): D = D_W + C
in the solve, the smoother and the Galerkin diagonal.

Schur-form post-smoother (``schur=True``; the introduction lists even-odd preconditioning
among the standard ones, Sec. 1): the post-smoother solves D e = r through the Schur
complement on the even sites, GMRES_post on D_hat r_hat with r_hat = r_e + kappa H_eo r_o,
then e_o = r_o + kappa H_oe e_e (``oracle.schur``).

Parity status: the pieces are pinned individually (Krylov, Dslash, Galerkin); the
solve itself is pinned by the true residual computed with the dense D and by a direct
dense solve on tiny lattices.  Iteration counts of the paper's Tables 1-3 need the
paper's gauge ensembles and stay parity unpinned.
"""
import numpy as np

from . import wilson
from .coarse import coarse_apply, galerkin, prolong, restrict
from .krylov import fgmres, gmres_fixed, gmres_tol
from . import schur as _schur


class TwoLevel:
    def __init__(self, links, dims, kappa, hop_weight, bc, block, Pt, coarse_tol=0.03,
                 coarse_restart=32, coarse_maxiter=1000, post=8, XY=None, schur=False,
                 clover=None):
        self.links, self.dims, self.kappa = links, dims, kappa
        self.w, self.bc, self.block, self.Pt = hop_weight, bc, block, Pt
        self.cd = [dims[m] // block[m] for m in range(4)]
        self.clover = clover
        self.X, self.Y = XY if XY is not None else galerkin(Pt, links, dims, block, kappa,
                                                          hop_weight, bc, clover=clover)
        self.coarse_tol, self.coarse_restart = coarse_tol, coarse_restart
        self.coarse_maxiter, self.post = coarse_maxiter, post
        self.schur = schur
        self.coarse_its = 0
        self.kcycles = 0

    def D(self, v):
        out = wilson.dslash(v, self.links, self.dims, self.kappa, self.w, self.bc).reshape(-1)
        if self.clover is not None:
            out = out + np.einsum('xrc,xc->xr', self.clover,
                                  np.asarray(v).reshape(-1, 12)).reshape(-1)
        return out

    def Dc(self, vc):
        return coarse_apply(self.X, self.Y, vc, self.cd).reshape(-1)

    def kcycle(self, v):
        vc = restrict(self.Pt, v, self.dims, self.block).reshape(-1)
        ec, its, _ = gmres_tol(self.Dc, vc, self.coarse_tol, self.coarse_restart,
                               self.coarse_maxiter)
        self.coarse_its += its
        self.kcycles += 1
        e = prolong(self.Pt, ec, self.dims, self.block).reshape(-1)
        r = np.asarray(v).reshape(-1) - self.D(e)
        return e + self.smooth(r)

    def smooth(self, r):
        """post GMRES steps on D e = r from zero: on D itself, or on the Schur system."""
        if not self.schur:
            return gmres_fixed(self.D, r, self.post)
        a = (self.links, self.dims, self.kappa, self.w, self.bc)
        Dh = lambda u: _schur.schur_op(u, *a).reshape(-1)
        rh = _schur.prepare(r, *a).reshape(-1)
        ee = gmres_fixed(Dh, rh, self.post)
        return _schur.reconstruct(ee, r, *a).reshape(-1)

    def solve(self, b, tol=1e-10, restart=16, maxiter=500):
        x, its, res = fgmres(self.D, self.kcycle, np.asarray(b).reshape(-1), tol, restart,
                             maxiter)
        return x, {'outer': its, 'coarse': self.coarse_its, 'residual': res}
