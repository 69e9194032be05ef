"""PyTorch-facing binding of the C ABI (marshalling only; all compute runs in the CUDA library).

Fields are torch tensors in the ABI layouts of include/wilson_mg.h:
spinors (nrhs, V, 4, 3) complex, links (4, V, 3, 3) complex, coarse vectors
(nrhs, d, 2, k) complex.  FP16/BF16 fields are real tensors with a trailing (re, im)
dimension of size 2.  Device tensors are passed by pointer on torch's current CUDA
stream; CPU tensors are staged by the library itself.
"""
import ctypes as C

import numpy as np
import torch

from . import _lib as L

_DT = {torch.complex128: L.MG_C128, torch.complex64: L.MG_C64,
       torch.float16: L.MG_F16, torch.bfloat16: L.MG_BF16}


def _stream(t=None):
    if t is not None and not t.is_cuda:
        return None
    if not torch.cuda.is_available():
        return None
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def params(dims, block, kappa, k, r, n_s, sweeps=5, seed=3000, hop_weight=(1, 1, 1, 1),
           bc=(1, 1, 1, 1), setup_dtype="c64", solve_dtype="c64", post_smooth=8,
           coarse_tol=0.03, coarse_restart=32, coarse_maxiter=2000, outer_restart=16,
           inner_tol=1e-5, svd_refine=-1, coarse_persistent=1, fp64_emulation=-1,
           link_compress=-1, schur_smoother=0, csw=0.0):
    """Build an mg_params structure (paper symbols k, r, n_s; aggregates of extent `block`)."""
    p = L.MgParams()
    L.lib().mg_params_default(C.byref(p))
    dmap = {"c128": L.MG_C128, "c64": L.MG_C64, "f16": L.MG_F16, "bf16": L.MG_BF16}
    p.dims = L.ivec(dims)
    p.block = L.ivec(block)
    p.kappa = float(kappa)
    p.hop_weight = L.dvec(hop_weight)
    p.bc_phase = L.ivec(bc)
    p.k, p.r, p.n_s, p.sweeps = int(k), int(r), int(n_s), int(sweeps)
    p.seed = int(seed)
    p.setup_dtype = dmap[setup_dtype]
    p.solve_dtype = dmap[solve_dtype]
    p.post_smooth = int(post_smooth)
    p.coarse_tol = float(coarse_tol)
    p.coarse_restart = int(coarse_restart)
    p.coarse_maxiter = int(coarse_maxiter)
    p.outer_restart = int(outer_restart)
    p.inner_tol = float(inner_tol)
    p.svd_refine = int(svd_refine)
    p.coarse_persistent = int(coarse_persistent)
    p.fp64_emulation = int(fp64_emulation)
    p.link_compress = int(link_compress)
    p.schur_smoother = int(schur_smoother)
    p.csw = float(csw)
    return p


def dslash(inp, links, dims, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1), parity=-1,
           dagger=False, out=None):
    """out = D in (parity -1) or the single-parity hop term (parity 0/1, half-lattice fields)."""
    dt = _DT[inp.dtype]
    if links.dtype != inp.dtype:
        raise ValueError("links and fields must share a dtype")
    if out is None:
        out = torch.empty_like(inp)
    V = dims[0] * dims[1] * dims[2] * dims[3]
    per = (V if parity < 0 else V // 2) * 12 * (2 if dt >= L.MG_F16 else 1)
    nrhs = inp.numel() // per
    L.check(L.lib().wilson_dslash(_ptr(out), _ptr(inp), _ptr(links), L.ivec(dims), float(kappa),
                                  L.dvec(hop_weight), L.ivec(bc), int(parity), int(dagger), dt,
                                  int(nrhs), _stream(inp)), "wilson_dslash")
    return out


def schur(inp, links, dims, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1), dagger=False,
          out=None):
    """out = D_hat in (even-odd Schur complement) on even half-lattice fields."""
    dt = _DT[inp.dtype]
    if links.dtype != inp.dtype:
        raise ValueError("links and fields must share a dtype")
    if out is None:
        out = torch.empty_like(inp)
    V = dims[0] * dims[1] * dims[2] * dims[3]
    nrhs = inp.numel() // ((V // 2) * 12 * (2 if dt >= L.MG_F16 else 1))
    L.check(L.lib().wilson_schur(_ptr(out), _ptr(inp), _ptr(links), L.ivec(dims), float(kappa),
                                 L.dvec(hop_weight), L.ivec(bc), int(dagger), dt, int(nrhs),
                                 _stream(inp)), "wilson_schur")
    return out


def clover_field(links, dims, kappa, csw):
    """The clover term C(x) as (V, 2, 6, 6) complex128 chiral blocks."""
    V = dims[0] * dims[1] * dims[2] * dims[3]
    out = torch.empty((V, 2, 6, 6), dtype=torch.complex128, device=links.device)
    L.check(L.lib().wilson_clover_field(_ptr(out), _ptr(links), L.ivec(dims), float(kappa),
                                        float(csw), _stream(links)), "wilson_clover_field")
    return out


def clover_dslash(inp, links, clover, dims, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1),
                  dagger=False, out=None):
    """out = (D_W + C) in (dagger: D_W^dag in + C in)."""
    dt = _DT[inp.dtype]
    if links.dtype != inp.dtype or clover.dtype != inp.dtype:
        raise ValueError("links, clover and fields must share a dtype")
    if out is None:
        out = torch.empty_like(inp)
    V = dims[0] * dims[1] * dims[2] * dims[3]
    nrhs = inp.numel() // (V * 12)
    L.check(L.lib().wilson_clover_apply(_ptr(out), _ptr(inp), _ptr(links), _ptr(clover),
                                        L.ivec(dims), float(kappa), L.dvec(hop_weight),
                                        L.ivec(bc), int(dagger), dt, int(nrhs), _stream(inp)),
            "wilson_clover_apply")
    return out


def test_vectors(links, p, stream_index, device=None):
    """The r smoothed test vectors of one stream (Eq. 2), complex128 (r, V, 4, 3)."""
    V = p.dims[0] * p.dims[1] * p.dims[2] * p.dims[3]
    dev = links.device if device is None else device
    out = torch.empty((p.r, V, 4, 3), dtype=torch.complex128, device=dev)
    L.check(L.lib().mg_test_vectors(_ptr(out), _ptr(links), C.byref(p), int(stream_index),
                                    _stream(out)), "mg_test_vectors")
    return out


def link_gradient(g_b, x, links, dims, kappa, hop_weight=(1, 1, 1, 1), bc=(1, 1, 1, 1)):
    V = dims[0] * dims[1] * dims[2] * dims[3]
    out = torch.empty((4, V, 8), dtype=torch.float64, device=x.device)
    L.check(L.lib().wilson_link_gradient(_ptr(out), _ptr(g_b), _ptr(x), _ptr(links), L.ivec(dims),
                                         float(kappa), L.dvec(hop_weight), L.ivec(bc),
                                         _stream(x)), "wilson_link_gradient")
    return out


class Hierarchy:
    """Owner of an mg_handle: iCSVD prolongator, Galerkin coarse operator, K-cycle solver."""

    def __init__(self, links, p, setup=True, vectors=None, smooth=False, ls_omega=None):
        """setup: run the iCSVD setup (Philox test vectors), else only create the handle.
        vectors: (n_s r, V, 4, 3) complex128 / complex64 fields for mg_setup_from_vectors
        (smooth: they are initial guesses phi of Eq. 2, else the test vectors themselves)."""
        self.p = p
        self.dims = tuple(p.dims)
        self.block = tuple(p.block)
        self.k = p.k
        self.V = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        self.nd = self.block[0] * self.block[1] * self.block[2] * self.block[3]
        self.d = self.V // self.nd
        self.device = links.device
        self._h = C.c_void_p()
        if ls_omega is not None:
            w = np.ascontiguousarray(np.asarray(ls_omega, dtype=np.float64))
            L.check(L.lib().mg_setup_ls(C.byref(self._h), _ptr(links), C.byref(p),
                                        C.c_void_p(w.ctypes.data), _stream(links)), "mg_setup_ls")
            return
        if vectors is not None:
            vdt = _DT[vectors.dtype]
            L.check(L.lib().mg_setup_from_vectors(C.byref(self._h), _ptr(links), C.byref(p),
                                                  _ptr(vectors), vdt, int(bool(smooth)),
                                                  _stream(links)), "mg_setup_from_vectors")
            return
        fn = L.lib().mg_setup_streaming_svd if setup else L.lib().mg_create
        L.check(fn(C.byref(self._h), _ptr(links), C.byref(p), _stream(links)),
                "mg_setup_streaming_svd" if setup else "mg_create")

    def close(self):
        if self._h:
            L.lib().mg_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def coarse_build(self):
        L.check(L.lib().coarse_build(self._h, _stream()), "coarse_build")
        self.levels = []          # the library drops levels built on the old operator

    def coarse_build_noalloc(self):
        L.check(L.lib().coarse_build_noalloc(self._h, _stream()), "coarse_build_noalloc")

    def solve(self, b, tol=1e-10, maxiter=1000, adjoint=False, x=None):
        nrhs = b.numel() // (self.V * 12)
        if x is None:
            # a host solution follows the pinning of the host right-hand side, so that the
            # library's device-to-host copy of x runs at the pinned rate
            pin = (not b.is_cuda) and b.is_pinned()
            x = torch.empty(b.shape, dtype=b.dtype, device=b.device, pin_memory=pin)
        info = L.MgSolveInfo()
        fn = L.lib().mg_solve_adjoint if adjoint else L.lib().mg_solve
        L.check(fn(self._h, _ptr(x), _ptr(b), int(nrhs), float(tol), int(maxiter),
                   C.byref(info), _stream(b)), "mg_solve")
        return x, {"outer": info.outer_iterations, "refinements": info.refinements,
                   "kcycles": info.kcycles, "coarse": info.coarse_iterations,
                   "residual": info.true_residual}

    def apply_fine(self, v, dagger=False, out=None):
        """D v with the hierarchy's operator (lane-contiguous link copy)."""
        dt = _DT[v.dtype]
        nrhs = v.numel() // (self.V * 12 * (2 if dt >= L.MG_F16 else 1))
        if out is None:
            out = torch.empty_like(v)
        L.check(L.lib().mg_apply_fine(self._h, _ptr(out), _ptr(v), nrhs, dt, int(dagger),
                                      _stream(v)), "mg_apply_fine")
        return out

    def prolongator(self):
        P = torch.empty((self.d, 2, self.k, 6 * self.nd), dtype=torch.complex128,
                        device=self.device)
        S = torch.empty((self.d, 2, self.k), dtype=torch.float64, device=self.device)
        L.check(L.lib().mg_get_prolongator(self._h, _ptr(P), _ptr(S), _stream(P)),
                "mg_get_prolongator")
        return P, S

    def sigma_history(self):
        H = torch.empty((self.p.n_s, self.d, 2, self.k), dtype=torch.float64, device=self.device)
        L.check(L.lib().mg_get_sigma_history(self._h, _ptr(H), _stream(H)), "mg_get_sigma_history")
        return H

    def set_prolongator(self, P):
        L.check(L.lib().mg_set_prolongator(self._h, _ptr(P), _stream(P)), "mg_set_prolongator")
        self.levels = []

    def restrict(self, v):
        nrhs = v.numel() // (self.V * 12)
        out = torch.empty((nrhs, self.d, 2, self.k), dtype=torch.complex128, device=v.device)
        L.check(L.lib().mg_restrict(self._h, _ptr(out), _ptr(v), nrhs, _stream(v)), "mg_restrict")
        return out

    def prolong(self, vc):
        nrhs = vc.numel() // (self.d * 2 * self.k)
        out = torch.empty((nrhs, self.V, 4, 3), dtype=torch.complex128, device=vc.device)
        L.check(L.lib().mg_prolong(self._h, _ptr(out), _ptr(vc), nrhs, _stream(vc)), "mg_prolong")
        return out

    def coarse_op(self):
        n2k = 2 * self.k
        X = torch.empty((self.d, n2k, n2k), dtype=torch.complex128, device=self.device)
        Y = torch.empty((8, self.d, n2k, n2k), dtype=torch.complex128, device=self.device)
        L.check(L.lib().mg_get_coarse_op(self._h, _ptr(X), _ptr(Y), _stream(X)), "mg_get_coarse_op")
        return X, Y

    def add_level(self, block, k, r, n_s, tol=0.03):
        """One more level below the coarsest (Algorithm 3 + Eq. 5 on the coarse operator)."""
        L.check(L.lib().mg_add_level(self._h, L.ivec(block), int(k), int(r), int(n_s), float(tol),
                                     _stream()), "mg_add_level")
        self.levels = getattr(self, "levels", [])
        prev = self.levels[-1] if self.levels else dict(dims=[self.dims[m] // self.block[m]
                                                              for m in range(4)], k=self.k)
        dims = [prev["dims"][m] // block[m] for m in range(4)]
        self.levels.append(dict(dims=dims, k=int(k), k_in=prev["k"], block=tuple(block),
                                nd=int(np.prod(block))))

    def num_levels(self):
        return L.lib().mg_num_levels(self._h)

    def level_iterations(self):
        n = max(self.num_levels() - 1, 1)
        buf = (C.c_longlong * n)()
        L.check(L.lib().mg_level_iterations(self._h, buf, n), "mg_level_iterations")
        return [int(v) for v in buf]

    def level(self, l):
        """(P tiles (d', 2, k, n_d k_in), sigma (d', 2, k), X (d', 2k, 2k), Y (8, d', 2k, 2k))
        of level l >= 2 (P: from level l - 1 to l; X, Y: the level-l operator)."""
        lv = self.levels[l - 2]
        d = int(np.prod(lv["dims"]))
        k = lv["k"]
        P = torch.empty((d, 2, k, lv["nd"] * lv["k_in"]), dtype=torch.complex128, device=self.device)
        S = torch.empty((d, 2, k), dtype=torch.float64, device=self.device)
        X = torch.empty((d, 2 * k, 2 * k), dtype=torch.complex128, device=self.device)
        Y = torch.empty((8, d, 2 * k, 2 * k), dtype=torch.complex128, device=self.device)
        L.check(L.lib().mg_get_level(self._h, int(l), _ptr(P), _ptr(S), _ptr(X), _ptr(Y),
                                     _stream(P)), "mg_get_level")
        return P, S, X, Y

    def coarse_apply(self, vc):
        dt = _DT[vc.dtype]
        nrhs = vc.numel() // (self.d * 2 * self.k)
        out = torch.empty_like(vc)
        L.check(L.lib().mg_coarse_apply(self._h, _ptr(out), _ptr(vc), nrhs, dt, _stream(vc)),
                "mg_coarse_apply")
        return out


class MGSolve(torch.autograd.Function):
    """x = D^{-1} b through the multigrid solver, differentiable in b and in link angles.

    Forward: mg_solve.  Backward (recomputed, nothing stored but b, x): g_b = D^{-dag} g_x
    via mg_solve_adjoint (gamma_5-hermiticity, D^dag = gamma_5 D gamma_5), and the link-angle
    gradient -Re[g_b^dag dD x] for U_mu(y) -> exp(i omega^a T^a) U_mu(y) at omega = 0.

    omega marks the point of differentiation and must be zero: the hierarchy and the solve
    use the links as given (the rotated links exp(i omega T) U are never formed), so a
    non-zero omega is rejected rather than silently solved at omega = 0.
    """

    @staticmethod
    def forward(ctx, b, omega, hier, links, tol):
        if getattr(getattr(hier, "p", None), "csw", 0.0) != 0.0:
            raise ValueError("MGSolve: link-angle gradients of the clover term are not "
                             "implemented (csw must be 0)")
        if omega is not None and bool(torch.any(omega != 0)):
            raise ValueError("MGSolve: omega must be zero (gradients are taken at the given "
                             "links; rotate the links and rebuild the hierarchy instead)")
        x, _ = hier.solve(b.contiguous(), tol=tol)
        ctx.hier, ctx.links, ctx.tol = hier, links, tol
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, g_x):
        (x,) = ctx.saved_tensors
        h = ctx.hier
        g_b, _ = h.solve(g_x.contiguous(), tol=ctx.tol, adjoint=True)
        g_om = link_gradient(g_b, x, ctx.links, h.dims, h.p.kappa, tuple(h.p.hop_weight),
                             tuple(h.p.bc_phase))
        return g_b, g_om, None, None, None


def mg_solve_autograd(b, omega, hier, links, tol=1e-10):
    return MGSolve.apply(b, omega, hier, links, tol)
