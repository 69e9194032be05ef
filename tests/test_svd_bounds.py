"""The error bounds of tests/svd_bounds.py, pinned on the CPU against a plain emulation of the
library's Gram route (G = A^dag A, Hermitian eigen-decomposition, A V) in numpy.

The emulation computes G in a chosen precision (FP64, or FP32 as a stand-in for any coarser
arithmetic), so the measured error against the oracle's dense SVD can be set against the bound
for that unit roundoff: it must lie below it, and not absurdly far below (the bound is not
vacuous)."""
import numpy as np
import pytest

from oracle import icsvd
import svd_bounds


def gram_route(stream_tiles, k, gram_dtype, known_diag=False):
    """Algorithm 3 through the Gram matrix, as the library runs it (single pass).  known_diag:
    the Gram block of the kept columns Phi = A V_k is taken as the previous stream's
    eigenvalues (Phi^dag Phi = Lambda_k) instead of being summed, as the double-float route
    does."""
    d, _, rows, _ = stream_tiles[0].shape
    Phi = [[np.zeros((rows, 0), dtype=np.complex128) for _ in range(2)] for _ in range(d)]
    lam_prev = [[None, None] for _ in range(d)]
    hist, P = [], None
    for s, T in enumerate(stream_tiles):
        last = s == len(stream_tiles) - 1
        kk = min(k, Phi[0][0].shape[1] + T.shape[3])
        sig = np.zeros((d, 2, kk))
        if last:
            P = np.zeros((d, 2, kk, rows), dtype=np.complex128)
        for j in range(d):
            for a in range(2):
                A = np.concatenate([Phi[j][a], T[j, a]], axis=1)
                Al = A.astype(gram_dtype)
                G = (Al.conj().T @ Al).astype(np.complex128)
                kd = Phi[j][a].shape[1]
                if known_diag and kd:
                    G[:kd, :kd] = np.diag(lam_prev[j][a])
                lam, V = np.linalg.eigh(G)
                order = np.argsort(-lam, kind="stable")[:kk]
                lam, V = lam[order], V[:, order]
                lam_prev[j][a] = lam
                sig[j, a] = np.sqrt(np.maximum(lam, 0))
                B = A @ V
                if last:
                    U = icsvd.canonical_phase(B / sig[j, a][None, :])
                    P[j, a] = U.T
                else:
                    Phi[j][a] = B
        hist.append(sig)
    return P, hist


def graded_tiles(d, rows, r, n_s, decades, seed):
    rng = np.random.default_rng(seed)
    scale = 10.0 ** (-decades * np.arange(r * n_s) / (r * n_s - 1))
    out = []
    for s in range(n_s):
        g = rng.standard_normal((d, 2, rows, r)) + 1j * rng.standard_normal((d, 2, rows, r))
        out.append(g * scale[s * r:(s + 1) * r][None, None, None, :])
    return out


@pytest.mark.parametrize("known_diag", [False, True])
@pytest.mark.parametrize("gram_dtype,u", [(np.complex128, svd_bounds.U64),
                                          (np.complex64, 2.0 ** -24)])
@pytest.mark.parametrize("decades", [0.0, 2.0, 4.0])
def test_gram_route_within_bound(gram_dtype, u, decades, known_diag):
    k, r, n_s = 6, 5, 3
    tiles = graded_tiles(6, 48, r, n_s, decades, 11)
    P, hist = gram_route(tiles, k, gram_dtype, known_diag)
    Pt, S_o, hist_o = icsvd.icsvd_tiles(tiles, k)
    spectra = svd_bounds.stream_spectra(tiles, k)
    bounds = svd_bounds.arithmetic_bounds(spectra, u, 48)
    ratios = []
    for s in range(n_s):
        bp, bs = bounds[s]
        es = np.abs(hist[s] - hist_o[s]).max(axis=-1)
        assert np.all(es <= bs), (s, (es / bs).max())
        ratios.append((es / bs).max())
    ep = svd_bounds.projector_errors(P, Pt)
    assert np.all(ep <= bounds[-1][0]), (ep / bounds[-1][0]).max()
    ratios.append((ep / bounds[-1][0]).max())
    if gram_dtype == np.complex64:
        # coarse arithmetic reaches the first-order estimate with gamma = u (not M u) within a
        # factor of 10^4 on every result (graded columns keep the Gram rounding relative to the
        # column norms, far inside ||A||_F^2): the bound is not vacuous
        assert 48 * min(ratios) > (1e-4 if decades == 0 else 5e-6), ratios


def test_bound_catches_a_wrong_update():
    """A Gram route that keeps Phi = A V without the stream memory (Phi dropped between
    streams) violates the bound: the bound is tight enough to see method mistakes."""
    k, r, n_s = 6, 5, 3
    tiles = graded_tiles(6, 48, r, n_s, 1.0, 12)
    wrong = [tiles[-1]]
    P, _ = gram_route(wrong, k, np.complex128)
    Pt, _, _ = icsvd.icsvd_tiles(tiles, k)
    bounds = svd_bounds.arithmetic_bounds(svd_bounds.stream_spectra(tiles, k), svd_bounds.U64, 48)
    ep = svd_bounds.projector_errors(P, Pt)
    assert np.all(ep > bounds[-1][0])


def test_vector_bound_covers_perturbed_vectors():
    """Test vectors with a relative error delta (FP32 rounding of every entry plus a scaled
    perturbation) stay within the test-vector bound."""
    k, r, n_s = 6, 5, 3
    tiles = graded_tiles(6, 48, r, n_s, 2.0, 13)
    rng = np.random.default_rng(5)
    delta = 1e-6
    pert = []
    for T in tiles:
        n = rng.standard_normal(T.shape) + 1j * rng.standard_normal(T.shape)
        n *= delta * np.linalg.norm(T, axis=2, keepdims=True) / np.linalg.norm(n, axis=2,
                                                                              keepdims=True)
        pert.append(T + n)
    P, hist = gram_route(pert, k, np.complex128)
    Pt, _, hist_o = icsvd.icsvd_tiles(tiles, k)
    vb = svd_bounds.vector_bounds(svd_bounds.stream_spectra(tiles, k), delta, svd_bounds.U64, 48)
    for s in range(n_s):
        assert np.all(np.abs(hist[s] - hist_o[s]).max(axis=-1) <= vb[s][1])
    assert np.all(svd_bounds.projector_errors(P, Pt) <= vb[-1][0])
