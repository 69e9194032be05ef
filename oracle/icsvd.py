"""Test vectors, chiral split and the streaming chiral SVD, FP64 oracle (test infrastructure only).

* Test vectors (Eq. 2, Sec. 2.1; Algorithm 3 first inner loop): psi = phi + psi' where
  psi' is ``sweeps`` steps of GMRES on D psi' = -D phi from zero (the smoother of Sec. 4)
  and phi is a complex-Gaussian Philox field (``oracle.philox``).  Stream s draws the
  global vector ids s*r .. s*r + r - 1.
* Chiral split (Eq. 3): chirality alpha = 0 takes spins 1,2 and alpha = 1 spins 3,4,
  restricted to each aggregate Lambda_j.  The rows of the tile of block j, chirality
  alpha are ordered (local site, spin within the chirality, colour), 6 n_d rows, with
  the local site lexicographic inside the block.
* iCSVD (Algorithm 3, Eqs. 7-8): Phi_{-1} is empty; for every stream the tile
  A = [Phi_{s-1} | Psi_s] gets a dense SVD (numpy/LAPACK), kk = min(k, cols) columns
  are kept as Phi_s = U_kk Sigma_kk; after the last stream U_k is the prolongator block
  of Eq. (6).  All blocks and both chiralities are updated in every stream (the loop
  nesting of Algorithm 3 read that way).
* Least-squares interpolation (Eq. 9): P_j = V_f Omega V_c^dag (V_c Omega V_c^dag)^{-1} with
  V_c = Sigma_k V_k^dag; the weights Omega (positive, one per test vector) are an input.
* Canonical phase (library convention; singular vectors are only defined up to a phase):
  every kept column u is multiplied by conj(q)/|q| with q = sum of its entries, so
  that the sum of its entries is real and positive.
"""
import numpy as np

from . import wilson
from .krylov import gmres_fixed
from .philox import gaussian_vectors


def block_geometry(dims, block):
    """Per fine site: (coarse site index, local site index); plus coarse dims and n_d."""
    c = wilson.coords(dims)
    b = np.asarray(block)
    cd = [dims[m] // block[m] for m in range(4)]
    cc = c // b
    lc = c % b
    coarse = cc[:, 0] + cd[0] * (cc[:, 1] + cd[1] * (cc[:, 2] + cd[2] * cc[:, 3]))
    local = lc[:, 0] + block[0] * (lc[:, 1] + block[1] * (lc[:, 2] + block[2] * lc[:, 3]))
    nd = int(np.prod(block))
    return coarse, local, cd, nd


def smooth(phi, links, dims, kappa, w, bc, sweeps, clover=None):
    """psi = phi + GMRES_sweeps(D, -D phi, x0 = 0)  (Eq. 2); D = D_W + C with a clover term
    C (V, 12, 12) when given."""
    if clover is None:
        A = lambda v: wilson.dslash(v, links, dims, kappa, w, bc).reshape(-1)
    else:
        from . import clover as _cl
        A = lambda v: _cl.dslash(v, links, dims, kappa, 0.0, w, bc, C=clover).reshape(-1)
    b = -A(phi.reshape(-1))
    return phi.reshape(-1) + gmres_fixed(A, b, sweeps)


def test_vectors(links, dims, kappa, w, bc, seed, r, stream, sweeps, clover=None):
    """The r smoothed test vectors of one stream, shape (r, V, 4, 3)."""
    V = wilson.volume(dims)
    ids = np.arange(stream * r, stream * r + r)
    phis = gaussian_vectors(seed, ids, V)
    return np.stack([smooth(phis[i], links, dims, kappa, w, bc, sweeps, clover).reshape(V, 4, 3)
                     for i in range(r)])


def chiral_split(vectors, dims, block):
    """Eq. 3 + blocking: (m, V, 4, 3) -> tiles (d, 2, 6 n_d, m)."""
    coarse, local, cd, nd = block_geometry(dims, block)
    d = int(np.prod(cd))
    m = vectors.shape[0]
    T = np.zeros((d, 2, nd, 2, 3, m), dtype=np.complex128)
    for a in range(2):
        # (m, V, 2, 3) -> (V, 2, 3, m)
        part = np.moveaxis(vectors[:, :, 2 * a:2 * a + 2, :], 0, -1)
        T[coarse, a, local] = part
    return T.reshape(d, 2, 6 * nd, m)


def canonical_phase(U):
    """Make the entry sum of every column real positive."""
    q = U.sum(axis=0)
    ph = np.where(np.abs(q) > 0, np.conj(q) / np.where(np.abs(q) > 0, np.abs(q), 1), 1)
    return U * ph[None, :]


def rank_k_svd(A, k):
    """Best rank-k factors of A (Sec. 3): U_kk, Sigma_kk with kk = min(k, cols)."""
    U, S, _ = np.linalg.svd(A, full_matrices=False)
    kk = min(k, A.shape[1])
    return U[:, :kk], S[:kk]


def icsvd_tiles(stream_tiles, k):
    """Algorithm 3 on precomputed chirally split tiles.

    stream_tiles: list over streams of arrays (d, 2, 6 n_d, r).
    Returns (P tiles (d, 2, 6 n_d, kk) canonicalised, Sigma (d, 2, kk),
    per-stream singular values list of (d, 2, kk)).
    """
    d, _, rows, _ = stream_tiles[0].shape
    Phi = [[np.zeros((rows, 0), dtype=np.complex128) for _ in range(2)] for _ in range(d)]
    hist = []
    n_s = len(stream_tiles)
    Pt = None
    Sig = None
    for s in range(n_s):
        kk = min(k, Phi[0][0].shape[1] + stream_tiles[s].shape[3])
        Sig_s = np.zeros((d, 2, kk))
        if s == n_s - 1:
            Pt = np.zeros((d, 2, rows, kk), dtype=np.complex128)
        for j in range(d):
            for a in range(2):
                A = np.concatenate([Phi[j][a], stream_tiles[s][j, a]], axis=1)
                Uk, Sk = rank_k_svd(A, k)
                Sig_s[j, a] = Sk
                if s == n_s - 1:
                    Pt[j, a] = canonical_phase(Uk)
                else:
                    Phi[j][a] = Uk * Sk[None, :]
        hist.append(Sig_s)
        Sig = Sig_s
    return Pt, Sig, hist


def ls_prolongator_tiles(tiles, k, omega):
    """Least-squares interpolation (Eq. 9, Sec. 5) on every tile (d, 2, rows, m) of m test
    vectors: P_j = V_f Omega V_c^dag (V_c Omega V_c^dag)^{-1} with V_f the tile, V_c =
    Sigma_k V_k^dag from its SVD, Omega = diag(omega) (m positive weights, the same on every
    tile).  Columns get the canonical phase (the SVD fixes V_k only up to a phase per column,
    which P inherits).  Omega = I gives U_k.  Returns (P tiles (d, 2, rows, k), Sigma_k)."""
    d, _, rows, m = tiles.shape
    Om = np.diag(np.asarray(omega, dtype=np.float64))
    P = np.zeros((d, 2, rows, k), dtype=np.complex128)
    S = np.zeros((d, 2, k))
    for j in range(d):
        for a in range(2):
            Vf = tiles[j, a]
            _, s, Vh = np.linalg.svd(Vf, full_matrices=False)
            Vc = np.diag(s[:k]) @ Vh[:k]
            Pj = Vf @ Om @ Vc.conj().T @ np.linalg.inv(Vc @ Om @ Vc.conj().T)
            P[j, a] = canonical_phase(Pj)
            S[j, a] = s[:k]
    return P, S


def icsvd(links, dims, kappa, w, bc, block, k, r, n_s, sweeps, seed, clover=None):
    """Algorithm 3 end to end: smooth, split, stream. Returns (P tiles, Sigma, history)."""
    tiles = []
    for s in range(n_s):
        vecs = test_vectors(links, dims, kappa, w, bc, seed, r, s, sweeps, clover)
        tiles.append(chiral_split(vecs, dims, block))
    return icsvd_tiles(tiles, k)


def dense_prolongator(Pt, dims, block):
    """Eq. 6 as a dense n x 2kd matrix; columns ordered (coarse site, alpha, i)."""
    coarse, local, cd, nd = block_geometry(dims, block)
    d, _, rows, k = Pt.shape
    V = wilson.volume(dims)
    P = np.zeros((V, 4, 3, d, 2, k), dtype=np.complex128)
    T = Pt.reshape(d, 2, nd, 2, 3, k)
    for a in range(2):
        # P[x, 2a+sp, c, coarse(x), a, :] = T[coarse(x), a, local(x), sp, c, :]
        P[np.arange(V), 2 * a:2 * a + 2, :, coarse, a, :] = T[coarse, a, local]
    return P.reshape(12 * V, d * 2 * k)
