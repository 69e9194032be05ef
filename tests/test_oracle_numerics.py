"""Pins for the oracle's RNG, Krylov solvers, chiral SVD, Galerkin operator, solve and adjoint."""
import os

import numpy as np
import pytest

from oracle import adjoint, coarse, icsvd, krylov, mg, philox, wilson
from paper_2505_14399_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(np.array(v[:4], dtype=np.uint64), v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_gaussian_moments():
    z = philox.gaussian_vectors(12345, np.arange(4), 2048).reshape(-1)
    n = z.size
    for part in (z.real, z.imag):
        assert abs(part.mean()) < 5 / np.sqrt(n)
        assert abs(part.var() - 1) < 6 * np.sqrt(2 / n)
        # fourth moment of N(0,1) is 3
        assert abs((part ** 4).mean() - 3) < 0.15
    assert abs(np.mean(z.real * z.imag)) < 5 / np.sqrt(n)
    # different vector ids and seeds give different streams
    a = philox.gaussian_vectors(1, [0], 16)
    b = philox.gaussian_vectors(1, [1], 16)
    c = philox.gaussian_vectors(2, [0], 16)
    assert not np.allclose(a, b) and not np.allclose(a, c)


# ----------------------------------------------------------------------------- Krylov
def _rand_system(n, seed, shift=4.0):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n) \
        + shift * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b


def test_gmres_full_krylov_is_exact_solve():
    A, b = _rand_system(8, 1)
    x = krylov.gmres_fixed(lambda v: A @ v, b, 8)
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-11


def test_gmres_one_step_is_minimal_residual_step():
    A, b = _rand_system(12, 2)
    x = krylov.gmres_fixed(lambda v: A @ v, b, 1)
    Ab = A @ b
    alpha = np.vdot(Ab, b) / np.vdot(Ab, Ab)
    assert np.abs(x - alpha * b).max() < 1e-13


def test_gmres_minimises_over_krylov_space():
    A, b = _rand_system(30, 3, shift=1.0)
    m = 5
    x = krylov.gmres_fixed(lambda v: A @ v, b, m)
    K = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(m)], axis=1)
    y = np.linalg.lstsq(A @ K, b, rcond=None)[0]
    assert np.abs(x - K @ y).max() < 1e-9 * np.abs(x).max()


def test_gmres_fixed_is_odd_in_the_right_hand_side():
    """GMRES_m(D, -b) = -GMRES_m(D, b) bit for bit (every Arnoldi quantity changes sign or
    not at all, and sign changes are exact), so the test vectors of Eq. 2 equal
    phi - GMRES_m(D, D phi) exactly: the form the library evaluates them in."""
    dims = (4, 4, 4, 4)
    U = synthetic.haar_links(dims, 31)
    phi = synthetic.gaussian_rhs(dims, 32)[0].reshape(-1)
    D = lambda v: wilson.dslash(v, U, dims, 0.125, (1, 1, 1, 1), (1, 1, 1, -1)).reshape(-1)
    Dphi = D(phi)
    for m in (1, 3, 5):
        xp = krylov.gmres_fixed(D, Dphi, m)
        xn = krylov.gmres_fixed(D, -Dphi, m)
        assert np.array_equal(xn, -xp)
        assert np.array_equal(phi + xn, phi - xp)


def test_gmres_tol_and_fgmres():
    A, b = _rand_system(60, 4, shift=2.0)
    x, its, res = krylov.gmres_tol(lambda v: A @ v, b, 1e-10, 10, 500)
    assert res <= 1e-10 and its > 0
    Ainv = np.linalg.inv(A)
    x2, its2, res2 = krylov.fgmres(lambda v: A @ v, lambda v: Ainv @ v, b, 1e-10, 10, 50)
    assert its2 == 1 and res2 < 1e-10
    # identity preconditioner: FGMRES iterates are GMRES iterates
    x3, its3, res3 = krylov.fgmres(lambda v: A @ v, lambda v: v, b, 1e-10, 10, 500)
    assert its3 == its and np.abs(x3 - x).max() < 1e-8


# ----------------------------------------------------------------------------- chiral SVD
def test_chiral_split_places_spins():
    dims, block = (4, 2, 2, 2), (2, 2, 1, 2)
    V = wilson.volume(dims)
    v = np.arange(V * 12, dtype=np.float64).reshape(1, V, 4, 3) + 0j
    T = icsvd.chiral_split(v, dims, block)
    coarse_idx, local, cd, nd = icsvd.block_geometry(dims, block)
    assert T.shape == (int(np.prod(cd)), 2, 6 * nd, 1)
    x = 13
    j, l = coarse_idx[x], local[x]
    for a in range(2):
        for sp in range(2):
            for c in range(3):
                assert T[j, a, (l * 2 + sp) * 3 + c, 0] == v[0, x, 2 * a + sp, c]


def _lowrank_tiles(d, rows, k, r, n_s, seed):
    rng = np.random.default_rng(seed)
    W = rng.standard_normal((d, 2, rows, k)) + 1j * rng.standard_normal((d, 2, rows, k))
    tiles = []
    for s in range(n_s):
        C = rng.standard_normal((d, 2, k, r)) + 1j * rng.standard_normal((d, 2, k, r))
        tiles.append(np.einsum('jarK,jaKc->jarc', W, C))
    return tiles


def test_icsvd_single_stream_is_csvd():
    rng = np.random.default_rng(1)
    t = rng.standard_normal((3, 2, 48, 10)) + 1j * rng.standard_normal((3, 2, 48, 10))
    Pt, S, _ = icsvd.icsvd_tiles([t], 4)
    for j in range(3):
        for a in range(2):
            # independent route: eigen-decomposition of A A^dag
            lam, vec = np.linalg.eigh(t[j, a] @ t[j, a].conj().T)
            assert np.allclose(np.sqrt(lam[::-1][:4]), S[j, a], rtol=1e-12)
            Ptrue = vec[:, ::-1][:, :4]
            assert np.abs(Ptrue @ Ptrue.conj().T - Pt[j, a] @ Pt[j, a].conj().T).max() < 1e-11


def test_icsvd_exact_when_stream_lies_in_rank_k_subspace():
    tiles = _lowrank_tiles(2, 36, 5, 3, 4, 2)
    Pt, S, hist = icsvd.icsvd_tiles(tiles, 5)
    allv = np.concatenate(tiles, axis=3)
    for j in range(2):
        for a in range(2):
            s_all = np.linalg.svd(allv[j, a], compute_uv=False)[:5]
            assert np.allclose(S[j, a], s_all, rtol=1e-11)
            U = np.linalg.svd(allv[j, a])[0][:, :5]
            assert np.abs(U @ U.conj().T - Pt[j, a] @ Pt[j, a].conj().T).max() < 1e-10


def test_icsvd_singular_values_bounded_by_dense_svd():
    rng = np.random.default_rng(3)
    tiles = [rng.standard_normal((2, 2, 30, 4)) + 1j * rng.standard_normal((2, 2, 30, 4))
             for _ in range(4)]
    Pt, S, hist = icsvd.icsvd_tiles(tiles, 6)
    allv = np.concatenate(tiles, axis=3)
    for j in range(2):
        for a in range(2):
            s_all = np.linalg.svd(allv[j, a], compute_uv=False)[:6]
            assert np.all(S[j, a] <= s_all * (1 + 1e-12))
            assert np.abs(Pt[j, a].conj().T @ Pt[j, a] - np.eye(6)).max() < 1e-13
            q = Pt[j, a].sum(axis=0)
            assert np.all(np.abs(q.imag) < 1e-13) and np.all(q.real > 0)
    # stream history: stream 0 keeps min(k, r) = 4 values, later streams k
    assert hist[0].shape[-1] == 4 and hist[1].shape[-1] == 6


def test_icsvd_stream_recursion_and_energy_identity():
    """Stream by stream (Alg. 3, Eqs. 7-8): Phi_s Phi_s^dag is the rank-k spectral truncation
    of A_s A_s^dag = Phi_{s-1} Phi_{s-1}^dag + Psi_s Psi_s^dag, and the energy identity
    ||Phi_final||_F^2 + sum_s sum_{i>k} sigma_i(A_s)^2 = sum_s ||Psi_s||_F^2 holds.

    Phi_s is read off the oracle's public output for the first s + 1 streams (P Sigma); the
    reference route is the Hermitian eigen-decomposition of the Gram matrix, not an SVD."""
    rng = np.random.default_rng(12)
    k, n_s = 5, 4
    tiles = [rng.standard_normal((2, 2, 30, 3 + s)) + 1j * rng.standard_normal((2, 2, 30, 3 + s))
             for s in range(n_s)]
    for j in range(2):
        for a in range(2):
            G_prev = np.zeros((30, 30), dtype=np.complex128)
            lost = 0.0
            for s in range(n_s):
                Pt, S, _ = icsvd.icsvd_tiles(tiles[:s + 1], k)
                Phi = Pt[j, a] * S[j, a][None, :]
                Psi = tiles[s][j, a]
                lam, vec = np.linalg.eigh(G_prev + Psi @ Psi.conj().T)
                lam, vec = lam[::-1], vec[:, ::-1]
                kk = min(k, np.count_nonzero(lam > 1e-9 * lam[0]))
                trunc = (vec[:, :kk] * lam[:kk]) @ vec[:, :kk].conj().T
                G = Phi @ Phi.conj().T
                assert np.abs(G - trunc).max() < 1e-11 * lam[0]
                lost += lam[kk:].clip(min=0).sum()
                G_prev = G
            total = sum(np.vdot(t[j, a], t[j, a]).real for t in tiles)
            assert abs(np.trace(G_prev).real + lost - total) < 1e-11 * total


def test_single_stream_r_equals_k_spans_gram_schmidt_basis():
    """n_s = 1, r = k: the SVD basis spans the same space as block orthonormalisation (Alg. 1)."""
    rng = np.random.default_rng(4)
    t = rng.standard_normal((2, 2, 24, 4)) + 1j * rng.standard_normal((2, 2, 24, 4))
    Pt, S, _ = icsvd.icsvd_tiles([t], 4)
    for j in range(2):
        for a in range(2):
            Q = np.linalg.qr(t[j, a])[0]
            assert np.abs(Q @ Q.conj().T - Pt[j, a] @ Pt[j, a].conj().T).max() < 1e-12


def test_least_squares_interpolation_identity():
    """Eq. 9 with Omega = I, V_f = U_k S_k V_k^dag, V_c = S_k V_k^dag gives P_j = U_k."""
    rng = np.random.default_rng(6)
    A = rng.standard_normal((36, 12)) + 1j * rng.standard_normal((36, 12))
    Pt, S, _ = icsvd.icsvd_tiles([A[None, None].repeat(2, axis=1)], 5)
    Uk = Pt[0, 0]
    # right singular vectors: any orthonormal rows give the same P_j (the identity is algebraic)
    Vk_h = np.linalg.svd(A, full_matrices=False)[2][:5]
    Vf = Uk @ np.diag(S[0, 0]) @ Vk_h
    Vc = np.diag(S[0, 0]) @ Vk_h
    Pj = Vf @ Vc.conj().T @ np.linalg.inv(Vc @ Vc.conj().T)
    assert np.abs(Pj - Uk).max() < 1e-12


def _tiny_setup(dims, block, k, r, n_s, seed=21, kappa=0.12):
    U = synthetic.smooth_links(dims, seed)
    w, bc = (1, 1, 1, 1), (1, 1, 1, -1)
    Pt, S, _ = icsvd.icsvd(U, dims, kappa, w, bc, block, k, r, n_s, 3, 77)
    return U, w, bc, Pt, S


def test_prolongator_is_orthonormal_and_chiral():
    dims, block = (4, 2, 2, 2), (2, 2, 2, 2)
    U, w, bc, Pt, S = _tiny_setup(dims, block, 3, 3, 2)
    P = icsvd.dense_prolongator(Pt, dims, block)
    assert np.abs(P.conj().T @ P - np.eye(P.shape[1])).max() < 1e-13
    V = wilson.volume(dims)
    G5 = np.kron(np.eye(V), np.kron(wilson.GAMMA5, np.eye(3)))
    d = Pt.shape[0]
    sig3 = np.kron(np.eye(d), np.kron(np.diag([1, -1]), np.eye(Pt.shape[3])))
    assert np.abs(G5 @ P - P @ sig3).max() == 0.0


def test_test_vectors_follow_eq2():
    dims = (2, 2, 2, 4)
    U = synthetic.haar_links(dims, 3)
    w, bc = (1, 1, 1, 1), (1, 1, 1, 1)
    tv = icsvd.test_vectors(U, dims, 0.12, w, bc, 99, 2, 1, 4)
    phi = philox.gaussian_vectors(99, [2, 3], wilson.volume(dims))
    D = wilson.dense_dirac(U, dims, 0.12, w, bc)
    for i in range(2):
        p = phi[i].reshape(-1)
        corr = tv[i].reshape(-1) - p
        # psi' is the best 4-step Krylov approximation to -D^{-1} D phi = -phi
        K = np.stack([np.linalg.matrix_power(D, j) @ (-D @ p) for j in range(4)], axis=1)
        y = np.linalg.lstsq(D @ K, -D @ p, rcond=None)[0]
        assert np.abs(corr - K @ y).max() < 1e-8 * np.abs(corr).max()


def test_icsvd_without_truncation_keeps_every_stream():
    """Algorithm 3 with k = n_s r (nothing truncated): the final singular values of each
    chirality's tile are those of all n_s r smoothed test vectors at once (a library SVD of
    vectors built here from their definition: Philox ids 0 .. n_s r - 1, Eq. 2's Krylov
    minimiser by least squares on the dense operator), so every stream's own vectors -- ids
    s r .. s r + r - 1 -- enter the basis."""
    dims, block = (2, 2, 2, 2), (2, 2, 2, 2)          # one aggregate: rows (site, spin, colour)
    U = synthetic.haar_links(dims, 11)
    w, bc, kappa = (1, 1, 1, 1), (1, 1, 1, -1), 0.12
    r, n_s, sweeps, seed = 2, 3, 3, 5
    _, S, _ = icsvd.icsvd(U, dims, kappa, w, bc, block, n_s * r, r, n_s, sweeps, seed)
    V = wilson.volume(dims)
    D = wilson.dense_dirac(U, dims, kappa, w, bc)
    phi = philox.gaussian_vectors(seed, np.arange(n_s * r), V)
    psi = []
    for i in range(n_s * r):
        p = phi[i].reshape(-1)
        K = np.stack([np.linalg.matrix_power(D, j) @ (-D @ p) for j in range(sweeps)], axis=1)
        y = np.linalg.lstsq(D @ K, -D @ p, rcond=None)[0]
        psi.append((p + K @ y).reshape(V, 4, 3))
    psi = np.stack(psi)
    for a in range(2):
        tile = np.moveaxis(psi[:, :, 2 * a:2 * a + 2, :], 0, -1).reshape(6 * V, n_s * r)
        ref = np.linalg.svd(tile, compute_uv=False)
        assert np.abs(S[0, a] - ref).max() < 1e-10 * ref[0]


# ----------------------------------------------------------------------------- Galerkin
@pytest.mark.parametrize("dims,block", [((4, 4, 2, 2), (2, 2, 2, 2)),      # coarse extent 2 and 1
                                        ((6, 2, 2, 4), (2, 2, 1, 2))])     # extent 3, block 1
def test_galerkin_stencil_equals_dense_product(dims, block):
    U, w, bc, Pt, S = _tiny_setup(dims, block, 3, 2, 2)
    kappa = 0.12
    X, Y = coarse.galerkin(Pt, U, dims, block, kappa, w, bc)
    cd = [dims[m] // block[m] for m in range(4)]
    Dc = coarse.dense_coarse(X, Y, cd)
    P = icsvd.dense_prolongator(Pt, dims, block)
    D = wilson.dense_dirac(U, dims, kappa, w, bc)
    ref = P.conj().T @ D @ P
    assert np.abs(Dc - ref).max() < 1e-13
    # sigma_3 D_c sigma_3 = D_c^dag (from gamma_5 P = P sigma_3)
    d, k = Pt.shape[0], Pt.shape[3]
    sig3 = np.kron(np.eye(d), np.kron(np.diag([1, -1]), np.eye(k)))
    assert np.abs(sig3 @ Dc @ sig3 - Dc.conj().T).max() < 1e-13
    # restrict / prolong are P^dag and P; coarse apply is the dense product
    rng = np.random.default_rng(0)
    v = rng.standard_normal(P.shape[0]) + 1j * rng.standard_normal(P.shape[0])
    vc = rng.standard_normal(P.shape[1]) + 1j * rng.standard_normal(P.shape[1])
    assert np.abs(coarse.restrict(Pt, v, dims, block).reshape(-1) - P.conj().T @ v).max() < 1e-13
    assert np.abs(coarse.prolong(Pt, vc, dims, block).reshape(-1) - P @ vc).max() < 1e-13
    assert np.abs(coarse.coarse_apply(X, Y, vc, cd).reshape(-1) - ref @ vc).max() < 1e-12
    rt = coarse.restrict(Pt, coarse.prolong(Pt, vc, dims, block), dims, block).reshape(-1)
    assert np.abs(rt - vc).max() < 1e-13


def test_full_rank_coarse_operator_is_unitarily_equivalent():
    dims, block = (2, 2, 2, 2), (2, 1, 1, 1)        # n_d = 2, 6 n_d = 12 = k
    U = synthetic.haar_links(dims, 5)
    rng = np.random.default_rng(8)
    t = rng.standard_normal((8, 2, 12, 12)) + 1j * rng.standard_normal((8, 2, 12, 12))
    Pt, S, _ = icsvd.icsvd_tiles([t], 12)
    X, Y = coarse.galerkin(Pt, U, dims, block, 0.12)
    Dc = coarse.dense_coarse(X, Y, [1, 2, 2, 2])
    D = wilson.dense_dirac(U, dims, 0.12)
    a = np.sort_complex(np.round(np.linalg.eigvals(Dc), 9))
    b = np.sort_complex(np.round(np.linalg.eigvals(D), 9))
    assert np.abs(a - b).max() < 1e-8


# ----------------------------------------------------------------------------- solve
def test_two_level_solve_matches_direct_solve():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    U = synthetic.haar_links(dims, 1000)
    w, bc, kappa = (1, 1, 1, 1), (1, 1, 1, 1), 0.124
    Pt, S, _ = icsvd.icsvd(U, dims, kappa, w, bc, block, 4, 4, 2, 5, 3000)
    tl = mg.TwoLevel(U, dims, kappa, w, bc, block, Pt)
    b = synthetic.gaussian_rhs(dims, 2000)[0].reshape(-1)
    x, info = tl.solve(b, tol=1e-10)
    D = wilson.dense_dirac(U, dims, kappa, w, bc)
    assert np.linalg.norm(b - D @ x) <= 1e-10 * np.linalg.norm(b)
    xs = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert info['outer'] > 0 and info['coarse'] > 0


def test_kcycle_with_exact_coarse_solve_is_coarse_grid_correction():
    """One K-cycle (Sec. 2.1 end) with the coarse system solved exactly and no post-smoothing
    is the coarse-grid correction P (P^dag D P)^{-1} P^dag v; with a post-smoother that spans
    the whole space it is D^{-1} v; with a full-rank P (k = 6 n_d) the correction alone is
    D^{-1} v and FGMRES stops after one iteration."""
    dims, block = (4, 2, 2, 2), (2, 2, 2, 2)
    U, w, bc, Pt, S = _tiny_setup(dims, block, 3, 3, 2)
    kappa = 0.12
    n = 12 * wilson.volume(dims)
    P = icsvd.dense_prolongator(Pt, dims, block)
    D = wilson.dense_dirac(U, dims, kappa, w, bc)
    rng = np.random.default_rng(14)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    tl = mg.TwoLevel(U, dims, kappa, w, bc, block, Pt, coarse_tol=1e-14, coarse_restart=64,
                     post=0)
    cgc = P @ np.linalg.solve(P.conj().T @ D @ P, P.conj().T @ v)
    assert np.abs(tl.kcycle(v) - cgc).max() < 1e-10 * np.abs(cgc).max()
    tl.post = n
    x = np.linalg.solve(D, v)
    assert np.abs(tl.kcycle(v) - x).max() < 1e-8 * np.abs(x).max()
    # full rank: n_d = 2, k = 12
    dims, block = (2, 2, 2, 2), (2, 1, 1, 1)
    U = synthetic.haar_links(dims, 5)
    t = rng.standard_normal((8, 2, 12, 12)) + 1j * rng.standard_normal((8, 2, 12, 12))
    Pt, S, _ = icsvd.icsvd_tiles([t], 12)
    tl = mg.TwoLevel(U, dims, kappa, (1, 1, 1, 1), (1, 1, 1, 1), block, Pt, coarse_tol=1e-14,
                     coarse_restart=200, post=0)
    D = wilson.dense_dirac(U, dims, kappa)
    v = rng.standard_normal(192) + 1j * rng.standard_normal(192)
    x = np.linalg.solve(D, v)
    assert np.abs(tl.kcycle(v) - x).max() < 1e-10 * np.abs(x).max()
    xs, info = tl.solve(v, tol=1e-10)
    assert info['outer'] == 1 and np.linalg.norm(xs - x) < 1e-9 * np.linalg.norm(x)


# ----------------------------------------------------------------------------- adjoint
def test_adjoint_gradients_match_finite_differences():
    dims = (2, 2, 2, 4)
    U = synthetic.smooth_links(dims, 4)
    w, bc, kappa = (1, 1, 1, 0.5), (1, 1, 1, -1), 0.12
    V = wilson.volume(dims)
    b = synthetic.gaussian_rhs(dims, 5)[0].reshape(-1)

    def loss(links, src):
        D = wilson.dense_dirac(links, dims, kappa, w, bc)
        x = np.linalg.solve(D, src)
        return float(np.vdot(x, x).real), x, D

    L0, x, D = loss(U, b)
    lam2 = np.linalg.solve(D.conj().T, 2 * x)                  # g_b for g_x = 2x
    # gamma_5-hermiticity route for D^{-dag}
    G5 = np.kron(np.eye(V), np.kron(wilson.GAMMA5, np.eye(3)))
    assert np.abs(G5 @ np.linalg.solve(D, G5 @ (2 * x)) - lam2).max() < 1e-12
    rng = np.random.default_rng(6)
    h = 1e-4
    # source gradient: dL = Re(g_b^dag db)
    for _ in range(4):
        db = rng.standard_normal(b.size) + 1j * rng.standard_normal(b.size)
        fd = (loss(U, b + h * db)[0] - loss(U, b - h * db)[0]) / (2 * h)
        assert abs(fd - np.real(np.vdot(lam2, db))) < 1e-6 * max(1, abs(fd))
    # link-angle gradient
    G = adjoint.grad_link_angles(lam2, x, U, dims, kappa, w, bc)
    for _ in range(8):
        om = rng.standard_normal((4, V, 8))
        fd = (loss(adjoint.perturb_links(U, h * om), b)[0]
              - loss(adjoint.perturb_links(U, -h * om), b)[0]) / (2 * h)
        an = float((G * om).sum())
        assert abs(fd - an) < 1e-6 * max(1, abs(fd))


def test_gell_mann_normalisation():
    T = adjoint.T_GEN
    for a in range(8):
        assert np.allclose(T[a], T[a].conj().T) and abs(np.trace(T[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(T[a] @ T[b]) - 0.5 * (a == b)) < 1e-15


def _ls_tiles(seed, m=10, rows=30):
    rng = np.random.default_rng(seed)
    t = rng.standard_normal((2, 2, rows, m)) + 1j * rng.standard_normal((2, 2, rows, m))
    return t * (10.0 ** (-np.arange(m) / (m - 1)))[None, None, None, :]


def test_ls_prolongator_reduces_to_left_singular_vectors():
    """Eq. 9 with Omega = c I (any c > 0) gives U_k: the Omega = I identity of the paper,
    with the weights' scale cancelling."""
    t = _ls_tiles(8)
    Pu, Su, _ = icsvd.icsvd_tiles([t], 4)
    for c in (1.0, 3.7):
        P, S = icsvd.ls_prolongator_tiles(t, 4, c * np.ones(t.shape[3]))
        assert np.abs(P - Pu).max() < 1e-12
        assert np.abs(S - Su).max() < 1e-12


def test_ls_prolongator_minimises_the_weighted_interpolation_error():
    """P_j minimises sum_i omega_i ||v_f,i - P v_c,i||^2: it equals (up to the phase of each
    column, which the canonical phase fixes) the solution of that weighted least-squares problem
    by an independent route (a library least-squares solve of the row-scaled system), and the
    unweighted minimiser differs from it."""
    t = _ls_tiles(9)
    rng = np.random.default_rng(10)
    omega = rng.uniform(0.2, 5.0, t.shape[3])
    P, _ = icsvd.ls_prolongator_tiles(t, 4, omega)
    P1, _ = icsvd.ls_prolongator_tiles(t, 4, np.ones(t.shape[3]))
    w = np.sqrt(omega)
    for j in range(2):
        for a in range(2):
            Vf = t[j, a]
            _, s, Vh = np.linalg.svd(Vf, full_matrices=False)
            Vc = np.diag(s[:4]) @ Vh[:4]
            Q = np.linalg.lstsq((Vc * w[None, :]).T, (Vf * w[None, :]).T, rcond=None)[0].T
            for i in range(4):
                ov = abs(np.vdot(Q[:, i], P[j, a][:, i]))
                assert abs(ov - np.linalg.norm(Q[:, i]) * np.linalg.norm(P[j, a][:, i])) < 1e-10 * ov
                assert abs(np.linalg.norm(Q[:, i]) - np.linalg.norm(P[j, a][:, i])) < 1e-10 * ov ** 0.5
            assert np.abs(P[j, a] - P1[j, a]).max() > 1e-3
