"""Pins for the oracle's deeper hierarchy (Galerkin product and chiral SVD on a coarse level,
multilevel K-cycle): dense products, sigma_3 hermiticity, spectra, exact solves."""
import numpy as np
import pytest

from oracle import coarse, icsvd, krylov, mg, multilevel, philox, wilson
from paper_2505_14399_gb300 import synthetic


def _fine_level(dims, block1, k1, seed=21, kappa=0.12):
    U = synthetic.smooth_links(dims, seed)
    w, bc = (1, 1, 1, 1), (1, 1, 1, -1)
    Pt, _, _ = icsvd.icsvd(U, dims, kappa, w, bc, block1, k1, k1, 2, 3, 77)
    X, Y = coarse.galerkin(Pt, U, dims, block1, kappa, w, bc)
    cd1 = [dims[m] // block1[m] for m in range(4)]
    return U, w, bc, kappa, Pt, X, Y, cd1


def _random_level_tiles(cd1, block2, k1, k2, seed):
    """Orthonormal, chirally block-diagonal tiles for the level-1 -> level-2 prolongator."""
    _, _, cd2, nd2 = multilevel.coarse_block_geometry(cd1, block2)
    d2 = int(np.prod(cd2))
    rng = np.random.default_rng(seed)
    t = rng.standard_normal((d2, 2, nd2 * k1, k2)) + 1j * rng.standard_normal((d2, 2, nd2 * k1, k2))
    return icsvd.icsvd_tiles([t], k2)[0]


def test_coarse_gaussian_fields():
    z = philox.gaussian_field(99, np.arange(3), 512, 8, 1).reshape(-1)
    n = z.size
    for part in (z.real, z.imag):
        assert abs(part.mean()) < 5 / np.sqrt(n) and abs(part.var() - 1) < 6 * np.sqrt(2 / n)
    # the level word decorrelates levels drawn with the same seed and vector ids
    a = philox.gaussian_field(99, [0], 16, 12, 0).reshape(16, 4, 3)
    assert np.array_equal(a, philox.gaussian_vectors(99, [0], 16)[0])
    assert not np.allclose(a.reshape(-1), philox.gaussian_field(99, [0], 16, 12, 1).reshape(-1))


def test_coarse_chiral_split_places_components():
    cd, block = (4, 2, 2, 2), (2, 1, 2, 1)
    d, k = int(np.prod(cd)), 3
    v = np.arange(d * 2 * k, dtype=np.float64).reshape(1, d, 2 * k) + 0j
    T = multilevel.chiral_split(v, cd, block)
    agg, local, cd2, nd = multilevel.coarse_block_geometry(cd, block)
    assert T.shape == (int(np.prod(cd2)), 2, nd * k, 1)
    for j in (0, 5, 13):
        for a in range(2):
            for i in range(k):
                assert T[agg[j], a, local[j] * k + i, 0] == v[0, j, a * k + i]


CASES = [((6, 2, 2, 4), (2, 2, 1, 2), 3, (1, 1, 2, 1), 4),     # level-1 extent 3 in x
         ((4, 4, 2, 2), (2, 2, 1, 1), 2, (2, 1, 2, 2), 3),     # level-2 lattice (1, 2, 1, 1)
         ((8, 2, 2, 2), (2, 2, 2, 2), 2, (2, 1, 1, 1), 3)]     # aggregates of 2 sites, 2 of them in x


@pytest.mark.parametrize("dims,block1,k1,block2,k2", CASES)
def test_coarse_level_galerkin_equals_dense_product(dims, block1, k1, block2, k2):
    U, w, bc, kappa, Pt, X, Y, cd1 = _fine_level(dims, block1, k1)
    Pt2 = _random_level_tiles(cd1, block2, k1, k2, 5)
    Ps = multilevel.site_prolongator(Pt2, cd1, block2, 2 * k1)
    X2, Y2 = multilevel.galerkin(Ps, X, Y, cd1, block2)
    cd2 = [cd1[m] // block2[m] for m in range(4)]
    D2 = coarse.dense_coarse(X2, Y2, cd2)
    D1 = coarse.dense_coarse(X, Y, cd1)
    P2 = multilevel.dense_site_prolongator(Ps, cd1, block2)
    assert np.abs(P2.conj().T @ P2 - np.eye(P2.shape[1])).max() < 1e-13
    ref = P2.conj().T @ D1 @ P2
    assert np.abs(D2 - ref).max() < 1e-13
    # the composite prolongator P1 P2 against the dense Wilson-Dirac operator
    P1 = icsvd.dense_prolongator(Pt, dims, block1)
    D = wilson.dense_dirac(U, dims, kappa, w, bc)
    P12 = P1 @ P2
    assert np.abs(D2 - P12.conj().T @ D @ P12).max() < 1e-13
    # sigma_3 P2 = P2 sigma_3 (P2 keeps the chirality), so sigma_3 hermiticity carries over
    d1, d2 = int(np.prod(cd1)), int(np.prod(cd2))
    s3_1 = np.kron(np.eye(d1), np.kron(np.diag([1, -1]), np.eye(k1)))
    s3 = np.kron(np.eye(d2), np.kron(np.diag([1, -1]), np.eye(k2)))
    assert np.abs(s3_1 @ P2 - P2 @ s3).max() == 0.0
    assert np.abs(s3 @ D2 @ s3 - D2.conj().T).max() < 1e-13
    # restrict / prolong are P2^dag and P2
    rng = np.random.default_rng(2)
    v = rng.standard_normal(P2.shape[0]) + 1j * rng.standard_normal(P2.shape[0])
    vc = rng.standard_normal(P2.shape[1]) + 1j * rng.standard_normal(P2.shape[1])
    assert np.abs(multilevel.restrict(Ps, v, cd1, block2).reshape(-1) - P2.conj().T @ v).max() < 1e-13
    assert np.abs(multilevel.prolong(Ps, vc, cd1, block2).reshape(-1) - P2 @ vc).max() < 1e-13


def test_full_rank_level_is_unitarily_equivalent():
    dims, block1, k1 = (6, 2, 2, 4), (2, 2, 1, 2), 3
    U, w, bc, kappa, Pt, X, Y, cd1 = _fine_level(dims, block1, k1)
    block2 = (1, 1, 1, 2)                                  # n_d = 2: 2 * k1 = 6 rows per chirality
    Pt2 = _random_level_tiles(cd1, block2, k1, 6, 7)
    Ps = multilevel.site_prolongator(Pt2, cd1, block2, 2 * k1)
    X2, Y2 = multilevel.galerkin(Ps, X, Y, cd1, block2)
    cd2 = [cd1[m] // block2[m] for m in range(4)]
    a = np.sort_complex(np.round(np.linalg.eigvals(coarse.dense_coarse(X2, Y2, cd2)), 9))
    b = np.sort_complex(np.round(np.linalg.eigvals(coarse.dense_coarse(X, Y, cd1)), 9))
    assert np.abs(a - b).max() < 1e-8


def test_coarse_test_vectors_follow_eq2():
    dims, block1, k1 = (4, 4, 2, 2), (2, 2, 1, 1), 2
    U, w, bc, kappa, Pt, X, Y, cd1 = _fine_level(dims, block1, k1)
    sweeps = 3
    tv = multilevel.test_vectors(X, Y, cd1, 41, 2, 1, sweeps, 1)
    d, n = X.shape[0], X.shape[1]
    phi = philox.gaussian_field(41, [2, 3], d, n, 1)
    D1 = coarse.dense_coarse(X, Y, cd1)
    for i in range(2):
        p = phi[i].reshape(-1)
        corr = tv[i].reshape(-1) - p
        K = np.stack([np.linalg.matrix_power(D1, j) @ (-D1 @ p) for j in range(sweeps)], axis=1)
        y = np.linalg.lstsq(D1 @ K, -D1 @ p, rcond=None)[0]
        assert np.abs(corr - K @ y).max() < 1e-9 * np.abs(corr).max()


def _three_levels(post, coarse_tol=0.03, setup=False):
    dims, block1, k1, block2, k2 = (4, 2, 2, 4), (2, 2, 2, 2), 4, (2, 1, 1, 1), 4
    U = synthetic.haar_links(dims, 1000)
    w, bc, kappa = (1, 1, 1, 1), (1, 1, 1, -1), 0.124
    if setup:
        h = multilevel.Hierarchy(U, dims, kappa, w, bc, [block1, block2], [k1, k2], [4, 4],
                                 [2, 2], sweeps=5, seed=3000, coarse_tol=coarse_tol,
                                 coarse_restart=64, post=post)
    else:
        Pt1 = icsvd.icsvd(U, dims, kappa, w, bc, block1, k1, 4, 2, 5, 3000)[0]
        cd1 = [dims[m] // block1[m] for m in range(4)]
        Pt2 = _random_level_tiles(cd1, block2, k1, k2, 9)
        h = multilevel.Hierarchy(U, dims, kappa, w, bc, [block1, block2], [k1, k2],
                                 Pts=[Pt1, Pt2], coarse_tol=coarse_tol, coarse_restart=64,
                                 post=post)
    return h, U, dims, w, bc, kappa


def test_level1_kcycle_with_exact_coarsest_solve_is_coarse_grid_correction():
    h, *_ = _three_levels(post=0, coarse_tol=1e-14)
    X, Y = h.XY[0]
    D1 = coarse.dense_coarse(X, Y, h.cd[1])
    P2 = multilevel.dense_site_prolongator(h.Ps[1], h.cd[1], h.blocks[1])
    rng = np.random.default_rng(3)
    v = rng.standard_normal(D1.shape[0]) + 1j * rng.standard_normal(D1.shape[0])
    cgc = P2 @ np.linalg.solve(P2.conj().T @ D1 @ P2, P2.conj().T @ v)
    assert np.abs(h.kcycle(1, v) - cgc).max() < 1e-10 * np.abs(cgc).max()
    # with a post-smoother spanning level 1 the K-cycle is D_1^{-1}
    h.post = D1.shape[0]
    x = np.linalg.solve(D1, v)
    assert np.abs(h.kcycle(1, v) - x).max() < 1e-8 * np.abs(x).max()


def test_three_level_solve_matches_direct_solve():
    h, U, dims, w, bc, kappa = _three_levels(post=8, setup=True)
    b = synthetic.gaussian_rhs(dims, 2000)[0].reshape(-1)
    x, info = h.solve(b, tol=1e-10)
    D = wilson.dense_dirac(U, dims, kappa, w, bc)
    assert np.linalg.norm(b - D @ x) <= 1e-10 * np.linalg.norm(b)
    xs = np.linalg.solve(D, b)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert info['outer'] > 0 and info['coarse'] > 0
    # the level-1 setup produced an orthonormal, chirally block-diagonal P_2
    P2 = multilevel.dense_site_prolongator(h.Ps[1], h.cd[1], h.blocks[1])
    assert np.abs(P2.conj().T @ P2 - np.eye(P2.shape[1])).max() < 1e-13


def test_two_level_hierarchy_is_the_two_level_solver():
    dims, block = (4, 2, 2, 4), (2, 2, 2, 2)
    U = synthetic.haar_links(dims, 1000)
    w, bc, kappa = (1, 1, 1, 1), (1, 1, 1, -1), 0.124
    Pt = icsvd.icsvd(U, dims, kappa, w, bc, block, 4, 4, 2, 5, 3000)[0]
    h = multilevel.Hierarchy(U, dims, kappa, w, bc, [block], [4], Pts=[Pt])
    tl = mg.TwoLevel(U, dims, kappa, w, bc, block, Pt)
    rng = np.random.default_rng(4)
    v = rng.standard_normal(12 * wilson.volume(dims)) + 1j * rng.standard_normal(12 * wilson.volume(dims))
    assert np.abs(h.kcycle(0, v) - tl.kcycle(v)).max() < 1e-13 * np.abs(v).max()
