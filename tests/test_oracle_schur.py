"""Pins for the oracle's even-odd Schur form: dense block algebra, the spectral map
1 - (1 - lambda)^2, gamma_5 hermiticity and the reconstructed solve."""
import numpy as np
import pytest

from oracle import schur, wilson
from paper_2505_14399_gb300 import synthetic

ANISO = (1.0, 1.0, 1.0, 1 / 3.5)


def _dense_schur(U, dims, kappa, w, bc, dagger=False):
    n = 12 * wilson.volume(dims) // 2
    M = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = schur.schur_op(e, U, dims, kappa, w, bc, dagger).reshape(-1)
    return M


@pytest.mark.parametrize("bc,w", [((1, 1, 1, 1), (1, 1, 1, 1)), ((1, 1, 1, -1), ANISO)])
def test_schur_complement_of_the_dense_blocks(bc, w):
    dims, kappa = (4, 2, 2, 2), 0.13
    U = synthetic.haar_links(dims, 3)
    D = wilson.dense_dirac(U, dims, kappa, w, bc)
    par = np.repeat(wilson.parity_of_sites(dims), 12)
    e, o = par == 0, par == 1
    Dee, Deo, Doe, Doo = D[np.ix_(e, e)], D[np.ix_(e, o)], D[np.ix_(o, e)], D[np.ix_(o, o)]
    assert np.abs(Dee - np.eye(Dee.shape[0])).max() == 0 and np.abs(Doo - np.eye(Doo.shape[0])).max() == 0
    ref = Dee - Deo @ np.linalg.solve(Doo, Doe)
    S = _dense_schur(U, dims, kappa, w, bc)
    assert np.abs(S - ref).max() < 1e-14
    # gamma_5 acts site by site, so D_hat inherits gamma_5 hermiticity; the dagger form is D_hat^dag
    G5 = np.kron(np.eye(wilson.volume(dims) // 2), np.kron(wilson.GAMMA5, np.eye(3)))
    assert np.abs(G5 @ S @ G5 - S.conj().T).max() < 1e-14
    assert np.abs(_dense_schur(U, dims, kappa, w, bc, dagger=True) - S.conj().T).max() < 1e-14


def test_spectrum_is_the_image_of_the_full_spectrum():
    """H anticommutes with the parity sign, so spec(kappa H) is symmetric and
    spec(D_hat) = {1 - (1 - lambda)^2 : lambda in spec(D)}, each value taken half as often."""
    dims, kappa = (4, 2, 2, 2), 0.12
    U = synthetic.smooth_links(dims, 8)
    lam = np.linalg.eigvals(wilson.dense_dirac(U, dims, kappa))
    mapped = 1 - (1 - lam) ** 2
    ev = np.linalg.eigvals(_dense_schur(U, dims, kappa, (1, 1, 1, 1), (1, 1, 1, 1)))
    a = np.sort_complex(np.round(np.repeat(ev, 2), 8))
    b = np.sort_complex(np.round(mapped, 8))
    assert np.abs(a - b).max() < 1e-7
    # free field: the closed form carried through the same map
    Uf = synthetic.unit_links(dims)
    evf = np.linalg.eigvals(_dense_schur(Uf, dims, kappa, (1, 1, 1, 1), (1, 1, 1, -1)))
    ref = 1 - (1 - wilson.free_spectrum(dims, kappa, (1, 1, 1, 1), (1, 1, 1, -1))) ** 2
    assert np.abs(np.sort_complex(np.round(np.repeat(evf, 2), 9))
                  - np.sort_complex(np.round(ref, 9))).max() < 1e-8


def test_schur_solve_reconstructs_the_full_solution():
    dims, kappa = (4, 4, 2, 4), 0.124
    U = synthetic.haar_links(dims, 1000)
    w, bc = ANISO, (1, 1, 1, -1)
    b = synthetic.gaussian_rhs(dims, 2000)[0]
    x, its = schur.solve(b, U, dims, kappa, w, bc, tol=1e-12)
    r = b.reshape(-1) - wilson.dslash(x, U, dims, kappa, w, bc).reshape(-1)
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(b)
    D = wilson.dense_dirac(U, dims, kappa, w, bc)
    xs = np.linalg.solve(D, b.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - xs) <= 1e-9 * np.linalg.norm(xs)
    # the even half solves the Schur system; the odd half is the reconstruction
    xe, xo = schur.split(x, dims)
    bh = schur.prepare(b, U, dims, kappa, w, bc)
    assert np.abs(schur.schur_op(xe, U, dims, kappa, w, bc) - bh).max() < 1e-10
    assert np.array_equal(schur.join(xe, xo, dims), x)


def _tiny_level(schur, post):
    from oracle import icsvd, mg
    dims, block, kappa = (4, 2, 2, 2), (2, 2, 2, 2), 0.12
    U = synthetic.haar_links(dims, 9)
    Pt, _, _ = icsvd.icsvd(U, dims, kappa, (1, 1, 1, 1), (1, 1, 1, 1), block, 4, 4, 1, 2, 3000)
    return mg.TwoLevel(U, dims, kappa, (1, 1, 1, 1), (1, 1, 1, 1), block, Pt, post=post,
                       schur=schur), U, dims, kappa


def test_schur_smoother_satisfies_the_odd_equations():
    """For any number of steps the Schur-form correction e solves the odd rows exactly:
    (D e)_o = r_o, because e_o = r_o + kappa H_oe e_e."""
    lvl, U, dims, kappa = _tiny_level(True, 3)
    rng = np.random.default_rng(4)
    r = rng.standard_normal(12 * wilson.volume(dims)) + 1j * rng.standard_normal(12 * wilson.volume(dims))
    e = lvl.smooth(r)
    De = wilson.dslash(e, U, dims, kappa).reshape(-1, 4, 3)
    _, ro = schur.split(r, dims)
    _, Deo = schur.split(De, dims)
    assert np.abs(Deo - ro).max() < 1e-13
    # and the even rows only approximately after 3 steps (the smoother is not a solve)
    de, re = schur.split(De, dims)[0], schur.split(r, dims)[0]
    assert np.abs(de - re).max() > 1e-6


def test_schur_smoother_with_a_spanning_krylov_space_is_the_exact_inverse():
    """GMRES with as many steps as the even space has dimensions solves D_hat exactly, so the
    Schur-form smoother returns D^{-1} r (to rounding); the plain smoother with the same number
    of steps does not (its space has twice the dimension)."""
    n_even = 12 * 32 // 2
    lvl, U, dims, kappa = _tiny_level(True, n_even)
    rng = np.random.default_rng(5)
    n = 12 * wilson.volume(dims)
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = np.linalg.solve(wilson.dense_dirac(U, dims, kappa, (1, 1, 1, 1), (1, 1, 1, 1)), r)
    e = lvl.smooth(r)
    assert np.linalg.norm(e - x) / np.linalg.norm(x) < 1e-9


def test_schur_smoothed_kcycle_solve():
    """The two-level FGMRES with the Schur-form post-smoother reaches 1e-10 and matches the
    dense solve."""
    lvl, U, dims, kappa = _tiny_level(True, 4)
    rng = np.random.default_rng(6)
    n = 12 * wilson.volume(dims)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, info = lvl.solve(b, tol=1e-10)
    xd = np.linalg.solve(wilson.dense_dirac(U, dims, kappa, (1, 1, 1, 1), (1, 1, 1, 1)), b)
    assert info["residual"] <= 1e-10
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8
