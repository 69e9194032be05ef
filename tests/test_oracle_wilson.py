"""Pins for the oracle's Wilson-Dirac operator (closed forms, brute force, symmetries)."""
import numpy as np
import pytest

from oracle import wilson
from paper_2505_14399_gb300 import synthetic

ANISO = (1.0, 1.0, 1.0, 1 / 3.5)


def test_gamma_algebra_and_chirality():
    g, g5 = wilson.GAMMA, wilson.GAMMA5
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            anti = g[m] @ g[n] + g[n] @ g[m]
            assert np.allclose(anti, 2 * np.eye(4) * (m == n))
    # Eq. 3 needs spins 1,2 / 3,4 to be the two chiralities
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize("bc,w", [((1, 1, 1, 1), (1, 1, 1, 1)), ((1, 1, 1, -1), ANISO),
                                  ((-1, 1, 1, 1), (1.0, 0.5, 1.0, 1.0))])
def test_gamma5_hermiticity_dense(bc, w):
    dims = (4, 2, 2, 2)
    U = synthetic.haar_links(dims, 7)
    D = wilson.dense_dirac(U, dims, 0.13, w, bc)
    G5 = np.kron(np.eye(wilson.volume(dims)), np.kron(wilson.GAMMA5, np.eye(3)))
    assert np.abs(G5 @ D @ G5 - D.conj().T).max() < 1e-14
    Dd = wilson.dense_dirac(U, dims, 0.13, w, bc, dagger=True)
    assert np.abs(Dd - D.conj().T).max() < 1e-14


@pytest.mark.parametrize("bc,w", [((1, 1, 1, 1), (1, 1, 1, 1)), ((1, 1, 1, -1), ANISO),
                                  ((-1, 1, 1, 1), (1.0, 0.5, 1.0, 1.0))])
def test_free_field_spectrum_dense(bc, w):
    dims = (4, 2, 2, 4)
    U = synthetic.unit_links(dims)
    D = wilson.dense_dirac(U, dims, 0.11, w, bc)
    ev = np.linalg.eigvals(D)
    ref = wilson.free_spectrum(dims, 0.11, w, bc)
    key = lambda z: np.lexsort((np.round(z.imag, 9), np.round(z.real, 9)))
    assert np.abs(np.sort_complex(np.round(ev, 10)) - np.sort_complex(np.round(ref, 10))).max() < 1e-9
    assert len(ev) == len(ref)


def test_plane_wave_momentum_space_form():
    """D exp(ipx) u = [1 - 2k sum w cos p + 2ik sum w sin p gamma_mu] exp(ipx) u (pins signs)."""
    dims = (8, 4, 6, 8)
    kappa = 0.12
    w = ANISO
    U = synthetic.unit_links(dims)
    c = wilson.coords(dims)
    rng = np.random.default_rng(3)
    n = np.array([1, 3, 2, 5])
    p = 2 * np.pi * n / np.array(dims)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    ph = np.exp(1j * (c @ p))
    psi = ph[:, None, None] * u[None]
    M = (1 - 2 * kappa * sum(w[m] * np.cos(p[m]) for m in range(4))) * np.eye(4) \
        + 2j * kappa * sum(w[m] * np.sin(p[m]) * wilson.GAMMA[m] for m in range(4))
    ref = ph[:, None, None] * (M @ u)[None]
    out = wilson.dslash(psi, U, dims, kappa, w)
    assert np.abs(out - ref).max() < 1e-13


def test_gauge_covariance():
    """D[U^g] = G D[U] G^dag with U^g_mu(x) = G(x) U_mu(x) G(x+mu)^dag."""
    dims = (4, 4, 2, 4)
    U = synthetic.haar_links(dims, 11)
    G = synthetic.haar_links(dims, 12)[0]            # one SU(3) matrix per site
    V = wilson.volume(dims)
    c = wilson.coords(dims)
    strides = [1, dims[0], dims[0] * dims[1], dims[0] * dims[1] * dims[2]]
    Ug = np.empty_like(U)
    for mu in range(4):
        nb = np.where(c[:, mu] == dims[mu] - 1, np.arange(V) - (dims[mu] - 1) * strides[mu],
                      np.arange(V) + strides[mu])
        Ug[mu] = G @ U[mu] @ np.conj(np.swapaxes(G[nb], 1, 2))
    rng = np.random.default_rng(5)
    psi = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
    bc = (1, 1, 1, -1)
    lhs = wilson.dslash(np.einsum('xab,xsb->xsa', G, psi), Ug, dims, 0.12, ANISO, bc)
    rhs = np.einsum('xab,xsb->xsa', G, wilson.dslash(psi, U, dims, 0.12, ANISO, bc))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_parity_split_reassembles_full_operator():
    dims = (4, 4, 4, 2)
    U = synthetic.haar_links(dims, 2)
    V = wilson.volume(dims)
    rng = np.random.default_rng(9)
    psi = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
    par = wilson.parity_of_sites(dims)
    full = wilson.dslash(psi, U, dims, 0.1, ANISO, (1, 1, 1, -1))
    for p in (0, 1):
        hop = wilson.dslash_parity(psi[par == 1 - p], U, dims, 0.1, p, ANISO, (1, 1, 1, -1))
        assert np.abs(full[par == p] - (psi[par == p] + hop)).max() < 1e-14
    # checkerboard index = site // 2 lists the sites of one parity in increasing order
    for p in (0, 1):
        idx = np.nonzero(par == p)[0]
        assert np.array_equal(idx // 2, np.arange(V // 2))


def test_links_are_special_unitary():
    for U in (synthetic.haar_links((2, 2, 2, 2), 1), synthetic.smooth_links((2, 2, 2, 2), 1)):
        I = np.einsum('mxab,mxcb->mxac', U, U.conj())
        assert np.abs(I - np.eye(3)).max() < 1e-13
        assert np.abs(np.linalg.det(U) - 1).max() < 1e-13


def test_kappa_crit_bound_on_free_field():
    """Unit links: H is normal with largest real eigenvalue 2 sum w (periodic), so the
    Hermitian-part bound is exact: kappa_crit = 1 / (2 sum_mu w_mu)."""
    from oracle import critical_kappa
    dims = (4, 4, 2, 4)
    w = (1.0, 1.0, 1.0, 1 / 3.5)
    kc = critical_kappa.kappa_crit(synthetic.unit_links(dims), dims, w, (1, 1, 1, 1), tol=1e-10)
    assert abs(kc - 1 / (2 * sum(w))) < 1e-9
    # and it lower-bounds the singular point on random links: D at 0.999 kappa_crit has
    # every eigenvalue with positive real part
    U = synthetic.smooth_links(dims, 3)
    kc = critical_kappa.kappa_crit(U, dims, tol=1e-10)
    ev = np.linalg.eigvals(wilson.dense_dirac(U, dims, 0.999 * kc))
    assert ev.real.min() > 0
