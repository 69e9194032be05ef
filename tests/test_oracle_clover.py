"""Pins for the oracle's clover term: Clifford algebra, closed forms of the field strength on
abelian fields, hermiticity, chirality blocks, gamma_5 hermiticity, gauge covariance, and the
Galerkin product with the clover term."""
import numpy as np
import pytest

from oracle import clover, coarse, icsvd, wilson
from paper_2505_14399_gb300 import synthetic

CSW = 1.7


def test_sigma_hermitian_and_chiral():
    g5 = wilson.GAMMA5
    for mu, nu in clover.PAIRS:
        s = clover.sigma(mu, nu)
        assert np.abs(s - s.conj().T).max() < 1e-15
        assert np.abs(s @ g5 - g5 @ s).max() < 1e-15
        assert np.abs(s @ s - np.eye(4)).max() < 1e-15          # sigma_mu_nu^2 = 1 for mu != nu


def _abelian_links(dims, b):
    """U_1(x) = diag(e^{i b(x_0)}, e^{-i b(x_0)}, 1), every other link 1."""
    V = wilson.volume(dims)
    U = np.zeros((4, V, 3, 3), dtype=np.complex128)
    U[:] = np.eye(3)
    x0 = wilson.coords(dims)[:, 0]
    U[1, :, 0, 0] = np.exp(1j * b[x0])
    U[1, :, 1, 1] = np.exp(-1j * b[x0])
    return U


def test_field_strength_of_abelian_fields():
    dims = (6, 4, 2, 2)
    L0 = dims[0]
    x0 = wilson.coords(dims)[:, 0]
    diag = np.diag([1.0, -1.0, 0.0])
    # constant field: every plaquette of the 0-1 plane has angle B
    B = 2 * np.pi / L0
    F = clover.field_strength(_abelian_links(dims, B * np.arange(L0)), dims)
    assert np.abs(F[0] - np.sin(B) * diag).max() < 1e-15
    assert np.abs(F[1:]).max() < 1e-15
    # varying field: the four leaves around x carry the plaquette angles p(x0) (twice) and
    # p(x0 - 1) (twice), p(t) = b(t + 1) - b(t) with the lattice periodic in x0
    rng = np.random.default_rng(1)
    b = rng.uniform(-np.pi, np.pi, L0)
    p = np.roll(b, -1) - b
    F = clover.field_strength(_abelian_links(dims, b), dims)
    ref = (np.sin(p[x0]) + np.sin(p[(x0 - 1) % L0])) / 2
    assert np.abs(F[0] - ref[:, None, None] * diag).max() < 1e-14
    assert np.abs(F[1:]).max() < 1e-15
    # unit links: no field
    assert np.abs(clover.field_strength(synthetic.unit_links(dims), dims)).max() == 0


def test_clover_term_is_hermitian_and_chirally_block_diagonal():
    dims = (4, 2, 2, 4)
    U = synthetic.haar_links(dims, 4)
    F = clover.field_strength(U, dims)
    assert np.abs(F - np.conj(np.swapaxes(F, -1, -2))).max() < 1e-15
    assert np.abs(np.trace(F, axis1=2, axis2=3)).max() < 1e-15
    C = clover.clover_term(U, dims, 0.12, CSW)
    assert np.abs(C - np.conj(np.swapaxes(C, 1, 2))).max() < 1e-15
    # rows 0-5 (spins 1, 2) and 6-11 (spins 3, 4) do not mix
    assert np.abs(C[:, :6, 6:]).max() == 0 and np.abs(C[:, 6:, :6]).max() == 0
    # the constant abelian field gives -kappa c_sw sigma_01 (x) F_01 exactly
    B = 2 * np.pi / dims[0]
    Ua = _abelian_links(dims, B * np.arange(dims[0]))
    Ca = clover.clover_term(Ua, dims, 0.12, CSW)
    ref = -0.12 * CSW * np.kron(clover.sigma(0, 1), np.sin(B) * np.diag([1.0, -1.0, 0.0]))
    assert np.abs(Ca - ref[None]).max() < 1e-15


def test_clover_operator_gamma5_hermitian_and_free_field():
    dims = (4, 2, 2, 2)
    U = synthetic.haar_links(dims, 6)
    w, bc = (1.0, 1.0, 1.0, 1 / 3.5), (1, 1, 1, -1)
    D = clover.dense_dirac(U, dims, 0.12, CSW, w, bc)
    G5 = np.kron(np.eye(wilson.volume(dims)), np.kron(wilson.GAMMA5, np.eye(3)))
    assert np.abs(G5 @ D @ G5 - D.conj().T).max() < 1e-14
    rng = np.random.default_rng(2)
    psi = rng.standard_normal((wilson.volume(dims), 4, 3)) + 1j * rng.standard_normal((wilson.volume(dims), 4, 3))
    dd = clover.dslash(psi, U, dims, 0.12, CSW, w, bc, dagger=True).reshape(-1)
    assert np.abs(dd - D.conj().T @ psi.reshape(-1)).max() < 1e-13
    Uf = synthetic.unit_links(dims)
    assert np.abs(clover.dslash(psi, Uf, dims, 0.12, CSW, w, bc)
                  - wilson.dslash(psi, Uf, dims, 0.12, w, bc)).max() == 0


def test_clover_gauge_covariance():
    """F_mu_nu(x) -> G(x) F_mu_nu(x) G(x)^dag, so D_clover[U^g] = G D_clover[U] G^dag."""
    dims = (4, 4, 2, 2)
    U = synthetic.haar_links(dims, 11)
    G = synthetic.haar_links(dims, 12)[0]
    V = wilson.volume(dims)
    c = wilson.coords(dims)
    strides = [1, dims[0], dims[0] * dims[1], dims[0] * dims[1] * dims[2]]
    Ug = np.empty_like(U)
    for mu in range(4):
        nb = np.where(c[:, mu] == dims[mu] - 1, np.arange(V) - (dims[mu] - 1) * strides[mu],
                      np.arange(V) + strides[mu])
        Ug[mu] = G @ U[mu] @ np.conj(np.swapaxes(G[nb], 1, 2))
    F, Fg = clover.field_strength(U, dims), clover.field_strength(Ug, dims)
    assert np.abs(Fg - G[None] @ F @ np.conj(np.swapaxes(G, 1, 2))[None]).max() < 1e-13
    rng = np.random.default_rng(5)
    psi = rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3))
    lhs = clover.dslash(np.einsum('xab,xsb->xsa', G, psi), Ug, dims, 0.12, CSW)
    rhs = np.einsum('xab,xsb->xsa', G, clover.dslash(psi, U, dims, 0.12, CSW))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_galerkin_with_clover_equals_dense_product():
    dims, block, k = (4, 4, 2, 2), (2, 2, 2, 2), 3
    U = synthetic.smooth_links(dims, 21)
    w, bc, kappa = (1, 1, 1, 1), (1, 1, 1, -1), 0.12
    Pt = icsvd.icsvd(U, dims, kappa, w, bc, block, k, 2, 2, 3, 77)[0]
    C = clover.clover_term(U, dims, kappa, CSW)
    X, Y = coarse.galerkin(Pt, U, dims, block, kappa, w, bc, clover=C)
    cd = [dims[m] // block[m] for m in range(4)]
    P = icsvd.dense_prolongator(Pt, dims, block)
    ref = P.conj().T @ clover.dense_dirac(U, dims, kappa, CSW, w, bc) @ P
    Dc = coarse.dense_coarse(X, Y, cd)
    assert np.abs(Dc - ref).max() < 1e-13
    d = Pt.shape[0]
    s3 = np.kron(np.eye(d), np.kron(np.diag([1, -1]), np.eye(k)))
    assert np.abs(s3 @ Dc @ s3 - Dc.conj().T).max() < 1e-13


def test_clover_test_vectors_follow_eq2():
    """Test vectors of the clover operator: psi - phi is the 4-step Krylov minimiser of
    ||-D phi - D psi'|| with the dense D_clover (Eq. 2 with D = D_W + C)."""
    from oracle import philox
    dims = (2, 2, 2, 4)
    U = synthetic.haar_links(dims, 13)
    C = clover.clover_term(U, dims, 0.12, CSW)
    tv = icsvd.test_vectors(U, dims, 0.12, (1, 1, 1, 1), (1, 1, 1, 1), 99, 2, 1, 4, clover=C)
    phi = philox.gaussian_vectors(99, [2, 3], wilson.volume(dims))
    D = clover.dense_dirac(U, dims, 0.12, CSW)
    for i in range(2):
        p = phi[i].reshape(-1)
        corr = tv[i].reshape(-1) - p
        K = np.stack([np.linalg.matrix_power(D, j) @ (-D @ p) for j in range(4)], axis=1)
        y = np.linalg.lstsq(D @ K, -D @ p, rcond=None)[0]
        assert np.abs(corr - K @ y).max() < 1e-8 * np.abs(corr).max()


def test_clover_two_level_solve():
    """The two-level K-cycle FGMRES with D = D_W + C solves the clover system: true residual
    1e-10 and the dense solution."""
    from oracle import mg
    dims, block, kappa = (4, 2, 2, 2), (2, 2, 2, 2), 0.12
    U = synthetic.smooth_links(dims, 14)
    C = clover.clover_term(U, dims, kappa, CSW)
    Pt, _, _ = icsvd.icsvd(U, dims, kappa, (1, 1, 1, 1), (1, 1, 1, 1), block, 4, 4, 1, 2, 3000,
                           clover=C)
    lvl = mg.TwoLevel(U, dims, kappa, (1, 1, 1, 1), (1, 1, 1, 1), block, Pt, clover=C)
    rng = np.random.default_rng(7)
    n = 12 * wilson.volume(dims)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, info = lvl.solve(b, tol=1e-10)
    xd = np.linalg.solve(clover.dense_dirac(U, dims, kappa, CSW), b)
    assert info["residual"] <= 1e-10
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8
