"""Planted mistakes in the oracle must fail its pins (mutation checks, CPU only).

Each mutant rewrites one or two expressions in the source of one oracle function — a flipped
sign, a dropped conjugate or transpose, a neighbour taken on the wrong side, a missing factor
— compiles the rewritten function against the oracle module's own globals, installs it in
every oracle module that refers to the original for the duration of one test, and runs the
pins chosen to catch that kind of mistake: at least one of them must fail.  Every rewritten
snippet must occur exactly once in the original source, so that a later edit of the oracle
cannot silently turn a mutant into the original function.
"""
import inspect
import sys
import textwrap

import numpy as np
import pytest

import oracle.adjoint
import oracle.clover
import oracle.coarse
import oracle.critical_kappa
import oracle.icsvd
import oracle.krylov
import oracle.mg
import oracle.multilevel
import oracle.philox
import oracle.schur
import oracle.wilson
import test_oracle_clover as TC
import test_oracle_multilevel as TM
import test_oracle_numerics as TN
import test_oracle_schur as TS
import test_oracle_wilson as TW

ANISO_T = ((1, 1, 1, -1), TW.ANISO)
ANTI_X = ((-1, 1, 1, 1), (1.0, 0.5, 1.0, 1.0))
# x antiperiodic and weighted: on the 4x2x2x2 lattice only x has momenta with sin p != 0
FREE_X = ((-1, 1, 1, 1), (0.5, 1.0, 1.0, 1.0))


def _free_spectrum_small(bc, w):
    """The closed-form free-field spectrum on a 4x2x2x2 lattice (cheaper than the 4x2x2x4 pin)."""
    from paper_2505_14399_gb300 import synthetic
    dims = (4, 2, 2, 2)
    D = oracle.wilson.dense_dirac(synthetic.unit_links(dims), dims, 0.11, w, bc)
    ev = np.sort_complex(np.round(np.linalg.eigvals(D), 10))
    ref = np.sort_complex(np.round(oracle.wilson.free_spectrum(dims, 0.11, w, bc), 10))
    assert np.abs(ev - ref).max() < 1e-9


def _link_gradient_fd(n_dirs=2):
    """Central finite differences of |x|^2, x = D^{-1} b, against the oracle's link gradient."""
    from paper_2505_14399_gb300 import synthetic
    W = oracle.wilson
    dims = (2, 2, 2, 2)
    U = synthetic.smooth_links(dims, 4)
    w, bc, kappa = (1, 1, 1, 0.5), (1, 1, 1, -1), 0.12
    b = synthetic.gaussian_rhs(dims, 5)[0].reshape(-1)

    def loss(links):
        x = np.linalg.solve(W.dense_dirac(links, dims, kappa, w, bc), b)
        return float(np.vdot(x, x).real), x

    x = loss(U)[1]
    D = W.dense_dirac(U, dims, kappa, w, bc)
    g_b = np.linalg.solve(D.conj().T, 2 * x)
    G = oracle.adjoint.grad_link_angles(g_b, x, U, dims, kappa, w, bc)
    rng = np.random.default_rng(6)
    h = 1e-4
    for _ in range(n_dirs):
        om = rng.standard_normal((4, W.volume(dims), 8))
        fd = (loss(oracle.adjoint.perturb_links(U, h * om))[0]
              - loss(oracle.adjoint.perturb_links(U, -h * om))[0]) / (2 * h)
        assert abs(fd - float((G * om).sum())) < 1e-6 * max(1, abs(fd))


def _galerkin(dims, block):
    return lambda: TN.test_galerkin_stencil_equals_dense_product(dims, block)


GAL_A = _galerkin((4, 4, 2, 2), (2, 2, 2, 2))
GAL_B = _galerkin((6, 2, 2, 4), (2, 2, 1, 2))
# aggregates of two level-1 sites with two aggregates along x: hops inside and across them
ML_GAL = lambda: TM.test_coarse_level_galerkin_equals_dense_product(*TM.CASES[2])
HERM = [lambda: TW.test_gamma5_hermiticity_dense(*ANISO_T)]
PLANE = [TW.test_plane_wave_momentum_space_form]
COV = [TW.test_gauge_covariance]

# (id, module, function or Class.method, [(original snippet, replacement)], pins)
MUTANTS = [
    # Wilson-Dirac operator (Eq. 1 with the documented conventions)
    ("projector_sign_forward", oracle.wilson, "hopping",
     [("eye + sgn * GAMMA[mu], up", "eye - sgn * GAMMA[mu], up")], HERM + PLANE),
    ("projectors_swapped", oracle.wilson, "hopping",
     [("eye + sgn * GAMMA[mu], up", "eye - sgn * GAMMA[mu], up"),
      ("eye - sgn * GAMMA[mu], bwd", "eye + sgn * GAMMA[mu], bwd")], HERM + PLANE),
    ("backward_link_not_conjugated", oracle.wilson, "hopping",
     [("'xba,xsb->xsa', U.conj()", "'xba,xsb->xsa', U")], HERM + COV),
    ("backward_link_not_transposed", oracle.wilson, "hopping",
     [("'xba,xsb->xsa', U.conj()", "'xab,xsb->xsa', U.conj()")], HERM + COV),
    ("backward_hop_from_wrong_side", oracle.wilson, "hopping",
     [("_shift(Udag_psi, dims, mu, -1, bc)", "_shift(Udag_psi, dims, mu, +1, bc)")],
     HERM + PLANE),
    ("backward_hop_weight_dropped", oracle.wilson, "hopping",
     [("out += hop_weight[mu] * np.einsum('st,xtb->xsb', eye - sgn",
       "out += np.einsum('st,xtb->xsb', eye - sgn")], HERM + PLANE),
    ("forward_link_taken_at_neighbour", oracle.wilson, "hopping",
     [("up = np.einsum('xab,xsb->xsa', U, fwd)",
       "up = _shift(np.einsum('xab,xsb->xsa', U, psi), dims, mu, +1, bc)")], HERM + COV),
    ("boundary_phase_on_wrong_slice", oracle.wilson, "_shift",
     [("sl[ax] = dims[mu] - 1 if direction > 0 else 0",
       "sl[ax] = 0 if direction > 0 else dims[mu] - 1")],
     # on unit links the free spectrum cannot see this mistake (the Wilson projectors
     # annihilate back-tracking paths, the only closed paths that feel it); gamma_5
     # hermiticity on random links with an antiperiodic direction of extent 4 does
     [lambda: TW.test_gamma5_hermiticity_dense(*ANTI_X)]),
    ("kappa_sign", oracle.wilson, "dslash",
     [("psi - kappa * hopping", "psi + kappa * hopping")], PLANE),
    ("parity_output_swapped", oracle.wilson, "dslash_parity",
     [("h[par == parity]", "h[par == 1 - parity]")],
     [TW.test_parity_split_reassembles_full_operator]),
    ("free_spectrum_missing_weight", oracle.wilson, "free_spectrum",
     [("(w[m] * np.sin(P[m])) ** 2", "np.sin(P[m]) ** 2")],
     [lambda: _free_spectrum_small(*FREE_X)]),
    # Philox4x32-10 (published definition) and the Gaussian map
    ("philox_key_bump_swapped", oracle.philox, "philox4x32_10",
     [("(int(k0) + W0)", "(int(k0) + W1)")], [TN.test_philox_known_answers]),
    ("philox_output_permutation", oracle.philox, "philox4x32_10",
     [("c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]",
       "c = [hi0 ^ c[1] ^ k0, lo0, hi1 ^ c[3] ^ k1, lo1]")], [TN.test_philox_known_answers]),
    # Krylov smoother / solvers (Sec. 4)
    ("gmres_rhs_squared", oracle.krylov, "gmres_fixed",
     [("rhs[0] = beta", "rhs[0] = beta * beta")], [TN.test_gmres_full_krylov_is_exact_solve]),
    ("gmres_projection_conjugated", oracle.krylov, "gmres_fixed",
     [("H[i, j] = np.vdot(V[i], w)", "H[i, j] = np.vdot(w, V[i])")],
     [TN.test_gmres_full_krylov_is_exact_solve, TN.test_gmres_minimises_over_krylov_space]),
    ("gmres_coefficients_conjugated", oracle.krylov, "gmres_fixed",
     [("x = x + y[i] * V[i]", "x = x + np.conj(y[i]) * V[i]")],
     [TN.test_gmres_full_krylov_is_exact_solve]),
    ("fgmres_updates_with_v_not_z", oracle.krylov, "fgmres",
     [("x = x + y[i] * Z[i]", "x = x + y[i] * V[i]")], [TN.test_gmres_tol_and_fgmres]),
    # test vectors (Eq. 2), chiral split (Eq. 3), streaming SVD (Alg. 3, Eqs. 6-8)
    ("test_vector_source_sign", oracle.icsvd, "smooth",
     [("b = -A(phi.reshape(-1))", "b = A(phi.reshape(-1))")], [TN.test_test_vectors_follow_eq2]),
    ("chiral_split_spin_offset", oracle.icsvd, "chiral_split",
     [("vectors[:, :, 2 * a:2 * a + 2, :]", "vectors[:, :, a:a + 2, :]")],
     [TN.test_chiral_split_places_spins, TN.test_prolongator_is_orthonormal_and_chiral]),
    ("phi_without_sigma", oracle.icsvd, "icsvd_tiles",
     [("Phi[j][a] = Uk * Sk[None, :]", "Phi[j][a] = Uk")],
     [TN.test_icsvd_exact_when_stream_lies_in_rank_k_subspace,
      TN.test_icsvd_stream_recursion_and_energy_identity]),
    ("phi_with_sigma_squared", oracle.icsvd, "icsvd_tiles",
     [("Phi[j][a] = Uk * Sk[None, :]", "Phi[j][a] = Uk * (Sk ** 2)[None, :]")],
     [TN.test_icsvd_exact_when_stream_lies_in_rank_k_subspace,
      TN.test_icsvd_stream_recursion_and_energy_identity]),
    ("stream_memory_dropped", oracle.icsvd, "icsvd_tiles",
     [("Phi[j][a] = Uk * Sk[None, :]", "Phi[j][a] = Phi[j][a]")],
     [TN.test_icsvd_stream_recursion_and_energy_identity]),
    ("keeps_smallest_singular_vectors", oracle.icsvd, "rank_k_svd",
     [("return U[:, :kk], S[:kk]", "return U[:, -kk:], S[-kk:]")],
     [TN.test_icsvd_single_stream_is_csvd]),
    ("phase_not_conjugated", oracle.icsvd, "canonical_phase",
     [("np.conj(q) / np.where", "q / np.where")],
     [TN.test_icsvd_singular_values_bounded_by_dense_svd]),
    # restriction, prolongation, Galerkin operator (Eqs. 4-6), coarse stencil
    ("restrict_without_conjugate", oracle.coarse, "restrict",
     [("Ps.conj(), v)", "Ps, v)")], [GAL_A]),
    ("galerkin_transpose_not_adjoint", oracle.coarse, "galerkin",
     [("C = np.einsum('xra,xrb->xab', Ps[sl].conj(), B)",
       "C = np.einsum('xra,xrb->xab', Ps[sl], B)")], [GAL_A, GAL_B]),
    ("galerkin_backward_projector_sign", oracle.coarse, "galerkin",
     [("spin = eye + wilson.GAMMA[mu]", "spin = eye - wilson.GAMMA[mu]")], [GAL_A, GAL_B]),
    ("galerkin_block_crossing_off_by_one", oracle.coarse, "galerkin",
     [("cross = (xm % block[mu]) == block[mu] - 1", "cross = (xm % block[mu]) == 0")],
     [GAL_A, GAL_B]),
    ("galerkin_boundary_phase_dropped", oracle.coarse, "galerkin",
     [("phase = np.where(wrap, float(bc[mu]), 1.0)", "phase = np.ones(V)")], [GAL_A, GAL_B]),
    ("galerkin_diagonal_dropped", oracle.coarse, "galerkin",
     [("np.add.at(X, coarse, np.einsum('xra,xrb->xab', Ps.conj(), Ps))", "pass")],
     [GAL_A, GAL_B]),
    ("coarse_apply_neighbours_swapped", oracle.coarse, "coarse_apply",
     [("vc[nbr[dr]]", "vc[nbr[dr ^ 1]]")], [GAL_B]),
    ("coarse_neighbour_direction", oracle.coarse, "coarse_neighbours",
     [("(n[:, mu] + sgn) % cd[mu]", "(n[:, mu] - sgn) % cd[mu]")], [GAL_B]),
    # K-cycle (Sec. 2.1 end, Sec. 4)
    ("kcycle_residual_sign", oracle.mg, "TwoLevel.kcycle",
     [("r = np.asarray(v).reshape(-1) - self.D(e)", "r = self.D(e) - np.asarray(v).reshape(-1)")],
     [TN.test_kcycle_with_exact_coarse_solve_is_coarse_grid_correction]),
    ("kcycle_prolongation_dropped", oracle.mg, "TwoLevel.kcycle",
     [("return e + self.smooth(r)", "return self.smooth(r)")],
     [TN.test_kcycle_with_exact_coarse_solve_is_coarse_grid_correction]),
    # deeper levels: chiral SVD and Galerkin product on a coarse operator, multilevel K-cycle
    ("level_split_half_offset", oracle.multilevel, "chiral_split",
     [("vectors[:, :, a * k:(a + 1) * k]", "vectors[:, :, a:a + k]")],
     [TM.test_coarse_chiral_split_places_components]),
    ("level_prolongator_swaps_chirality", oracle.multilevel, "site_prolongator",
     [("Ps[:, a, :, a, :] = T[agg, a, local]", "Ps[:, a, :, 1 - a, :] = T[agg, a, local]")],
     [ML_GAL]),
    ("level_galerkin_edge_off_by_one", oracle.multilevel, "galerkin",
     [("edge = block[mu] - 1 if sgn > 0 else 0", "edge = 0 if sgn > 0 else block[mu] - 1")],
     [ML_GAL]),
    ("level_galerkin_neighbour_p_at_site", oracle.multilevel, "galerkin",
     [("Y[dr], Ps[nbr[dr]])", "Y[dr], Ps)")], [ML_GAL]),
    ("level_restrict_without_conjugate", oracle.multilevel, "restrict",
     [("Ps.conj(), v)", "Ps, v)")], [ML_GAL]),
    ("level_test_vector_level_word", oracle.multilevel, "test_vectors",
     [("gaussian_field(seed, ids, d, n, level)", "gaussian_field(seed, ids, d, n, 0)")],
     [TM.test_coarse_test_vectors_follow_eq2]),
    ("multilevel_kcycle_prolongation_dropped", oracle.multilevel, "Hierarchy.kcycle",
     [("return e + gmres_fixed(D, v - D(e), self.post)", "return gmres_fixed(D, v - D(e), self.post)")],
     [TM.test_level1_kcycle_with_exact_coarsest_solve_is_coarse_grid_correction]),
    # even-odd Schur form
    ("schur_second_hop_parity", oracle.schur, "schur_op",
     [("return v - hop(t, links, dims, kappa, 0,", "return v + hop(t, links, dims, kappa, 0,")],
     [lambda: TS.test_schur_complement_of_the_dense_blocks((1, 1, 1, 1), (1, 1, 1, 1))]),
    ("schur_rhs_sign", oracle.schur, "prepare",
     [("return be - hop(bo,", "return be + hop(bo,")],
     [TS.test_schur_solve_reconstructs_the_full_solution]),
    ("schur_reconstruction_sign", oracle.schur, "reconstruct",
     [("xo = bo - hop(x_even,", "xo = bo + hop(x_even,")],
     [TS.test_schur_solve_reconstructs_the_full_solution]),
    # Wilson-clover term
    ("sigma_anticommutator", oracle.clover, "sigma",
     [("0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])", "0.5j * (g[mu] @ g[nu] + g[nu] @ g[mu])")],
     [TC.test_sigma_hermitian_and_chiral]),
    ("field_strength_hermitian_part", oracle.clover, "field_strength",
     [("f = (Q - _dag(Q)) / 8j", "f = (Q + _dag(Q)) / 8j")], [TC.test_field_strength_of_abelian_fields]),
    ("field_strength_trace_kept", oracle.clover, "field_strength",
     [("F[p] = f - (tr / 3.0)[:, None, None] * np.eye(3)", "F[p] = f")],
     [TC.test_clover_term_is_hermitian_and_chirally_block_diagonal]),
    ("schur_smoother_not_reconstructed", oracle.mg, "TwoLevel.smooth",
     [("return _schur.reconstruct(ee, r, *a).reshape(-1)",
       "return _schur.join(ee, 0 * ee, self.dims).reshape(-1)")],
     [TS.test_schur_smoother_satisfies_the_odd_equations]),
    ("schur_smoother_unprepared_rhs", oracle.mg, "TwoLevel.smooth",
     [("rh = _schur.prepare(r, *a).reshape(-1)", "rh = _schur.split(r, self.dims)[0].reshape(-1)")],
     [TS.test_schur_smoother_with_a_spanning_krylov_space_is_the_exact_inverse]),
    ("ls_weights_dropped_in_normal_matrix", oracle.icsvd, "ls_prolongator_tiles",
     [("np.linalg.inv(Vc @ Om @ Vc.conj().T)", "np.linalg.inv(Vc @ Vc.conj().T)")],
     [TN.test_ls_prolongator_minimises_the_weighted_interpolation_error]),
    ("ls_coarse_vectors_without_sigma", oracle.icsvd, "ls_prolongator_tiles",
     [("Vc = np.diag(s[:k]) @ Vh[:k]", "Vc = Vh[:k]")],
     [TN.test_ls_prolongator_reduces_to_left_singular_vectors]),
    ("leaf_two_open", oracle.clover, "field_strength",
     [("_dag(_at(Um, dims, [(nu, 1), (mu, -1)]))", "_dag(_at(Um, dims, [(nu, 1)]))")],
     [TC.test_clover_gauge_covariance]),
    ("leaf_three_last_link_unshifted", oracle.clover, "field_strength",
     [("@ _at(Un, dims, [(nu, -1)]))", "@ Un)")], [TC.test_clover_gauge_covariance]),
    ("leaf_four_wrong_corner", oracle.clover, "field_strength",
     [("_at(Un, dims, [(nu, -1), (mu, 1)])", "_at(Un, dims, [(nu, -1)])")],
     [TC.test_clover_gauge_covariance]),
    ("clover_sign", oracle.clover, "clover_term",
     [("(-kappa * csw) * C", "(kappa * csw) * C")],
     [TC.test_clover_term_is_hermitian_and_chirally_block_diagonal]),
    ("galerkin_clover_dropped", oracle.coarse, "galerkin",
     [("np.add.at(X, coarse, np.einsum('xra,xrs,xsb->xab', Ps.conj(), clover, Ps))", "pass")],
     [TC.test_galerkin_with_clover_equals_dense_product]),
    # link-angle gradient of the adjoint
    ("gradient_backward_projector_sign", oracle.adjoint, "grad_link_angles",
     [("eye + wilson.GAMMA[mu], t2", "eye - wilson.GAMMA[mu], t2")], [_link_gradient_fd]),
    ("gradient_neighbour_term_dropped", oracle.adjoint, "grad_link_angles",
     [("+ np.einsum('xsb,xsb->x', g_b[nb].conj(), t2))", ")")], [_link_gradient_fd]),
    ("gradient_generator_not_daggered", oracle.adjoint, "grad_link_angles",
     [("dUd = np.conj(np.swapaxes(dU, 1, 2))", "dUd = np.swapaxes(dU, 1, 2)")],
     [_link_gradient_fd]),
    # Gaussian draws (Box-Muller of the Philox uniforms)
    ("box_muller_radius_unscaled", oracle.philox, "gaussian_field",
     [("rho = np.sqrt(-2.0 * np.log(1.0 - ua))", "rho = np.sqrt(-np.log(1.0 - ua))")],
     [TN.test_gaussian_moments]),
    ("box_muller_half_circle", oracle.philox, "gaussian_field",
     [("th = 2.0 * np.pi * ub", "th = np.pi * ub")], [TN.test_gaussian_moments]),
    # the test vectors of one stream and the streams of Algorithm 3
    ("test_vector_ids_shifted", oracle.icsvd, "test_vectors",
     [("ids = np.arange(stream * r, stream * r + r)",
       "ids = np.arange(stream * r + 1, stream * r + r + 1)")],
     [TN.test_test_vectors_follow_eq2]),
    ("icsvd_streams_repeat_the_first", oracle.icsvd, "icsvd",
     [("test_vectors(links, dims, kappa, w, bc, seed, r, s, sweeps, clover)",
       "test_vectors(links, dims, kappa, w, bc, seed, r, 0, sweeps, clover)")],
     [TN.test_icsvd_without_truncation_keeps_every_stream]),
    # prolongation from the per-site blocks of P
    ("prolong_conjugates_p", oracle.coarse, "prolong",
     [("np.einsum('xra,xa->xr', Ps, vc[coarse])", "np.einsum('xra,xa->xr', Ps.conj(), vc[coarse])")],
     [GAL_A]),
    ("site_prolongator_swaps_chirality", oracle.coarse, "site_prolongator",
     [("Ps[:, 2 * a:2 * a + 2, :, a, :] = T[coarse, a, local]",
       "Ps[:, 2 * a:2 * a + 2, :, 1 - a, :] = T[coarse, a, local]")], [GAL_A]),
    # restarted GMRES to a tolerance
    ("gmres_tol_basis_not_normalised", oracle.krylov, "gmres_tol",
     [("V.append(w / H[j + 1, j])", "V.append(w)")], [TN.test_gmres_tol_and_fgmres]),
    # even-odd split and join
    ("schur_join_parities_swapped", oracle.schur, "join",
     [("out[par == 0] = np.asarray(ve)", "out[par == 1] = np.asarray(ve)"),
      ("out[par == 1] = np.asarray(vo)", "out[par == 0] = np.asarray(vo)")],
     [TS.test_schur_solve_reconstructs_the_full_solution]),
    # the near-critical hopping parameter of the synthetic workloads
    ("hermitian_part_not_halved", oracle.critical_kappa, "hermitian_part_lmax",
     [("return 0.5 * (h + hd)", "return h + hd")], [TW.test_kappa_crit_bound_on_free_field]),
    ("hermitian_part_smallest_eigenvalue", oracle.critical_kappa, "hermitian_part_lmax",
     [("which='LA'", "which='SA'")], [TW.test_kappa_crit_bound_on_free_field]),
    # the clover term added to the Wilson-Dirac operator, the level-l prolongation, and the
    # two-level solve's operator / preconditioner roles
    ("clover_term_subtracted", oracle.clover, "dslash",
     [("return out + np.einsum('xrc,xc->xr', C, psi.reshape(-1, 12))",
       "return out - np.einsum('xrc,xc->xr', C, psi.reshape(-1, 12))")],
     [TC.test_galerkin_with_clover_equals_dense_product]),
    ("level_prolong_conjugates_p", oracle.multilevel, "prolong",
     [("np.einsum('jna,ja->jn', Ps, vc[agg])", "np.einsum('jna,ja->jn', Ps.conj(), vc[agg])")],
     [TM.test_level1_kcycle_with_exact_coarsest_solve_is_coarse_grid_correction]),
    ("two_level_solve_roles_swapped", oracle.mg, "TwoLevel.solve",
     [("fgmres(self.D, self.kcycle,", "fgmres(self.kcycle, self.D,")],
     [TN.test_two_level_solve_matches_direct_solve]),
]


def _lookup(module, qual):
    obj = module
    for part in qual.split("."):
        obj = getattr(obj, part)
    return obj


def _build_mutant(module, qual, subs):
    orig = _lookup(module, qual)
    src = textwrap.dedent(inspect.getsource(orig))
    for old, new in subs:
        assert src.count(old) == 1, "snippet %r must occur once in %s.%s" % (old, module.__name__, qual)
        src = src.replace(old, new)
    ns = {}
    exec(compile(src, "<mutant of %s.%s>" % (module.__name__, qual), "exec"), module.__dict__, ns)
    return orig, ns[qual.split(".")[-1]]


def _install(monkeypatch, module, qual, orig, mutant):
    if "." in qual:
        cls_name, meth = qual.split(".")
        monkeypatch.setattr(getattr(module, cls_name), meth, mutant)
        return
    for name, mod in list(sys.modules.items()):
        if name == "oracle" or name.startswith("oracle."):
            if getattr(mod, qual, None) is orig:
                monkeypatch.setattr(mod, qual, mutant)


@pytest.mark.parametrize("mid,module,qual,subs,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(monkeypatch, mid, module, qual, subs, pins):
    orig, mutant = _build_mutant(module, qual, subs)
    _install(monkeypatch, module, qual, orig, mutant)
    caught = []
    for pin in pins:
        try:
            pin()
        except Exception as e:          # a failed assertion, or a pin that cannot even run
            caught.append((pin, e))
            break
    assert caught, "mutant %s passed every pin meant to catch it" % mid


def test_unmutated_pins_pass():
    """Every pin the mutants are run against holds for the oracle as it stands, so a mutant
    counts as caught only because of what it changed."""
    seen = set()
    for m in MUTANTS:
        for pin in m[4]:
            if id(pin) not in seen:
                seen.add(id(pin))
                pin()
