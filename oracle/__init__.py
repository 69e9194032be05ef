"""FP64 CPU oracle for the streaming chiral-SVD multigrid hot path (test infrastructure).

This package is TEST INFRASTRUCTURE ONLY.  It is a plain, slow, obviously correct
numpy restatement of what the GPU library computes, written from the paper
(Whyte, Stathopoulos, Romero, "Accelerating multigrid with streaming chiral SVD
for Wilson fermions in lattice QCD", arXiv:2505.14399):

* ``wilson``   -- the Wilson-Dirac operator D of Eq. (1) with the chiral gamma basis
                  that the chiral split of Eq. (3) presupposes; dense D for tiny lattices.
* ``philox``   -- the Philox4x32-10 counter-based generator (Salmon et al., SC'11) and
                  the complex-Gaussian map used for the random initial guesses of Eq. (2).
* ``krylov``   -- minimal-residual GMRES (fixed steps, tolerance-driven) and flexible
                  GMRES, the smoother and solver named in Sec. 4.
* ``icsvd``    -- test-vector generation (Eq. 2), chiral split (Eq. 3), the streaming
                  chiral SVD of Algorithm 3 (Eqs. 7-8) and the prolongator of Eq. (6).
* ``coarse``   -- restriction R = P^dag, prolongation, the Galerkin operator of Eq. (5)
                  as a nearest-neighbour coarse stencil, and its application.
* ``mg``       -- the two-level K-cycle preconditioned FGMRES solve of Eq. (1).
* ``multilevel`` -- the same setup and Galerkin product applied to a coarse operator
                  (sigma_3 as its chirality) and the K-cycle on every level of a deeper
                  hierarchy (Sec. 2.1 end, Sec. 4).
* ``schur``    -- the even-odd Schur-complement form of D x = b (Sec. 1 lists even-odd
                  preconditioning): D_hat = 1 - kappa^2 H_eo H_oe and the reconstruction.
* ``clover``   -- the Wilson-clover term (the action of Configuration B, Sec. 4): clover-leaf
                  field strength, sigma_mu_nu F_mu_nu, and D_clover.
* ``adjoint``  -- gradients of |x|^2, x = D^{-1} b, with respect to b and link angles.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import it.  The GPU library never imports, links or calls anything here, and nothing
here imports the GPU library: the two share no code.  Everything is complex128.

Parity pins: every function is pinned in ``tests/test_oracle_*.py`` against closed
forms, dense brute force, library routines or published known-answer values; the one
exception is noted in the ``mg`` module header.
"""
