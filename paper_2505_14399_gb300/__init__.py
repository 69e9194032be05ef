"""GB300 (sm_103a) streaming chiral-SVD multigrid for Wilson fermions.

Implements the hot path of Whyte, Stathopoulos, Romero, "Accelerating multigrid with
streaming chiral SVD for Wilson fermions in lattice QCD" (arXiv:2505.14399): the
Wilson-Dirac stencil, test-vector smoothing (Eq. 2), the streaming chiral SVD that
builds the prolongator (Algorithm 3, Eqs. 6-8), restriction/prolongation, the
Galerkin coarse operator (Eq. 5) and the K-cycle preconditioned FGMRES solve of
D x = b (Eq. 1), as hand-written CUDA behind the C ABI of include/wilson_mg.h.

``api`` holds the torch-facing binding; ``synthetic`` the seeded workload inputs.
The CUDA library is loaded lazily on first use and its absence is an error.
"""
