"""Error bounds of the batched streaming SVD against the oracle's dense SVD (Algorithm 3).

The library forms every tile's Gram matrix G = A^dag A, diagonalises it by Jacobi rotations and
rotates the tile (A V = U Sigma); the oracle takes a dense SVD of A.  Forming G in arithmetic of
unit roundoff u by sums over the M rows of a tile perturbs it by E with
|E_ij| <= gamma_M ||a_i|| ||a_j||, gamma_M = M u (the standard bound for a dot product of length
M), so ||E|| <= gamma_M ||A||_F^2, and first-order perturbation theory bounds the difference of
the two results, stream by stream:

* the kept subspace of stream s moves by at most ||E|| / g_s (Davis-Kahan), where g_s is the
  eigenvalue gap of G at the truncation, sigma_kk^2 - sigma_{kk+1}^2; a stream that keeps every
  column selects no subspace: Phi = A V is then a unitary rotation of A, correct to
  u ||A||_F (g_s = sigma_1^2), except in the last stream, whose normalised columns
  A V Sigma^-1 amplify the error by 1 / sigma_kk^2 (g_s = sigma_kk^2);
* the error carried into stream s + 1 is that of Phi_s = U_kk Sigma_kk, at most sigma_1 times the
  subspace error, and it moves the next stream's spectrum by no more (Weyl).
So with K_s = sum_{t <= s} ||A_t||_F^2 / g_t over the streams so far:

    || P P^dag - P_o P_o^dag ||_max <= C gamma_M K_s          (projector of the kept columns)
    | sigma_i - sigma_o,i |         <= C gamma_M K_s sigma_1   (kept singular values of stream s)

with C = 16 covering the constants of the Gram sums, the Jacobi rotations and the update (the
bound is pinned on the CPU against a plain Gram-route emulation in tests/test_svd_bounds.py).
Unit roundoffs: FP64 sums 2^-53; double-float sums (an unevaluated sum of two floats with
error-free products and sums) 2^-48.

The single-pass route (double-float) does not sum the Gram block of the kept columns
Phi_{s-1} = A_{s-1} V_k: it takes it as the diagonal of the previous stream's eigenvalues,
Phi^dag Phi = V_k^dag G V_k = Lambda_k.  That block is then off by the Jacobi residual (pairs
are left unrotated below tol sqrt(G_aa G_bb), tol = 1e-13) and by the rounding of Phi's
c-term sums, both below gamma_M ||A||_F^2 for c << M (c = 20, M = 1536 on the timed
workload), so the same bound holds.

For test vectors that themselves carry a relative error delta (the FP32 smoother against the
FP64 one), the tile moves by ||dA||_F <= delta ||A||_F and the same reasoning gives
    || dPi || <= C_v delta sum_t ||A_t||_F sigma_1,t / g_t,   | d sigma | <= C_v delta sum_t ||A_t||_F
(C_v = 4).
"""
import numpy as np

from oracle import icsvd

U64 = 2.0 ** -53
UDF = 2.0 ** -48
C_ARITH = 16.0
C_VEC = 4.0


def stream_spectra(stream_tiles, k):
    """Full singular values of A_s = [Phi_{s-1} | Psi_s] for every stream and tile, from the
    oracle's own recursion.  Returns a list over s of (sv (d, 2, c_s), kk_s)."""
    out = []
    for s in range(len(stream_tiles)):
        psi = stream_tiles[s]
        if s == 0:
            A = psi
        else:
            Pt, S, _ = icsvd.icsvd_tiles(stream_tiles[:s], k)
            # Phi_{s-1} = U Sigma up to a phase per column, which leaves the spectrum unchanged
            A = np.concatenate([Pt * S[:, :, None, :], psi], axis=3)
        sv = np.linalg.svd(A, compute_uv=False)
        out.append((sv, min(k, A.shape[3])))
    return out


def cumulative_conditions(spectra):
    """K_s (d, 2) for every stream: sum over t <= s of ||A_t||_F^2 / g_t, and sigma_1 of s.
    Also the sums used by the test-vector bound: sum_t ||A_t||_F sigma_1,t / g_t and
    sum_t ||A_t||_F."""
    K, Kv, Fv, s1 = [], [], [], []
    acc = accv = accf = 0.0
    for s, (sv, kk) in enumerate(spectra):
        F2 = (sv ** 2).sum(axis=-1)
        if sv.shape[-1] > kk:
            g = sv[..., kk - 1] ** 2 - sv[..., kk] ** 2
        elif s == len(spectra) - 1:
            g = sv[..., kk - 1] ** 2
        else:
            g = sv[..., 0] ** 2
        acc = acc + F2 / g
        accv = accv + np.sqrt(F2) * sv[..., 0] / g
        accf = accf + np.sqrt(F2)
        K.append(acc)
        Kv.append(accv)
        Fv.append(accf)
        s1.append(sv[..., 0])
    return K, Kv, Fv, s1


def gamma(u, rows):
    """gamma_M = M u of a sum of M products."""
    return rows * u


def arithmetic_bounds(spectra, u, rows):
    """Per stream: (projector bound (d, 2), singular-value bound (d, 2)) for Gram sums over
    `rows` rows in arithmetic of unit roundoff u."""
    K, _, _, s1 = cumulative_conditions(spectra)
    g = gamma(u, rows)
    return [(C_ARITH * g * K[s], C_ARITH * g * K[s] * s1[s]) for s in range(len(K))]


def vector_bounds(spectra, delta, u, rows):
    """As arithmetic_bounds, plus the effect of test vectors with relative error delta."""
    K, Kv, Fv, s1 = cumulative_conditions(spectra)
    g = gamma(u, rows)
    out = []
    for s in range(len(K)):
        bp = C_ARITH * g * K[s] + C_VEC * delta * Kv[s]
        bs = C_ARITH * g * K[s] * s1[s] + C_VEC * delta * Fv[s]
        out.append((bp, bs))
    return out


def projector_errors(P, Pt):
    """max |P P^dag - Pt Pt^dag| per tile; P in library layout (d, 2, k, rows), Pt (d, 2, rows, k)."""
    d = P.shape[0]
    err = np.zeros((d, 2))
    for j in range(d):
        for a in range(2):
            Ug = P[j, a].T
            Uo = Pt[j, a]
            err[j, a] = np.abs(Ug @ Ug.conj().T - Uo @ Uo.conj().T).max()
    return err
