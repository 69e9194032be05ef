"""Krylov solvers, FP64 oracle (test infrastructure only).

Sec. 4 uses FGMRES both as the smoother and as the solver on every level.  The
paper gives no restart lengths; the library's readings are:

* smoother (test vectors, Eq. 2; post-smoothing in the K-cycle): ``m`` steps of
  unrestarted GMRES from x0 = 0, i.e. the exact minimiser of ||b - A x|| over the
  Krylov space K_m(A, b);
* coarse solve: restarted GMRES until ||b - A x|| <= rtol ||b|| (0.03 in Sec. 4);
* outer solve: restarted flexible GMRES (right preconditioning whose action may change
  per step, which the K-cycle requires).

Arnoldi uses modified Gram-Schmidt and the small least-squares problem is solved with
numpy's lstsq; both are plain textbook forms (Saad, Iterative Methods, Alg. 6.9/9.6).
"""
import numpy as np


def _norm(v):
    return float(np.sqrt(np.vdot(v, v).real))


def gmres_fixed(A, b, m):
    """m steps of GMRES from x0 = 0; returns the minimiser of ||b - A x|| over K_m(A, b)."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    beta = _norm(b)
    x = np.zeros_like(b)
    if beta == 0.0 or m == 0:
        return x
    V = [b / beta]
    H = np.zeros((m + 1, m), dtype=np.complex128)
    steps = m
    for j in range(m):
        w = np.asarray(A(V[j]), dtype=np.complex128).reshape(-1)
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = _norm(w)
        if H[j + 1, j] == 0.0:
            steps = j + 1
            break
        V.append(w / H[j + 1, j])
    rhs = np.zeros(steps + 1, dtype=np.complex128)
    rhs[0] = beta
    y = np.linalg.lstsq(H[:steps + 1, :steps], rhs, rcond=None)[0]
    for i in range(steps):
        x = x + y[i] * V[i]
    return x


def gmres_tol(A, b, rtol, restart, maxiter, x0=None):
    """Restarted GMRES(restart) until ||b - A x|| <= rtol ||b||.

    Convergence is tested on the Arnoldi least-squares residual after every step.
    Returns (x, iterations, true relative residual).
    """
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    bn = _norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    if bn == 0.0:
        return x, 0, 0.0
    its = 0
    r = b - np.asarray(A(x)).reshape(-1) if x0 is not None else b.copy()
    while its < maxiter:
        beta = _norm(r)
        if beta <= rtol * bn:
            break
        V = [r / beta]
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        steps = 0
        y = None
        for j in range(restart):
            w = np.asarray(A(V[j]), dtype=np.complex128).reshape(-1)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = _norm(w)
            steps = j + 1
            its += 1
            rhs = np.zeros(steps + 1, dtype=np.complex128)
            rhs[0] = beta
            y = np.linalg.lstsq(H[:steps + 1, :steps], rhs, rcond=None)[0]
            res = _norm(rhs - H[:steps + 1, :steps] @ y)
            if res <= rtol * bn or its >= maxiter or H[j + 1, j] == 0.0:
                break
            V.append(w / H[j + 1, j])
        for i in range(steps):
            x = x + y[i] * V[i]
        r = b - np.asarray(A(x)).reshape(-1)
        if _norm(r) <= rtol * bn:
            break
    return x, its, _norm(b - np.asarray(A(x)).reshape(-1)) / bn


def fgmres(A, M, b, rtol, restart, maxiter, x0=None):
    """Restarted flexible GMRES with right preconditioner M (any map v -> z).

    x = x0 + Z y with Z = [M(v_0), ..., M(v_{j})] and y the Arnoldi least-squares
    minimiser; convergence is judged on the Arnoldi residual and confirmed on the
    true residual b - A x at the end of each cycle.
    Returns (x, iterations, true relative residual).
    """
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    bn = _norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    if bn == 0.0:
        return x, 0, 0.0
    its = 0
    r = b - np.asarray(A(x)).reshape(-1)
    while its < maxiter:
        beta = _norm(r)
        if beta <= rtol * bn:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        steps = 0
        y = None
        for j in range(restart):
            Z.append(np.asarray(M(V[j]), dtype=np.complex128).reshape(-1))
            w = np.asarray(A(Z[j]), dtype=np.complex128).reshape(-1)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = _norm(w)
            steps = j + 1
            its += 1
            rhs = np.zeros(steps + 1, dtype=np.complex128)
            rhs[0] = beta
            y = np.linalg.lstsq(H[:steps + 1, :steps], rhs, rcond=None)[0]
            res = _norm(rhs - H[:steps + 1, :steps] @ y)
            if res <= rtol * bn or its >= maxiter or H[j + 1, j] == 0.0:
                break
            V.append(w / H[j + 1, j])
        for i in range(steps):
            x = x + y[i] * Z[i]
        r = b - np.asarray(A(x)).reshape(-1)
    return x, its, _norm(r) / bn
