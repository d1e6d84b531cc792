"""Flexible GMRES with right preconditioning, the outer Krylov method of Sec. 5
(FGMRES(20) in Fig. cslp_rsms_comp, non-restarted FGMRES in Tables 3-5;
convergence when the relative residual drops below 1e-6).

Oracle module (test infrastructure only).

Arnoldi with modified Gram-Schmidt; the Hessenberg matrix is reduced by complex
Givens rotations G = [[c, s], [-conj(s), c]] with c real.  Stopping test:
|g_{j+1}| / ||b|| < tol.  At the end of every restart cycle the iterate is
formed and its true residual recomputed; the solve stops when that is below tol
or ``maxit`` preconditioner applications have been spent.  The iteration count
is the number of preconditioner applications.
"""
import numpy as np


def givens(a, b):
    """(c, s, r) with c real, c a + s b = r and -conj(s) a + c b = 0."""
    if a == 0:
        return 0.0, 1.0 + 0j, b
    t = np.hypot(abs(a), abs(b))
    ph = a / abs(a)
    return abs(a) / t, ph * np.conj(b) / t, ph * t


def fgmres(apply_A, b, apply_M, tol=1e-6, maxit=200, restart=None, x0=None,
           callback=None):
    """Solve A x = b.  Returns (x, info) with info keys ``iterations``,
    ``converged``, ``relres`` (true relative residual) and ``history`` (the
    estimated relative residual after every iteration)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    m = maxit if restart is None else int(restart)
    bnorm = np.linalg.norm(b)
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    hist = []
    if bnorm == 0.0:
        return x, dict(iterations=0, converged=True, relres=0.0, history=hist)
    r = b - apply_A(x)
    beta = np.linalg.norm(r)
    its = 0
    while True:
        if beta / bnorm < tol or its >= maxit:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        for j in range(m):
            z = apply_M(V[j])
            Z.append(z)
            w = apply_A(z)
            its += 1
            for i in range(j + 1):                 # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):                     # earlier rotations
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -np.conj(sn[i]) * hi + cs[i] * hi1
            hnext = H[j + 1, j]
            cs[j], sn[j], H[j, j] = givens(H[j, j], hnext)
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            est = abs(g[j + 1]) / bnorm
            hist.append(est)
            if callback is not None:
                callback(its, est)
            if est < tol or its >= maxit or hnext == 0.0:
                break
            V.append(w / hnext)
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        for i in range(k):
            x = x + y[i] * Z[i]
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
    relres = beta / bnorm
    return x, dict(iterations=its, converged=bool(relres < tol), relres=float(relres),
                   history=hist)


def stationary(apply_A, b, apply_M, tol=1e-6, maxit=200):
    """RS-CGC as a solver (Sec. 5, the parenthesised counts of Table 3): the iteration
    x_{k+1} = x_k + M (b - A x_k) from x_0 = 0, stopped once the relative residual
    ||b - A x|| / ||b|| is below tol or after maxit applications of M.  The iteration
    count is the number of applications of M."""
    b = np.asarray(b, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bnorm == 0:
        return x, dict(iterations=0, converged=True, relres=0.0)
    r = b.copy()
    relres = 1.0
    its = 0
    while its < maxit and relres >= tol:
        x = x + apply_M(r)
        r = b - apply_A(x)
        relres = np.linalg.norm(r) / bnorm
        its += 1
    return x, dict(iterations=its, converged=bool(relres < tol), relres=float(relres))
