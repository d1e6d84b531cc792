"""Pins of the oracle's flexible GMRES.

* every residual estimate equals the least-squares minimum of ||b - A x|| over
  x in span(Z_j), computed from the recorded preconditioned vectors with
  numpy.linalg.lstsq (the defining property of FGMRES);
* solutions equal a dense direct solve, with and without restarts, with the
  RS-CGC cycle as preconditioner;
* a tight iteration budget reports non-convergence.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import cycle as C
from oracle import grid as G
from oracle import hierarchy as Hy
from oracle import krylov as K


def _random_system(n, seed):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 3 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b


def test_estimates_are_least_squares_minima_flexible():
    A, b = _random_system(40, 1)
    rng = np.random.default_rng(2)
    Z = []

    def M(v):  # a different preconditioner on every call: the flexible case
        Mj = np.eye(40) + 0.3 * rng.standard_normal((40, 40))
        z = Mj @ v
        Z.append(z)
        return z

    x, info = K.fgmres(lambda v: A @ v, b, M, tol=1e-30, maxit=12)
    for j, est in enumerate(info["history"], start=1):
        Zj = np.stack(Z[:j], axis=1)
        y, *_ = np.linalg.lstsq(A @ Zj, b, rcond=None)
        best = np.linalg.norm(b - A @ Zj @ y) / np.linalg.norm(b)
        assert est == pytest.approx(best, rel=1e-8)
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) == pytest.approx(info["history"][-1], rel=1e-8)


@pytest.mark.parametrize("restart", [None, 4])
def test_solution_matches_dense_solve(restart):
    A, b = _random_system(30, 3)
    x, info = K.fgmres(lambda v: A @ v, b, lambda v: v, tol=1e-13, maxit=200, restart=restart)
    assert info["converged"]
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-11 * np.linalg.norm(x))


def test_maxit_reports_not_converged():
    A, b = _random_system(30, 4)
    x, info = K.fgmres(lambda v: A @ v, b, lambda v: v, tol=1e-14, maxit=3, restart=2)
    assert info["iterations"] == 3 and not info["converged"]


@pytest.mark.parametrize("cyc", ["V", "W"])
def test_preconditioned_helmholtz_matches_direct(cyc):
    grid = G.Grid([32, 32])
    gamma = G.abc_profile(grid, G.uniform_widths(2, 4), 1.0)
    omega = 2 * np.pi / 12
    kappa2 = np.ones(grid.shape)
    hier = Hy.Hierarchy(grid, kappa2, omega, gamma, "2nd", "fw", alpha3=1.117)
    cy = C.Cycle(hier, cycle=cyc)
    b = np.zeros(grid.size, dtype=np.complex128)
    b[grid.size // 2] = 1.0
    x, info = K.fgmres(lambda v: hier.A[0] @ v, b, cy, tol=1e-12, maxit=200, restart=10)
    xd = spla.spsolve(hier.A[0].tocsc(), b)
    assert info["converged"]
    np.testing.assert_allclose(x, xd, atol=1e-9 * np.max(np.abs(xd)))


def test_stationary_exact_preconditioner_one_step():
    """With M = A^-1 the stationary iteration solves in one step."""
    import numpy as np
    from oracle import krylov as K

    rng = np.random.default_rng(1)
    A = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12)) + 6 * np.eye(12)
    b = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    Ainv = np.linalg.inv(A)
    x, info = K.stationary(lambda v: A @ v, b, lambda v: Ainv @ v, tol=1e-10, maxit=5)
    assert info["iterations"] == 1 and info["converged"]
    np.testing.assert_allclose(A @ x, b, atol=1e-10)


def test_stationary_diagonal_contraction():
    """Closed form: for A = diag(d) and M = I / d_max the residual component i after k
    steps is (1 - d_i / d_max)^k b_i."""
    import numpy as np
    from oracle import krylov as K

    d = np.array([1.0, 2.0, 4.0, 8.0])
    b = np.array([1.0, -2.0, 0.5, 3.0]) + 0j
    for k in range(1, 6):
        x, info = K.stationary(lambda v: d * v, b, lambda v: v / 8.0, tol=0.0, maxit=k)
        assert info["iterations"] == k
        np.testing.assert_allclose(b - d * x, (1 - d / 8.0) ** k * b, rtol=1e-14, atol=1e-15)
