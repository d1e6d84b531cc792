"""Pin of the oracle's adjoint gradient against central finite differences of
the misfit (independent forward solves with a sparse direct solver)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import adjoint as Ad
from oracle import grid as G
from oracle import operators as O


@pytest.mark.parametrize("order", ["2nd", "4th"])
def test_gradient_matches_central_differences(order):
    rng = np.random.default_rng(21)
    grid = G.Grid([14, 12])
    gamma = G.abc_profile(grid, G.uniform_widths(2, 3), 1.0)
    omega = 0.7
    m = rng.uniform(0.3, 1.0, grid.shape)
    ns = 2
    q = np.zeros((ns,) + grid.shape, dtype=np.complex128)
    q[0, 6, 4] = 1.0
    q[1, 5, 9] = 1.0
    mask = np.zeros(grid.shape, dtype=bool)
    mask[0, :] = True
    d = (rng.standard_normal((ns,) + grid.shape) + 1j * rng.standard_normal((ns,) + grid.shape)) * 0.1

    def solve_all(mm, rhs):
        A = O.helmholtz(grid, G.coefficient(mm, omega, gamma), order).tocsc()
        return np.stack([spla.spsolve(A, r.ravel()).reshape(grid.shape) for r in rhs])

    def loss(mm):
        return Ad.misfit(solve_all(mm, q), d, mask)

    p = solve_all(m, q)
    mu = solve_all(m, Ad.adjoint_rhs(p, d, mask))
    g = Ad.gradient(grid, omega, gamma, p, mu, order)
    for j in [(3, 3), (6, 7), (1, 1), (10, 5), (0, 7)]:
        step = 1e-4 * m[j]
        mp, mm_ = m.copy(), m.copy()
        mp[j] += step
        mm_[j] -= step
        fd = (loss(mp) - loss(mm_)) / (2 * step)
        assert g[j] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.max(np.abs(g)))


def test_dot_product_symmetry():
    """<A x, y> = <x, A y> without conjugation (A = A^T)."""
    rng = np.random.default_rng(22)
    grid = G.Grid([10, 10])
    c = rng.uniform(0.5, 1, grid.shape) * (1 - 0.3j)
    A = O.helmholtz(grid, c, "4th")
    x = rng.standard_normal(grid.size) + 1j * rng.standard_normal(grid.size)
    y = rng.standard_normal(grid.size) + 1j * rng.standard_normal(grid.size)
    assert np.sum((A @ x) * y) == pytest.approx(np.sum(x * (A @ y)), rel=1e-13)
