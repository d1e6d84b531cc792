"""Pins of the oracle's grid, absorbing layer and fine operators.

* the Fourier symbol of each stencil against its closed form (the standard
  2nd-order symbol; Eqs. symbol_fourth and symbol_fourth_3D for the compact
  4th-order stencils), by applying the operator to a plane wave;
* the sparse operator against a dense one built by loops over nodes;
* complex symmetry; absorbing-layer values at a few closed-form points.
"""
import math

import numpy as np
import pytest

from oracle import grid as G
from oracle import operators as O
from tests import _brute


def _plane_wave(grid, theta):
    idx = np.indices(grid.shape)  # z, y, x order
    phase = sum(theta[k] * idx[grid.dim - 1 - k] for k in range(grid.dim))
    return np.exp(1j * phase), idx


def _interior(grid, idx, margin=1):
    m = np.ones(grid.shape, dtype=bool)
    for a in range(grid.dim):
        m &= (idx[a] >= margin) & (idx[a] <= grid.shape[a] - 1 - margin)
    return m.ravel()


@pytest.mark.parametrize("dim", [2, 3])
def test_second_order_symbol(dim):
    """(A u)_j = ((2d - 2 sum cos theta_k)/h^2 - k^2) u_j on interior nodes."""
    rng = np.random.default_rng(1)
    h, k2 = 0.7, 1.3
    grid = G.Grid([8] * dim, h)
    A = O.helmholtz(grid, np.full(grid.shape, k2), "2nd")
    for _ in range(3):
        theta = rng.uniform(-math.pi, math.pi, dim)
        u, idx = _plane_wave(grid, theta)
        Au = A @ u.ravel()
        sym = (2 * dim - 2 * np.sum(np.cos(theta))) / h**2 - k2
        m = _interior(grid, idx)
        np.testing.assert_allclose(Au[m], sym * u.ravel()[m], rtol=0, atol=1e-12)


def test_fourth_order_symbol_2d():
    """Eq. symbol_fourth."""
    rng = np.random.default_rng(2)
    h, k = 0.9, 1.1
    grid = G.Grid([8, 10], h)
    A = O.helmholtz(grid, np.full(grid.shape, k * k), "4th")
    kh2 = (k * h) ** 2
    for _ in range(3):
        t1, t2 = rng.uniform(-math.pi, math.pi, 2)
        u, idx = _plane_wave(grid, (t1, t2))
        sym = (10 / 3 - 2 / 3 * kh2 - (4 / 3 + kh2 / 6) * (math.cos(t1) + math.cos(t2))
               - 2 / 3 * math.cos(t1) * math.cos(t2)) / h**2
        m = _interior(grid, idx)
        np.testing.assert_allclose((A @ u.ravel())[m], sym * u.ravel()[m], atol=1e-12)


def test_fourth_order_symbol_3d():
    """Eq. symbol_fourth_3D."""
    rng = np.random.default_rng(3)
    h, k = 1.2, 0.8
    grid = G.Grid([6, 6, 8], h)
    A = O.helmholtz(grid, np.full(grid.shape, k * k), "4th")
    kh2 = (k * h) ** 2
    for _ in range(3):
        t = rng.uniform(-math.pi, math.pi, 3)
        u, idx = _plane_wave(grid, t)
        c = np.cos(t)
        sym = (4 - kh2 / 2 - (2 / 3 + kh2 / 6) * c.sum()
               - 2 / 3 * (c[0] * c[1] + c[0] * c[2] + c[1] * c[2])) / h**2
        m = _interior(grid, idx)
        np.testing.assert_allclose((A @ u.ravel())[m], sym * u.ravel()[m], atol=1e-12)


def _lap2nd(dim, h):
    s = {(0,) * dim: 2 * dim / h**2}
    for k in range(dim):
        for sg in (-1, 1):
            o = [0] * dim
            o[k] = sg
            s[tuple(o)] = -1 / h**2
    return s


@pytest.mark.parametrize("n,order", [((6, 4), "2nd"), ((4, 4, 2), "2nd"), ((6, 4), "4th")])
def test_operator_matches_dense_loops(n, order):
    rng = np.random.default_rng(4)
    grid = G.Grid(n, 0.5)
    c = rng.uniform(0.5, 2, grid.shape) * (1 - 1j * rng.uniform(0, 1, grid.shape))
    A = O.helmholtz(grid, c, order).toarray()
    if order == "2nd":
        lap, mass = _lap2nd(grid.dim, grid.h), {(0,) * grid.dim: 1.0}
    else:  # the 9-point stencil, typed from Eq. disc4thCompact
        t = [[-1, -4, -1], [-4, 20, -4], [-1, -4, -1]]
        lap = {(dx, dy): t[dy + 1][dx + 1] / (6 * grid.h**2) for dx in (-1, 0, 1) for dy in (-1, 0, 1)}
        mass = {(0, 0): 8 / 12, (1, 0): 1 / 12, (-1, 0): 1 / 12, (0, 1): 1 / 12, (0, -1): 1 / 12}
    B = _brute.dense_operator(n, grid.h, lap, mass, c.ravel())
    np.testing.assert_allclose(A, B, atol=1e-13)


@pytest.mark.parametrize("order,dim", [("2nd", 2), ("2nd", 3), ("4th", 2), ("4th", 3)])
def test_complex_symmetric(order, dim):
    rng = np.random.default_rng(5)
    grid = G.Grid([4] * dim)
    c = rng.uniform(0.5, 2, grid.shape) * (1 - 1j * rng.uniform(0, 1, grid.shape))
    A = O.helmholtz(grid, c, order)
    assert abs(A - A.T).max() == 0.0


def test_abc_profile_values():
    grid = G.Grid([20, 12])
    g = G.abc_profile(grid, G.uniform_widths(2, 4), gamma_max=2.0)
    assert g[6, 10] == 0.0                       # interior
    assert g[6, 0] == pytest.approx(2.0)         # x = 0 face: d = L
    assert g[0, 0] == pytest.approx(4.0)         # corner: two faces
    assert g[6, 1] == pytest.approx(2.0 * (3 / 4) ** 2)
    assert g[6, 20] == pytest.approx(2.0)        # x = N face
    assert g[6, 17] == pytest.approx(2.0 * (1 / 4) ** 2)
    gf = G.abc_profile(grid, G.uniform_widths(2, 4, free_top=True), gamma_max=2.0)
    assert gf[0, 10] == 0.0 and gf[12, 10] == pytest.approx(2.0)


def test_coefficient_sign():
    c = G.coefficient(np.array([2.0]), 3.0, np.array([0.5]))
    assert c[0] == pytest.approx(18.0 * (1 - 0.5j))
