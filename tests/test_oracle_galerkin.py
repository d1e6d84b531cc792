"""Pins of the oracle's grid transfers and Galerkin hierarchy.

* transfers against dense loop-built matrices and the interpolation identities
  (bilinear prolongation reproduces linear functions);
* the three-level hierarchy against a dense brute-force R2 R1 H^alpha P1 P2;
* closed-form constant-coefficient Galerkin stencils for the 5-point stencil
  with full weighting (derived from the tensor-product structure by hand, see
  the docstring of ``test_closed_form_galerkin_fw``);
* the interior rows of the sparse Galerkin products against the stencil
  convolution of the dispersion analysis (two independent computations);
* Galerkin orthogonality of the exact two-level correction;
* shift linearity, Eq. realShiftMeaning.
"""
import math

import numpy as np
import pytest

from oracle import dispersion as Dsp
from oracle import grid as G
from oracle import hierarchy as Hy
from oracle import operators as O
from oracle import transfers as T
from tests import _brute


@pytest.mark.parametrize("n,kind", [((8, 6), "fw"), ((8, 8), "cubic"), ((4, 4, 6), "fw"), ((4, 4, 4), "cubic")])
def test_restriction_matches_loops(n, kind):
    grid = G.Grid(n)
    R = T.restriction(grid, kind).toarray()
    w1 = {"fw": {-1: 0.25, 0: 0.5, 1: 0.25},
          "cubic": {-2: 1 / 16, -1: 4 / 16, 0: 6 / 16, 1: 4 / 16, 2: 1 / 16}}[kind]
    np.testing.assert_allclose(R, _brute.dense_restriction(n, w1), atol=0)
    np.testing.assert_allclose(T.prolongation(grid, kind).toarray(), 2.0**grid.dim * R.T, atol=0)


@pytest.mark.parametrize("n", [(8, 6), (4, 6, 4)])
def test_bilinear_prolongation_reproduces_linear(n):
    grid, cg = G.Grid(n), G.Grid(n).coarse()
    P = T.prolongation(grid, "fw")
    ic = np.indices(cg.shape)
    f = np.indices(grid.shape)
    coef = [0.3, -1.7, 0.9][: grid.dim]
    lin_c = 1.0 + sum(coef[k] * 2 * ic[k] for k in range(grid.dim))
    lin_f = 1.0 + sum(coef[k] * f[k] for k in range(grid.dim))
    np.testing.assert_allclose(P @ lin_c.ravel(), lin_f.ravel(), atol=1e-12)


@pytest.mark.parametrize("n,order,ig", [((8, 8), "2nd", "fw"), ((8, 8), "4th", "levdep"),
                                        ((8, 8), "4th", "cubic"), ((4, 4, 4), "2nd", "fw")])
def test_hierarchy_matches_dense_brute_force(n, order, ig):
    rng = np.random.default_rng(7)
    grid = G.Grid(n, 0.8)
    kappa2 = rng.uniform(0.2, 1.0, grid.shape)
    gamma = G.abc_profile(grid, G.uniform_widths(grid.dim, 2), 1.0)
    omega, a2, a3 = 1.3, 1.02, 1.07
    hier = Hy.Hierarchy(grid, kappa2, omega, gamma, order, ig, alpha2=a2, alpha3=a3)
    c = (omega**2 * kappa2 * (1 - 1j * gamma)).ravel()
    k2 = (omega**2 * kappa2).ravel()
    lap = O.laplacian_stencil(grid.dim, order, grid.h)
    mst = O.mass_stencil(grid.dim, order)
    H = _brute.dense_operator(n, grid.h, lap, mst, c)
    K = -_brute.dense_operator(n, grid.h, {}, mst, k2)
    w = {"fw": {-1: 0.25, 0: 0.5, 1: 0.25},
         "cubic": {-2: 1 / 16, -1: 4 / 16, 0: 6 / 16, 1: 4 / 16, 2: 1 / 16}}
    (r1, p1), (r2, p2) = {"fw": (("fw", "fw"), ("fw", "fw")), "cubic": (("cubic",) * 2, ("cubic",) * 2),
                          "levdep": (("cubic", "cubic"), ("fw", "cubic"))}[ig]
    nc = tuple(v // 2 for v in n)
    d2 = 2.0**grid.dim
    R1, P1 = _brute.dense_restriction(n, w[r1]), d2 * _brute.dense_restriction(n, w[p1]).T
    R2, P2 = _brute.dense_restriction(nc, w[r2]), d2 * _brute.dense_restriction(nc, w[p2]).T
    H2 = R1 @ (H + (1 - a2**2) * K) @ P1
    H3 = R2 @ (R1 @ (H + (1 - a3**2) * K) @ P1) @ P2
    np.testing.assert_allclose(hier.A[0].toarray(), H, atol=1e-12)
    np.testing.assert_allclose(hier.A[1].toarray(), H2, atol=1e-11)
    np.testing.assert_allclose(hier.A[2].toarray(), H3, atol=1e-10)


def test_closed_form_galerkin_fw():
    """5-point stencil, full weighting, constant k, no absorbing layer.

    In 1D, R = 1/4 [1 2 1] and P = 2 R^T give R [-1 2 -1] P = 1/4 [-1 2 -1] and
    R [1] P = [1/8 3/4 1/8]; a second coarsening maps 1/4 [-1 2 -1] to
    1/16 [-1 2 -1] and [1/8 3/4 1/8] to m3 = [5/32 11/16 5/32].  The 2D
    operators are Kronecker sums/products of these factors, so (h = grid step)
      H_2h    = ([-1 2 -1] x m2 + m2 x [-1 2 -1]) / (4 h^2)  - k^2 m2 x m2,
      H_4h^a  = ([-1 2 -1] x m3 + m3 x [-1 2 -1]) / (16 h^2) - a^2 k^2 m3 x m3.
    """
    h, k, alpha = 0.6, 0.9, 1.08
    grid = G.Grid([32, 32], h)
    hier = Hy.Hierarchy(grid, np.full(grid.shape, 1.0), k, np.zeros(grid.shape), "2nd", "fw",
                        alpha3=alpha)
    l1 = np.array([-1.0, 2.0, -1.0])
    m2 = np.array([1 / 8, 3 / 4, 1 / 8])
    m3 = np.array([5 / 32, 11 / 16, 5 / 32])
    H2 = (np.outer(m2, l1) + np.outer(l1, m2)) / (4 * h * h) - k * k * np.outer(m2, m2)
    H3 = (np.outer(m3, l1) + np.outer(l1, m3)) / (16 * h * h) - alpha**2 * k * k * np.outer(m3, m3)
    for lev, ref, node in ((1, H2, (8, 8)), (2, H3, (4, 4))):
        st = Hy.stencil_at(hier.A[lev], hier.grids[lev], node, 1)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                assert st[(dx, dy)] == pytest.approx(ref[dy + 1, dx + 1], abs=1e-13)


@pytest.mark.parametrize("dim,ig", [(2, "cubic"), (2, "levdep"), (3, "levdep")])
def test_sparse_galerkin_equals_stencil_convolution(dim, ig):
    """Interior rows of R A P (sparse products) equal the convolution stencils
    of the dispersion analysis (Sec. 4.2) for constant k."""
    G_ppw, alpha = 12, 1.0135
    kh = 2 * math.pi / G_ppw
    n = [64, 64] if dim == 2 else [32, 32, 32]
    grid = G.Grid(n, 1.0)
    hier = Hy.Hierarchy(grid, np.ones(grid.shape), kh, np.zeros(grid.shape), "4th", ig,
                        alpha3=alpha)
    s2 = Dsp.level2_stencil(dim, "4th", kh, ig, 1.0)
    s3 = Dsp.level3_stencil(dim, "4th", kh, ig, alpha)
    for lev, S in ((1, s2), (2, s3)):
        cg = hier.grids[lev]
        node = tuple(v // 2 for v in cg.n)
        rad = (S.shape[0] - 1) // 2
        st = Hy.stencil_at(hier.A[lev], cg, node, rad)
        for idx in np.ndindex(S.shape):
            off = tuple(i - rad for i in reversed(idx))
            assert st.get(off, 0.0) == pytest.approx(S[idx], abs=1e-12)


@pytest.mark.parametrize("ig", ["fw", "cubic"])
def test_two_level_galerkin_orthogonality(ig):
    """For the exact Galerkin correction x = P (R A P)^-1 R b, R (b - A x) = 0."""
    rng = np.random.default_rng(8)
    grid = G.Grid([16, 16])
    kappa2 = rng.uniform(0.3, 1.0, grid.shape)
    gamma = G.abc_profile(grid, G.uniform_widths(2, 3), 1.0)
    hier = Hy.Hierarchy(grid, kappa2, 1.1, gamma, "2nd", ig)
    A, R, P = hier.A[0], hier.R[0], hier.P[0]
    b = rng.standard_normal(grid.size) + 1j * rng.standard_normal(grid.size)
    Ac = (R @ A @ P).toarray()
    x = P @ np.linalg.solve(Ac, R @ b)
    assert np.max(np.abs(R @ (b - A @ x))) < 1e-12 * np.max(np.abs(R @ b))


def test_shift_linearity():
    """Eq. realShiftMeaning: H_4h^alpha = H_4h + (1 - alpha^2) k^2 M_4h, constant k."""
    grid = G.Grid([16, 16])
    gamma = G.abc_profile(grid, G.uniform_widths(2, 3), 1.0)
    k, alpha = 1.2, 1.05
    one = np.ones(grid.shape)
    hs = Hy.Hierarchy(grid, one, k, gamma, "4th", "cubic", alpha3=alpha)
    h0 = Hy.Hierarchy(grid, one, k, gamma, "4th", "cubic", alpha3=1.0)
    M = O.mass(grid, k * k * one, "4th")
    M4 = hs.R[1] @ (hs.R[0] @ M @ hs.P[0]) @ hs.P[1]
    diff = (hs.A[2] - (h0.A[2] + (1 - alpha**2) * M4)).toarray()
    assert np.max(np.abs(diff)) < 1e-13
