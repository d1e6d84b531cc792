"""Pin of the oracle's 3-level cycle against the matrix form of the two-grid
iteration, Eq. TG, applied recursively with dense matrices:

    E_l = S_l^nu2 (I - P_l B_{l+1} R_l A_l) S_l^nu1,   B_3 = A_3^-1,
    B_2 = (I - E_2^g) A_2^-1   (g = 1 for V, 2 for W),  cycle = (I - E_1) A_1^-1,

with S = I - w D^-1 A for damped Jacobi and
S = (I - w Pi_1 D^-1 A)(I - w Pi_0 D^-1 A) for the red-black sweep (Pi_c the
diagonal projector on colour c).  The cycle is applied to every unit vector
of a small grid and compared with that matrix.
"""
import numpy as np
import pytest

from oracle import cycle as C
from oracle import grid as G
from oracle import hierarchy as Hy


def _smoother_matrix(A, colour, kind, w):
    A = A.toarray()
    n = A.shape[0]
    Dinv = np.diag(1.0 / np.diag(A))
    I = np.eye(n)
    if kind == "jacobi":
        return I - w * Dinv @ A
    P0, P1 = np.diag((colour == 0) * 1.0), np.diag((colour == 1) * 1.0)
    return (I - w * P1 @ Dinv @ A) @ (I - w * P0 @ Dinv @ A)


@pytest.mark.parametrize("kind,cyc,nu", [("jacobi", "V", (1, 1)), ("jacobi", "W", (1, 1)),
                                         ("rb", "V", (1, 1)), ("jacobi", "V", (2, 1)),
                                         ("rb", "W", (1, 2))])
def test_cycle_equals_recursive_two_grid_matrix(kind, cyc, nu):
    rng = np.random.default_rng(11)
    grid = G.Grid([12, 16], 1.0)
    kappa2 = rng.uniform(0.3, 1.0, grid.shape)
    gamma = G.abc_profile(grid, G.uniform_widths(2, 3), 1.0)
    hier = Hy.Hierarchy(grid, kappa2, 0.6, gamma, "2nd", "fw", alpha2=1.0, alpha3=1.1)
    w = (0.8, 0.7) if kind == "jacobi" else None
    rbw = 0.9
    cy = C.Cycle(hier, cycle=cyc, nu1=nu[0], nu2=nu[1], smoother=kind,
                 weights=w if w else (0.8, 0.8), rb_weight=rbw)
    A = [a.toarray() for a in hier.A]
    R = [r.toarray() for r in hier.R]
    P = [p.toarray() for p in hier.P]
    S = [_smoother_matrix(hier.A[l], cy.colour[l], kind, w[l] if w else rbw) for l in range(2)]
    mp = np.linalg.matrix_power
    I2 = np.eye(A[1].shape[0])
    E2 = mp(S[1], nu[1]) @ (I2 - P[1] @ np.linalg.inv(A[2]) @ R[1] @ A[1]) @ mp(S[1], nu[0])
    g = 1 if cyc == "V" else 2
    B2 = (I2 - mp(E2, g)) @ np.linalg.inv(A[1])
    I1 = np.eye(A[0].shape[0])
    E1 = mp(S[0], nu[1]) @ (I1 - P[0] @ B2 @ R[0] @ A[0]) @ mp(S[0], nu[0])
    M = (I1 - E1) @ np.linalg.inv(A[0])
    cols = np.stack([cy(e) for e in np.eye(grid.size, dtype=np.complex128)], axis=1)
    np.testing.assert_allclose(cols, M, atol=1e-9 * np.max(np.abs(M)))


@pytest.mark.parametrize("order", ["2nd", "4th"])
def test_cslp_shift_of_the_cycle_operator(order):
    """RS-CGC + CSLP (Sec. 5): the cycle's fine operator is the outer operator plus
    i beta k^2 times the mass stencil.  Closed forms: for the 5-point operator the shift
    is diagonal with entries i beta omega^2 kappa^2; for the compact 4th-order operator
    (mass stencil weights summing to one) the interior row sums of the shift are
    i beta omega^2 kappa^2 in a constant medium.  The outer operator is unshifted."""
    import numpy as np
    from oracle import grid as G
    from oracle import hierarchy as Hy

    grid = G.Grid((16, 12))
    rng = np.random.default_rng(3)
    kappa2 = 1.0 + 0.0 * rng.random(grid.shape) if order == "4th" else 0.5 + rng.random(grid.shape)
    omega, beta = 0.7, 0.03
    gamma = G.abc_profile(grid, G.uniform_widths(2, 3), 1.0)
    h0 = Hy.Hierarchy(grid, kappa2, omega, gamma, order, "fw", alpha3=1.1)
    hb = Hy.Hierarchy(grid, kappa2, omega, gamma, order, "fw", alpha3=1.1, beta=beta)
    assert abs(hb.A_outer - h0.A[0]).max() == 0
    assert abs(h0.A_outer - h0.A[0]).max() == 0
    D = (hb.A[0] - hb.A_outer).toarray()
    k2 = omega**2 * kappa2.ravel()
    if order == "2nd":
        np.testing.assert_allclose(D, np.diag(1j * beta * k2), atol=1e-14)
    else:
        interior = [x + grid.nodes[0] * y for y in range(1, grid.nodes[1] - 1) for x in range(1, grid.nodes[0] - 1)]
        np.testing.assert_allclose(D.sum(axis=1)[interior], 1j * beta * k2[interior], rtol=1e-12)
        assert np.all(D.real == 0)
    # the coarse levels are built from the shifted operator: they change too
    assert abs(hb.A[1] - h0.A[1]).max() > 0 and abs(hb.A[2] - h0.A[2]).max() > 0
