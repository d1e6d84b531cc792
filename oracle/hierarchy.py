"""The three-level operator hierarchy of RS-CGC.

Oracle module (test infrastructure only).

* Level 1: H_h = -Lap_h - k^2 M_h with the absorbing layer (Sec. 3.1).
* Level 2: the Galerkin operator H_2h = I_h^2h H_h I_2h^h (Eq. Galerkin).
  An optional real shift alpha2 on this level, H_2h = I_h^2h H_h^alpha2 I_2h^h,
  is the variant the Remark at the end of Sec. 4 says standard (bilinear)
  transfers would need; alpha2 = 1 is the paper's method.
* Level 3: the real-shifted coarsest operator
  H_4h^alpha = I_2h^4h (I_h^2h H_h^alpha I_2h^h) I_4h^2h      (Eq. CoarseRealShifted)
  with H_h^alpha = H_h + (1 - alpha^2) k^2 M_h                 (Eq. realShift).

Reading: the real shift scales k^2 = omega^2 kappa^2 only, not the absorbing
term i gamma k^2 (the literal Eq. realShift with H_h including the layer).

RS-CGC + CSLP (Sec. 5, second experiment: the combination suggested for 10 points
per wavelength, with a complex shift of 0.03 k^2): with beta > 0 the cycle's
operators are built from the complex-shifted fine operator
H_h^beta = -Lap_h - k^2 (1 - i gamma - i beta) M_h = H_h + i beta K,
the shift entering like the absorbing term; the outer (Krylov) operator stays H_h.
The real shift of level 3 then acts on H_h^beta.

Transfers per level ("intergrid"):
  "fw"     full weighting / bilinear on both levels;
  "cubic"  Eq. intergrid on both levels;
  "levdep" Eq. intergrid between levels 1 and 2 and for the prolongation from
           level 3, full weighting (Eq. levdep) for the restriction to level 3.
The operators are built in the paper's order: shift the fine operator, then
coarsen twice with sparse matrix products.
"""
import numpy as np
import scipy.sparse as sp

from . import grid as grid_mod
from . import operators, transfers

INTERGRID = {
    "fw": (("fw", "fw"), ("fw", "fw")),
    "cubic": (("cubic", "cubic"), ("cubic", "cubic")),
    "levdep": (("cubic", "cubic"), ("fw", "cubic")),
}


class Hierarchy:
    """Operators of the 3-level RS-CGC method for one medium and frequency.

    Parameters: ``grid`` (:class:`Grid`), ``kappa2`` slowness squared on the
    nodes, ``omega`` angular frequency, ``gamma`` absorbing-layer profile,
    ``order`` "2nd" | "4th", ``intergrid`` "fw" | "cubic" | "levdep",
    ``alpha2`` / ``alpha3`` real shifts of levels 2 and 3, ``beta`` the complex
    shift of the cycle (0: plain RS-CGC).  ``A[0]`` is the cycle's fine operator,
    ``A_outer`` the operator the outer iteration solves.
    """

    def __init__(self, grid, kappa2, omega, gamma, order="2nd", intergrid="fw",
                 alpha2=1.0, alpha3=1.0, beta=0.0):
        self.grids = [grid, grid.coarse(), grid.coarse().coarse()]
        self.omega = float(omega)
        self.order = order
        self.gamma = np.asarray(gamma, dtype=np.float64)
        self.kappa2 = np.asarray(kappa2, dtype=np.float64)
        c = grid_mod.coefficient(self.kappa2, omega, self.gamma)
        k2 = omega**2 * self.kappa2
        H1 = operators.helmholtz(grid, c, order)
        K1 = operators.mass(grid, k2, order)
        self.A_outer = H1.tocsr()
        if beta != 0.0:
            # the complex shift enters like the absorbing term: gamma -> gamma + beta
            c_beta = grid_mod.coefficient(self.kappa2, omega, self.gamma + beta)
            H1 = operators.helmholtz(grid, c_beta, order)
        (r1, p1), (r2, p2) = INTERGRID[intergrid]
        self.R = [transfers.restriction(self.grids[0], r1),
                  transfers.restriction(self.grids[1], r2)]
        self.P = [transfers.prolongation(self.grids[0], p1),
                  transfers.prolongation(self.grids[1], p2)]
        H1_a2 = H1 + (1.0 - alpha2**2) * K1          # Eq. realShift (level-2 variant)
        H1_a3 = H1 + (1.0 - alpha3**2) * K1          # Eq. realShift
        H2 = (self.R[0] @ H1_a2 @ self.P[0]).tocsr()  # Eq. Galerkin
        H2_a3 = (self.R[0] @ H1_a3 @ self.P[0]).tocsr()
        H3 = (self.R[1] @ H2_a3 @ self.P[1]).tocsr()  # Eq. CoarseRealShifted
        self.A = [H1.tocsr(), H2, H3]
        self.K1 = K1
        self.diag = [A.diagonal() for A in self.A]
        self._lu = None

    @property
    def coarsest_lu(self):
        """Sparse LU of the coarsest operator (the exact coarse solve of Sec. 2)."""
        if self._lu is None:
            import scipy.sparse.linalg as spla

            self._lu = spla.splu(self.A[2].tocsc())
        return self._lu

    def coarse_solve(self, b):
        return self.coarsest_lu.solve(np.asarray(b, dtype=np.complex128))


def stencil_at(A, grid, node, radius):
    """Coefficients of row ``node`` (a grid index tuple, x first) of the sparse
    operator ``A`` as a dict offset -> value within ``radius``; a helper for
    reading assembled coarse stencils."""
    flat = 0
    stride = 1
    for k in range(grid.dim):
        flat += node[k] * stride
        stride *= grid.nodes[k]
    row = A.getrow(flat)
    out = {}
    for j, v in zip(row.indices, row.data):
        rem = j
        off = []
        for k in range(grid.dim):
            off.append(rem % grid.nodes[k] - node[k])
            rem //= grid.nodes[k]
        if max(abs(o) for o in off) <= radius:
            out[tuple(off)] = v
    return out
