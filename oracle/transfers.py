"""Grid-transfer operators between a grid and its every-second-node coarsening.

Oracle module (test infrastructure only).

Restriction stencils (one axis, offsets -1..1 or -2..2 in fine cells):

* ``"fw"``    full weighting 1/4 [1 2 1] (Eq. levdep; the standard transfer of the
  Remark at the end of Sec. 4);
* ``"cubic"`` 1/16 [1 4 6 4 1] (Eq. intergrid).

In d dimensions the restriction is the d-fold tensor product, centred on the
fine node 2I of coarse node I; fine nodes outside the grid are dropped.

Prolongation: the paper prints I_2h^h = 2^-d (I_h^2h)^T (Eq. intergrid).  The
coarse-grid correction P (R H P)^-1 R, the damped Jacobi iteration on the
coarse system and the zero set of every coarse symbol are unchanged when P is
scaled by a constant, so the oracle uses P = 2^d R^T, the scaling for which
bilinear interpolation maps constants to constants.
"""
import numpy as np
import scipy.sparse as sp

WEIGHTS = {
    "fw": {-1: 0.25, 0: 0.5, 1: 0.25},
    "cubic": {-2: 1.0 / 16, -1: 4.0 / 16, 0: 6.0 / 16, 1: 4.0 / 16, 2: 1.0 / 16},
}


def restriction_1d(ncells, kind):
    """(ncells/2 + 1) x (ncells + 1) restriction along one axis."""
    w = WEIGHTS[kind]
    nf = ncells + 1
    nc = ncells // 2 + 1
    rows, cols, vals = [], [], []
    for I in range(nc):
        for o, wt in w.items():
            i = 2 * I + o
            if 0 <= i < nf:
                rows.append(I)
                cols.append(i)
                vals.append(wt)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nc, nf))


def restriction(grid, kind):
    """Tensor-product restriction from ``grid`` to ``grid.coarse()``; x is the
    fastest index, so the Kronecker factors run z, y, x."""
    R = None
    for axis in reversed(range(grid.dim)):
        r1 = restriction_1d(grid.n[axis], kind)
        R = r1 if R is None else sp.kron(R, r1, format="csr")
    return R.tocsr()


def prolongation(grid, kind):
    """P = 2^d R^T for the transfer ``kind`` (see module docstring)."""
    return (2.0**grid.dim * restriction(grid, kind).T).tocsr()
