"""Point relaxations used as smoothers (Sec. 2: damped Jacobi; red-black
ordering as the second point smoother).

Oracle module (test infrastructure only).
"""
import numpy as np


def jacobi(A, diag, x, b, weight):
    """One damped-Jacobi sweep x <- x + w D^-1 (b - A x), D = diag(A)."""
    return x + weight * (b - A @ x) / diag


def colours(grid):
    """Checkerboard colour (sum of node indices mod 2) of every node, flat."""
    idx = np.indices(grid.shape)
    return (idx.sum(axis=0) % 2).ravel()


def red_black(A, diag, x, b, colour, weight=1.0):
    """One red-black sweep: every colour-0 node is updated simultaneously from
    the current x by x_i <- x_i + w (b - A x)_i / a_ii, then every colour-1 node
    from the updated x.  With the 5/7-point stencil this is Gauss-Seidel in
    red-black order; on wider coarse stencils same-coloured nodes couple and the
    simultaneous update keeps the sweep order-independent."""
    x = np.array(x, dtype=np.complex128, copy=True)
    for col in (0, 1):
        m = colour == col
        r = b - A @ x
        x[m] = x[m] + weight * r[m] / diag[m]
    return x
