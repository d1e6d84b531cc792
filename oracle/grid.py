"""Node grids, the absorbing-layer profile and the Helmholtz coefficient.

Oracle module (test infrastructure only).

The paper discretises -Lap p - k^2 p = q, k = omega * kappa (Sec. 1, Eq.
acousitcHelm), on a regular grid padded with an absorbing layer of 20 cells
(Sec. 5).  It gives no formula for the layer; the reading used here is

    gamma(x) = gamma_max * sum_k (d_k(x) / L_k)^2,

with d_k the distance in cells into the layer of width L_k along axis k (0 in
the interior), and the layer enters as k^2 -> k^2 (1 - i gamma).

Every node of an axis with n cells (n + 1 nodes) is an unknown; values beyond
the outermost nodes are zero (Dirichlet ghost).  Arrays are C-ordered with x
fastest.
"""
import numpy as np


class Grid:
    """A tensor grid with ``n`` cells per axis (x first) and spacing ``h``."""

    def __init__(self, n, h=1.0):
        self.n = tuple(int(v) for v in n)
        if len(self.n) not in (2, 3):
            raise ValueError("2D or 3D grids only")
        self.dim = len(self.n)
        self.h = float(h)
        self.nodes = tuple(v + 1 for v in self.n)
        self.shape = tuple(reversed(self.nodes))
        self.size = int(np.prod(self.nodes))

    def coarse(self):
        """The grid of every second node (Sec. 2, h -> 2h)."""
        if any(v % 2 for v in self.n):
            raise ValueError("cell counts must be even to coarsen")
        return Grid([v // 2 for v in self.n], 2.0 * self.h)

    def __repr__(self):
        return f"Grid(n={self.n}, h={self.h})"


def abc_profile(grid, widths, gamma_max=1.0):
    """Absorbing-layer profile gamma on the nodes of ``grid``.

    ``widths`` lists (low, high) layer widths in cells per axis (x, y[, z]); a
    width of 0 puts no layer on that face (the paper leaves the top face of its
    3D runs without a layer, Sec. 5.2).
    """
    gamma = np.zeros(grid.shape)
    for axis in range(grid.dim):
        lo, hi = widths[axis]
        nc = grid.n[axis]
        i = np.arange(nc + 1, dtype=np.float64)
        term = np.zeros_like(i)
        if lo > 0:
            term += np.where(i < lo, ((lo - i) / lo) ** 2, 0.0)
        if hi > 0:
            term += np.where(i > nc - hi, ((i - (nc - hi)) / hi) ** 2, 0.0)
        bshape = [1] * grid.dim
        bshape[grid.dim - 1 - axis] = nc + 1
        gamma = gamma + term.reshape(bshape)
    return gamma_max * gamma


def uniform_widths(dim, width, free_top=False):
    """Equal layer widths on every face; with ``free_top`` the top face (low end
    of the last axis, the depth axis) has none."""
    w = [(width, width) for _ in range(dim)]
    if free_top:
        w[-1] = (0, width)
    return w


def coefficient(kappa2, omega, gamma):
    """c = k^2 (1 - i gamma) with k^2 = omega^2 kappa^2 (Eq. acousitcHelm)."""
    return (omega**2) * np.asarray(kappa2, dtype=np.float64) * (1.0 - 1j * gamma)
