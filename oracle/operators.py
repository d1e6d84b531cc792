"""Fine-grid Helmholtz operators H_h = -Lap_h - k^2 M_h as sparse matrices.

Oracle module (test infrastructure only).

Stencils (offset -> weight, offsets ordered (x, y[, z])):

* ``"2nd"``: the standard second-order 5-point (2D) / 7-point (3D) Laplacian with
  the identity mass stencil, the stencil the paper compares against in Sec. 5.1.1.
* ``"4th"``: the compact fourth-order 9-point stencil of Eq. disc4thCompact (2D)
  and the 19-point stencil of Eq. disc4thCompact3D (3D), Sec. 3.1.

Reading for a variable coefficient (the paper analyses constant k only): the
mass coupling between nodes i and j uses the mean (c_i + c_j) / 2, which keeps
H complex-symmetric.  For the identity mass stencil this is simply diag(c).
Values beyond the boundary nodes are zero (Dirichlet ghost).
"""
import itertools

import numpy as np
import scipy.sparse as sp


def laplacian_stencil(dim, order, h=1.0):
    """Stencil of -Lap_h (offset tuple -> weight)."""
    s = {}
    zero = (0,) * dim
    if order == "2nd":
        s[zero] = 2.0 * dim / h**2
        for k in range(dim):
            for sgn in (-1, 1):
                off = [0] * dim
                off[k] = sgn
                s[tuple(off)] = -1.0 / h**2
        return s
    if order != "4th":
        raise ValueError(order)
    if dim == 2:
        # Eq. disc4thCompact: (1/6h^2) [[-1,-4,-1],[-4,20,-4],[-1,-4,-1]]
        table = np.array([[-1.0, -4.0, -1.0], [-4.0, 20.0, -4.0], [-1.0, -4.0, -1.0]])
        for dy, dx in itertools.product((-1, 0, 1), repeat=2):
            s[(dx, dy)] = table[dy + 1, dx + 1] / (6.0 * h**2)
        return s
    # Eq. disc4thCompact3D: -(1/6h^2) times three 3x3 slices along z
    outer = np.array([[0.0, 1.0, 0.0], [1.0, 2.0, 1.0], [0.0, 1.0, 0.0]])
    middle = np.array([[1.0, 2.0, 1.0], [2.0, -24.0, 2.0], [1.0, 2.0, 1.0]])
    slices = {-1: outer, 0: middle, 1: outer}
    for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
        w = -slices[dz][dy + 1, dx + 1] / (6.0 * h**2)
        if w != 0.0:
            s[(dx, dy, dz)] = w
    return s


def mass_stencil(dim, order):
    """Stencil of the mass operator M_h (offset tuple -> weight)."""
    zero = (0,) * dim
    if order == "2nd":
        return {zero: 1.0}
    if order != "4th":
        raise ValueError(order)
    s = {}
    centre = 8.0 if dim == 2 else 6.0  # Eqs. disc4thCompact / disc4thCompact3D
    s[zero] = centre / 12.0
    for k in range(dim):
        for sgn in (-1, 1):
            off = [0] * dim
            off[k] = sgn
            s[tuple(off)] = 1.0 / 12.0
    return s


def _pairs(grid, off):
    """Flat indices (i, j) of all node pairs with j = i + off inside the grid."""
    lo = [max(0, -o) for o in off]
    hi = [min(n, n - o) for n, o in zip(grid.nodes, off)]
    if any(b <= a for a, b in zip(lo, hi)):
        return np.zeros(0, dtype=np.int64), np.zeros(0, dtype=np.int64)
    axes = [np.arange(a, b, dtype=np.int64) for a, b in zip(lo, hi)]
    mesh = np.meshgrid(*axes, indexing="ij")
    flat = np.zeros(mesh[0].shape, dtype=np.int64)
    stride = 1
    for k in range(grid.dim):
        flat += mesh[k] * stride
        stride *= grid.nodes[k]
    stride = 1
    shift = 0
    for k in range(grid.dim):
        shift += off[k] * stride
        stride *= grid.nodes[k]
    i = flat.ravel()
    return i, i + shift


def stencil_matrix(grid, stencil, coef=None):
    """Sparse matrix with entries stencil[o] * w_ij for every in-grid pair
    j = i + o, where w_ij = (coef_i + coef_j) / 2 (1 when ``coef`` is None)."""
    rows, cols, vals = [], [], []
    cflat = None if coef is None else np.asarray(coef).ravel()
    for off, w in stencil.items():
        i, j = _pairs(grid, off)
        if cflat is None:
            v = np.full(i.shape, w, dtype=np.complex128)
        else:
            v = w * 0.5 * (cflat[i] + cflat[j])
        rows.append(i)
        cols.append(j)
        vals.append(v.astype(np.complex128))
    A = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
        shape=(grid.size, grid.size),
    )
    return A.tocsr()


def helmholtz(grid, c, order="2nd"):
    """H_h = -Lap_h - M_h[c] with c = k^2 (1 - i gamma) on the nodes (Sec. 3.1)."""
    L = stencil_matrix(grid, laplacian_stencil(grid.dim, order, grid.h))
    M = stencil_matrix(grid, mass_stencil(grid.dim, order), coef=c)
    return (L - M).tocsr()


def mass(grid, k2, order="2nd"):
    """k^2 M_h with a real k^2 field: the term the real shift scales (Eq. realShift)."""
    return stencil_matrix(grid, mass_stencil(grid.dim, order), coef=k2).tocsr()
