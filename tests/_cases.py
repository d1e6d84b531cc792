"""Shared set-up of parity cases: the same seeded medium handed to the oracle and to
the CUDA path."""
import numpy as np

import workloads
from oracle import grid as G
from oracle import hierarchy as Hy


def medium(n, seed=0, lo=0.3, hi=1.0):
    """Seeded smooth-ish slowness squared on the nodes of a grid with n cells."""
    rng = np.random.default_rng(seed)
    shape = tuple(v + 1 for v in reversed(n))
    base = rng.uniform(lo, hi, shape)
    return np.ascontiguousarray(base)


class Case:
    def __init__(self, n, omega=None, abc=3, gamma_max=1.0, alpha2=1.0, alpha3=1.0, seed=0, kappa2=None,
                 G_ppw=10.0, order="2nd", intergrid="fw", beta=0.0):
        self.order, self.intergrid = order, intergrid
        self.beta = beta
        self.n = tuple(n)
        self.dim = len(n)
        self.grid = G.Grid(self.n)
        self.kappa2 = medium(self.n, seed) if kappa2 is None else kappa2
        vmin = 1.0 / np.sqrt(self.kappa2.max())
        self.omega = workloads.omega_for_ppw(G_ppw, vmin) if omega is None else omega
        self.abc = abc
        self.widths = G.uniform_widths(self.dim, abc)
        self.gamma_max = gamma_max
        self.gamma = G.abc_profile(self.grid, self.widths, gamma_max)
        self.alpha2, self.alpha3 = alpha2, alpha3
        self._hier = None

    @property
    def hier(self):
        if self._hier is None:
            self._hier = Hy.Hierarchy(self.grid, self.kappa2, self.omega, self.gamma, self.order,
                                      self.intergrid, alpha2=self.alpha2, alpha3=self.alpha3, beta=self.beta)
        return self._hier

    def solver(self, **kw):
        import torch
        from paper_2604_19501_gb300 import Solver

        k = torch.from_numpy(self.kappa2).cuda()
        return Solver(k, self.n, self.omega, abc_width=self.abc, abc_gamma_max=self.gamma_max,
                      alpha2=self.alpha2, alpha3=self.alpha3, stencil=self.order, intergrid=self.intergrid,
                      cslp_beta=self.beta, **kw)


def rand_complex(shape, seed, dtype=np.complex128):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def stencil_to_dense(coef, r, grid):
    """Dense matrix of an assembled stencil [ncoef, nodes] on ``grid``."""
    W = 2 * r + 1
    N = grid.size
    A = np.zeros((N, N), dtype=np.complex128)
    idx = np.indices(grid.shape).reshape(grid.dim, -1)   # z, y, x order
    coords = idx[::-1]                                    # x, y, z
    flat = np.arange(N)
    strides = [1, grid.nodes[0], grid.nodes[0] * (grid.nodes[1] if grid.dim == 3 else 0)]
    for o in range(coef.shape[0]):
        off = [(o % W) - r, ((o // W) % W) - r, ((o // (W * W)) % W) - r][: grid.dim]
        ok = np.ones(N, dtype=bool)
        for a in range(grid.dim):
            c = coords[a] + off[a]
            ok &= (c >= 0) & (c < grid.nodes[a])
        j = flat + sum(off[a] * strides[a] for a in range(grid.dim))
        A[flat[ok], j[ok]] += coef[o][ok]
        assert np.all(coef[o][~ok] == 0), "out-of-grid coefficient must be zero"
    return A
