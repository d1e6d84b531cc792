"""Grid-to-grid dispersion analysis and the optimal real shift (Sec. 4).

Oracle module (test infrastructure only).  It is how the real shifts handed to
the solver are chosen, and its reproduction of Tables 1-2 pins the stencil,
transfer and Galerkin composition of the oracle.

Steps, in the paper's order:
1. The constant-coefficient fine stencil H_h^alpha = -Lap_h - (alpha k)^2 M_h
   with h = 1 and k = kh = 2 pi / G (Sec. 4.1, Eq. realShift).
2. The Galerkin stencils of levels 2 and 3 by stencil convolution and
   down-sampling (Sec. 4.2): for R(I, i) = r(i - 2I), A(i, j) = a(j - i),
   P(j, J) = p(j - 2J), the coarse stencil is
   C(D) = sum_{u + v - s = 2D} r(u) a(v) p(s).
3. The symbol H~(theta) = sum_o s_o exp(i o . theta) (Eq. general_stencil).
4. The discrete radius along a ray of direction phi: the distance from the
   origin to the first sign change of the symbol (Sec. 4.1).
5. e_g(alpha, phi) = V_1 / (4 V_3) - 1 = r_3 / (4 r_1) - 1 (Eq. disp_grids_err;
   the phase speed is inversely proportional to the dimensionless radius,
   Eq. inverse_ratio).
6. alpha* = argmin_alpha max_phi |e_g(alpha, phi)| by exhaustive search
   (Eq. minmax): alpha step 5e-4, phi in [0, pi/4] every 0.1 rad in 2D; in 3D
   azimuth in [0, pi/4] and polar angle in [pi/2 - arccos(1/sqrt 3), pi/2],
   each every 0.1 rad.

Reading: the ray is sampled every 1e-3 (Sec. 4.3) and the root inside the
first bracketing interval is refined by bisection, so the radius is resolved
beyond the sampling step.
"""
import itertools
import math

import numpy as np
from scipy.signal import convolve

from . import operators
from .hierarchy import INTERGRID
from .transfers import WEIGHTS


def to_array(stencil, dim):
    """Dense, centred array of a stencil dict (axis order z, y, x)."""
    rad = max(max(abs(o) for o in off) for off in stencil)
    a = np.zeros((2 * rad + 1,) * dim, dtype=np.float64)
    for off, w in stencil.items():
        a[tuple(rad + o for o in reversed(off))] += np.real(w)
    return a


def fine_stencil(dim, order, kh, alpha=1.0):
    """Array of H_h^alpha = -Lap_h - (alpha kh)^2 M_h with h = 1 (Eq. realShift)."""
    L = to_array(operators.laplacian_stencil(dim, order, 1.0), dim)
    M = to_array(operators.mass_stencil(dim, order), dim)
    M = np.pad(M, (L.shape[0] - M.shape[0]) // 2)
    return L - (alpha * kh) ** 2 * M


def transfer_stencil(kind, dim):
    """Restriction stencil r (tensor product of the 1D weights)."""
    w1 = np.array([WEIGHTS[kind][o] for o in sorted(WEIGHTS[kind])])
    r = w1
    for _ in range(dim - 1):
        r = np.multiply.outer(r, w1)
    return r


def galerkin_stencil(a, r, p):
    """Coarse stencil C(D) = sum_{u+v-s=2D} r(u) a(v) p(s) (Sec. 4.2)."""
    ra = convolve(r, a, mode="full")
    full = convolve(ra, p[(slice(None, None, -1),) * p.ndim], mode="full")
    c = (full.shape[0] - 1) // 2
    half = c // 2
    idx = tuple(slice(c - 2 * half, c + 2 * half + 1, 2) for _ in range(full.ndim))
    return full[idx]


def level2_stencil(dim, order, kh, intergrid, alpha):
    """Stencil of I_h^2h H_h^alpha I_2h^h for constant k (Eq. Galerkin applied to
    the shifted operator of Eq. realShift)."""
    (r1, p1), _ = INTERGRID[intergrid]
    d2 = 2.0**dim
    a1 = fine_stencil(dim, order, kh, alpha)
    return galerkin_stencil(a1, transfer_stencil(r1, dim), d2 * transfer_stencil(p1, dim))


def level3_stencil(dim, order, kh, intergrid, alpha):
    """Stencil of H_4h^alpha (Eq. CoarseRealShifted) for constant k."""
    _, (r2, p2) = INTERGRID[intergrid]
    d2 = 2.0**dim
    a2 = level2_stencil(dim, order, kh, intergrid, alpha)
    return galerkin_stencil(a2, transfer_stencil(r2, dim), d2 * transfer_stencil(p2, dim))


def symbol(S, theta):
    """Real part of sum_o S[o] exp(i o . theta) for theta of shape (..., dim)
    (Eq. general_stencil); theta components ordered (x, y[, z])."""
    dim = S.ndim
    rad = (S.shape[0] - 1) // 2
    idx = np.argwhere(S != 0.0)
    w = S[tuple(idx.T)]
    offs = (idx[:, ::-1] - rad).astype(np.float64)      # (x, y[, z]) offsets
    theta = np.asarray(theta, dtype=np.float64)
    return np.cos(theta @ offs.T) @ w


def radius(S, direction, step=1e-3, bisect=True):
    """Distance from the origin to the first sign change of the symbol of S
    along the unit ``direction`` (Sec. 4.1), inside [-pi, pi]^d."""
    direction = np.asarray(direction, dtype=np.float64)
    rho_max = math.pi / np.max(np.abs(direction))
    rho = np.arange(0.0, rho_max + step / 2, step)
    vals = symbol(S, rho[:, None] * direction[None, :])
    s0 = np.sign(vals[0])
    hits = np.nonzero(np.sign(vals[1:]) != s0)[0]
    if hits.size == 0:
        return np.nan
    i = hits[0]
    lo, hi = rho[i], rho[i + 1]
    if not bisect:
        return hi
    flo = vals[i]
    for _ in range(48):
        mid = 0.5 * (lo + hi)
        fm = symbol(S, (mid * direction)[None, :])[0]
        if np.sign(fm) == np.sign(flo):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def directions(dim, res=0.1):
    """Sampled propagation directions (Sec. 4.3)."""
    if dim == 2:
        return [np.array([math.cos(p), math.sin(p)]) for p in np.arange(0.0, math.pi / 4 + 1e-12, res)]
    out = []
    lo2 = math.pi / 2 - math.acos(1.0 / math.sqrt(3.0))
    for p1 in np.arange(0.0, math.pi / 4 + 1e-12, res):
        for p2 in np.arange(lo2, math.pi / 2 + 1e-12, res):
            out.append(np.array([math.sin(p2) * math.cos(p1), math.sin(p2) * math.sin(p1), math.cos(p2)]))
    return out


def grid_to_grid_error(dim, order, G, intergrid, alpha, dirs=None, step=1e-3, bisect=True,
                       r1=None, level=3):
    """e_g(alpha, phi) for every sampled direction (Eq. disp_grids_err).

    ``level=3`` compares the fine grid with the coarsest, r_3 / (4 r_1) - 1, as
    the paper does.  ``level=2`` is the same measure between the first two grids,
    r_2 / (2 r_1) - 1, used to tune the optional level-2 shift of standard
    transfers (Remark at the end of Sec. 4)."""
    kh = 2.0 * math.pi / G
    dirs = directions(dim) if dirs is None else dirs
    if r1 is None:
        a1 = fine_stencil(dim, order, kh, 1.0)
        r1 = [radius(a1, d, step, bisect) for d in dirs]
    if level == 3:
        ac, scale = level3_stencil(dim, order, kh, intergrid, alpha), 4.0
    else:
        ac, scale = level2_stencil(dim, order, kh, intergrid, alpha), 2.0
    return np.array([radius(ac, d, step, bisect) / (scale * q) - 1.0 for d, q in zip(dirs, r1)])


def optimal_shift(dim, order, G, intergrid, alphas=None, step=1e-3, bisect=True, level=3):
    """alpha* and max_phi |e_g(alpha*, phi)| by exhaustive search (Eq. minmax)."""
    if alphas is None:
        alphas = np.round(np.arange(1.0, 1.06 + 1e-12, 5e-4), 6)
    dirs = directions(dim)
    a1 = fine_stencil(dim, order, 2.0 * math.pi / G, 1.0)
    r1 = [radius(a1, d, step, bisect) for d in dirs]
    best = (None, np.inf)
    for a in alphas:
        e = np.max(np.abs(grid_to_grid_error(dim, order, G, intergrid, a, dirs, step, bisect,
                                             r1, level)))
        if e < best[1]:
            best = (float(a), float(e))
    return best
