"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module holds no arithmetic of the solver: it only draws media (slowness
fields), point sources and receiver masks.  Both the oracle and the GPU path
receive these arrays as plain inputs.

Grid convention (shared by every consumer): an axis with ``n`` cells has
``n + 1`` nodes; arrays are C-ordered with x fastest, i.e. shape ``(ny+1, nx+1)``
in 2D and ``(nz+1, ny+1, nx+1)`` in 3D.  Depth is the y axis in 2D and the z axis
in 3D, and index 0 on that axis is the top surface.

The media stand in for the geophysical models the paper uses (Marmousi, the
SEG/EAGE Overthrust, linear and wedge models, Section 5), which are not
reproduced here.
"""
import math

import numpy as np

__all__ = [
    "omega_for_ppw",
    "constant_medium",
    "layered_faulted_2d",
    "layered_3d",
    "linear_2d",
    "wedge_2d",
    "point_source",
    "surface_sources",
]


def omega_for_ppw(G, v_min, h=1.0):
    """Angular frequency giving ``G`` grid points per wavelength at the slowest
    velocity: k_max h = omega h / v_min = 2 pi / G (Section 4.1, r = kh = 2 pi / G)."""
    return 2.0 * math.pi * v_min / (G * h)


def constant_medium(n, velocity=1.0):
    """Slowness squared (kappa^2 = 1/v^2) of a homogeneous medium on a grid with
    ``n`` cells per axis."""
    shape = tuple(int(v) + 1 for v in reversed(tuple(n)))
    return np.full(shape, 1.0 / velocity**2, dtype=np.float64)


def _smooth_noise(rng, shape, sigma):
    from scipy.ndimage import gaussian_filter

    xi = gaussian_filter(rng.standard_normal(shape), sigma=sigma, mode="reflect")
    return xi / np.max(np.abs(xi))


def layered_faulted_2d(n_interior, pad, seed=0, v_range=(1.5, 4.5), n_layers=8,
                       n_faults=3, blob=True, noise=0.05, sigma=8.0):
    """Seeded 2D layered medium with dipping faults, one fast elliptical blob and
    a Gaussian-smoothed multiplicative perturbation.

    ``n_interior`` cells per axis inside the absorbing layer, ``pad`` cells of
    padding on every side filled by edge extension.  Returns kappa^2 = 1/v^2 on
    the nodes of the padded grid, shape ``(N+1, N+1)`` with ``N = n_interior +
    2 pad``.
    """
    rng = np.random.default_rng(seed)
    m = int(n_interior) + 1
    vmin, vmax = v_range
    x = np.linspace(0.0, 1.0, m)[None, :]
    z = np.linspace(0.0, 1.0, m)[:, None]
    # layer interfaces: sorted depths with a small random dip each
    depths = np.sort(rng.uniform(0.06, 0.94, n_layers - 1))
    dips = rng.uniform(-0.08, 0.08, n_layers - 1)
    vel_layers = np.sort(rng.uniform(vmin, 0.9 * vmax, n_layers))
    vel_layers[0] = vmin
    # faults: a line x = x0 + (z - 0.5) tan(dip); on its right the stack drops by a throw
    shift = np.zeros((m, m))
    for _ in range(n_faults):
        x0 = rng.uniform(0.15, 0.85)
        tan_dip = math.tan(math.radians(rng.uniform(-30.0, 30.0)))
        throw = rng.uniform(0.02, 0.08)
        shift += np.where(x > x0 + (z - 0.5) * tan_dip, throw, 0.0)
    zz = z - shift
    layer = np.zeros((m, m), dtype=np.int64)
    for d, s in zip(depths, dips):
        layer += (zz > d + s * (x - 0.5)).astype(np.int64)
    v = vel_layers[layer]
    if blob:
        cx, cz = rng.uniform(0.3, 0.7), rng.uniform(0.45, 0.8)
        ax, az = rng.uniform(0.06, 0.12), rng.uniform(0.03, 0.07)
        v = np.where(((x - cx) / ax) ** 2 + ((z - cz) / az) ** 2 <= 1.0, vmax, v)
    if noise > 0:
        v = v * (1.0 + noise * _smooth_noise(rng, (m, m), sigma))
    v = np.clip(v, vmin, vmax)
    v = np.pad(v, int(pad), mode="edge")
    return (1.0 / v**2).astype(np.float64)


def layered_3d(n_interior, pad, seed=0, v_range=(1.5, 4.5), n_layers=8,
               noise=0.05, sigma=8.0):
    """Seeded 3D analogue of :func:`layered_faulted_2d`: dipping layers with
    velocity increasing with depth (z) and a smoothed multiplicative
    perturbation.  ``n_interior`` is a 3-tuple of interior cells (nx, ny, nz)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = (int(v) + 1 for v in n_interior)
    vmin, vmax = v_range
    x = np.linspace(0.0, 1.0, nx)[None, None, :]
    y = np.linspace(0.0, 1.0, ny)[None, :, None]
    z = np.linspace(0.0, 1.0, nz)[:, None, None]
    depths = np.sort(rng.uniform(0.06, 0.94, n_layers - 1))
    dx = rng.uniform(-0.08, 0.08, n_layers - 1)
    dy = rng.uniform(-0.08, 0.08, n_layers - 1)
    vel_layers = np.sort(rng.uniform(vmin, vmax, n_layers))
    vel_layers[0] = vmin
    layer = np.zeros((nz, ny, nx), dtype=np.int64)
    for d, sx, sy in zip(depths, dx, dy):
        layer += (z > d + sx * (x - 0.5) + sy * (y - 0.5)).astype(np.int64)
    v = vel_layers[layer]
    if noise > 0:
        v = v * (1.0 + noise * _smooth_noise(rng, (nz, ny, nx), sigma))
    v = np.clip(v, vmin, vmax)
    v = np.pad(v, int(pad), mode="edge")
    return (1.0 / v**2).astype(np.float64)


def _unit_square(n_interior):
    """Node coordinates (x, z) of an ``n_interior``-cell grid on the unit square."""
    t = np.linspace(0.0, 1.0, int(n_interior) + 1)
    return np.meshgrid(t, t, indexing="xy")


def linear_2d(n_interior, pad, kappa_min=0.5, kappa_max=1.0):
    """The linear model of Section 5 (heterogeneous 2D media): slowness kappa varying
    linearly with depth over the unit square, from ``kappa_max`` at the surface to
    ``kappa_min`` at the bottom (velocity increasing with depth), padded by edge
    extension.  Returns kappa^2 on the nodes, shape ``(N+1, N+1)``,
    ``N = n_interior + 2 pad``."""
    _, z = _unit_square(n_interior)
    kappa = kappa_max + (kappa_min - kappa_max) * z
    return np.pad(kappa, int(pad), mode="edge") ** 2


def wedge_2d(n_interior, pad, kappa_min=0.5, kappa_max=1.0):
    """A wedge model for Section 5 (heterogeneous 2D media): three regions of constant
    slowness on the unit square separated by two straight interfaces,
    z1(x) = 0.4 + 0.2 x and z2(x) = 0.8 - 0.4 x, which meet at x = 2/3 and enclose a
    wedge of the slowest material (``kappa_max``) on the left.  Above the wedge the
    slowness is (kappa_min + kappa_max) / 2, below it ``kappa_min`` (for [0.5, 1] the
    slowness ratios of 2000 / 1500 / 3000 m/s layers).  Padded by edge extension;
    returns kappa^2 on the nodes, shape ``(N+1, N+1)``."""
    x, z = _unit_square(n_interior)
    z1 = 0.4 + 0.2 * x
    z2 = 0.8 - 0.4 * x
    kappa = np.where(z < z1, 0.5 * (kappa_min + kappa_max), kappa_min)
    kappa = np.where((z >= z1) & (z < z2), kappa_max, kappa)
    return np.pad(kappa, int(pad), mode="edge") ** 2


def point_source(n, h=1.0, node=None):
    """Unit point source q = e_c / h^d at ``node`` (default: the centre node) on a
    grid with ``n`` cells per axis; complex128 array in the grid layout."""
    n = tuple(int(v) for v in n)
    shape = tuple(v + 1 for v in reversed(n))
    q = np.zeros(shape, dtype=np.complex128)
    if node is None:
        node = tuple(v // 2 for v in n)
    q[tuple(reversed(tuple(node)))] = 1.0 / h ** len(n)
    return q


def surface_sources(n, count, pad, seed=0, h=1.0, depth=None):
    """``count`` point sources at seeded distinct positions along the top of the
    interior (depth index ``pad`` unless ``depth`` is given), returned as a
    complex128 array of shape ``(count,) + grid shape``."""
    n = tuple(int(v) for v in n)
    rng = np.random.default_rng(seed)
    dim = len(n)
    shape = tuple(v + 1 for v in reversed(n))
    d = pad if depth is None else depth
    q = np.zeros((count,) + shape, dtype=np.complex128)
    lateral = [np.arange(pad, n[k] - pad + 1) for k in range(dim - 1)]
    for s in range(count):
        pos = [int(rng.choice(lat)) for lat in lateral]
        node = tuple(pos) + (d,)
        q[(s,) + tuple(reversed(node))] = 1.0 / h**dim
    return q
