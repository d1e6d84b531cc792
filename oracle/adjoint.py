"""Least-squares misfit and its gradient with respect to the slowness squared
m = kappa^2, by the adjoint-state method.

Oracle module (test infrastructure only).  The paper has no adjoint; this is the
standard derivation for the operator of Sec. 3.1:

    L(m) = 1/2 sum_s || P_r p_s - d_s ||^2,   H(m) p_s = q_s,
    H(m) = -Lap_h - omega^2 M_h[m (1 - i gamma)].

With H^H lambda_s = P_r^T (P_r p_s - d_s):  dL/dm_j = -Re(lambda_s^H dH/dm_j p_s).
H is complex-symmetric, so H^H = conj(H) and mu_s = conj(lambda_s) solves
H mu_s = conj(P_r^T (P_r p_s - d_s)) with the same solver.  For the identity
mass stencil dH/dm_j = -omega^2 (1 - i gamma_j) e_j e_j^T, so

    dL/dm_j = omega^2 sum_s Re((1 - i gamma_j) mu_{s,j} p_{s,j}).

For a mass stencil with neighbours (coefficient mean (c_i + c_j)/2 on each
coupling) the same steps give
    dL/dm_j = omega^2 sum_s Re((1 - i gamma_j) sum_o w_o (mu_j p_{j+o} + mu_{j+o} p_j) / 2).
"""
import numpy as np

from . import operators


def misfit(p, d, mask):
    """1/2 sum over sources of || P_r p_s - d_s ||^2 (receivers where ``mask``)."""
    r = (np.asarray(p) - np.asarray(d))[..., mask]
    return 0.5 * float(np.sum(np.abs(r) ** 2))


def adjoint_rhs(p, d, mask):
    """conj(P_r^T (P_r p - d)) on the full grid (zero off the receivers)."""
    g = np.where(mask, np.asarray(p) - np.asarray(d), 0.0)
    return np.conj(g)


def gradient(grid, omega, gamma, p, mu, order="2nd"):
    """dL/dm on the nodes from forward fields ``p`` and adjoint fields ``mu``
    (both shaped (sources,) + grid.shape)."""
    one_m_ig = (1.0 - 1j * np.asarray(gamma)).ravel()
    st = operators.mass_stencil(grid.dim, order)
    g = np.zeros(grid.size)
    for ps, ms in zip(np.reshape(p, (-1, grid.size)), np.reshape(mu, (-1, grid.size))):
        acc = np.zeros(grid.size, dtype=np.complex128)
        for off, w in st.items():
            i, j = operators._pairs(grid, off)
            acc[i] += 0.5 * w * (ms[i] * ps[j] + ms[j] * ps[i])
        g += omega**2 * np.real(one_m_ig * acc)
    return g.reshape(grid.shape)
