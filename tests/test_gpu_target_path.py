"""The mixed-precision batched forward + adjoint path against the oracle.

A mixed-precision context (FP32 cycle; double-float Krylov basis, true residual and
coarsest solve) with blocks of four right-hand sides solves six surface sources (a full
block and a ragged block of two) and then runs helm_adjoint_grad on the receiver
residuals.  The paper has no adjoint; the pins are the oracle's adjoint-state gradient
from direct (SuperLU) solves of the oracle operator, and central finite differences of
the misfit, which involve no adjoint at all.

Tolerances:
* forward solves to 1e-6: per source, the oracle FGMRES count +-1 and the field within
  1e-5 (the perturbation of the preconditioner by the cycle's FP32 arithmetic);
* solves to 1e-10: fields and gradient within 1e-7 of the oracle's exact solves.  The
  outer iteration refines in double-float (about 48 bits) to a true residual of 1e-10;
  the error of the field is that residual amplified by the operator's conditioning on
  these grids (below 1e3), well under 1e-7;
* finite differences: step 1e-4 relative, solves to 1e-10, agreement to 1e-4 relative
  or 1e-5 of the largest gradient entry (the solve tolerance divided by the step bounds
  the noise of a difference quotient).
"""
import numpy as np
import pytest

import workloads
from oracle import adjoint as OA
from oracle import cycle as OC
from oracle import krylov as OK
from tests._cases import Case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(n, nsrc, seed, pad=8):
    rng = np.random.default_rng(seed)
    if len(n) == 2:
        kappa2 = workloads.layered_faulted_2d(n[0] - 2 * pad, pad, seed=seed, sigma=2.0)
        order, ig, alpha3 = "4th", "cubic", 1.0045
    else:
        kappa2 = workloads.layered_3d([v - 2 * pad for v in n], pad, seed=seed, sigma=2.0)
        order, ig, alpha3 = "4th", "levdep", 1.012
    c = Case(n, abc=pad, alpha3=alpha3, kappa2=kappa2, G_ppw=12, order=order, intergrid=ig)
    q = workloads.surface_sources(n, nsrc, pad, seed=seed)
    mask = np.zeros(c.grid.shape, dtype=bool)
    if len(n) == 2:
        mask[pad, pad:n[0] - pad + 1] = True
    else:
        mask[pad, pad:n[1] - pad + 1, pad:n[0] - pad + 1] = True
    d = (rng.standard_normal(q.shape) + 1j * rng.standard_normal(q.shape)) * 0.01 * mask
    return c, q, mask, d


def _weights(c):
    return (0.89, 0.89) if c.dim == 2 else (0.6, 0.4)


def _direct(c, rhs):
    import scipy.sparse.linalg as spla

    lu = spla.splu(c.hier.A_outer.tocsc())
    return np.stack([lu.solve(r.ravel()).reshape(r.shape) for r in rhs])


@pytest.mark.parametrize("n", [(96, 96), (24, 24, 16)])
def test_mixed_block_forward_matches_oracle_fgmres(n):
    c, q, mask, d = _problem(n, 6, seed=21, pad=6)
    s = c.solver(precision="mixed", max_rhs=4, jacobi_w=_weights(c))
    p, st = s.solve(torch.from_numpy(q).cuda(), tol=1e-6, maxit=400)
    torch.cuda.synchronize()
    pn = p.cpu().numpy()
    s.close()
    cy = OC.Cycle(c.hier, weights=_weights(c))
    for k in range(q.shape[0]):
        xo, info = OK.fgmres(lambda v: c.hier.A_outer @ v, q[k].ravel(), cy, tol=1e-6, maxit=400, restart=10)
        print(k, "oracle", info["iterations"], "gpu", st[k]["iterations"], "rel", rel(pn[k].ravel(), xo))
        assert st[k]["converged"] and info["converged"]
        assert abs(st[k]["iterations"] - info["iterations"]) <= 1
        assert rel(pn[k].ravel(), xo) < 1e-5


@pytest.mark.parametrize("n", [(128, 128), (24, 24, 16)])
def test_mixed_block_adjoint_gradient_matches_oracle(n):
    c, q, mask, d = _problem(n, 6, seed=23, pad=6)
    s = c.solver(precision="mixed", max_rhs=4, jacobi_w=_weights(c))
    qd = torch.from_numpy(q).cuda()
    p, st = s.solve(qd, tol=1e-10, maxit=600)
    assert all(a["converged"] for a in st)
    pn = p.cpu().numpy()
    resid = np.where(mask, pn - d, 0.0)
    grad = torch.zeros(c.grid.shape, dtype=torch.float64, device="cuda")
    adj = torch.empty_like(p)
    ast = s.adjoint_grad(p, torch.from_numpy(resid).cuda(), grad, adj, tol=1e-10, maxit=600)
    torch.cuda.synchronize()
    s.close()
    assert all(a["converged"] for a in ast)
    po = _direct(c, q)
    mu = _direct(c, OA.adjoint_rhs(po, d, mask))
    go = OA.gradient(c.grid, c.omega, c.gamma, po, mu, "4th")
    e_p, e_mu, e_g = rel(pn, po), rel(adj.cpu().numpy(), mu), rel(grad.cpu().numpy(), go)
    print("forward", e_p, "adjoint", e_mu, "gradient", e_g, [a["iterations"] for a in st],
          [a["iterations"] for a in ast])
    assert e_p < 1e-7 and e_mu < 1e-7 and e_g < 1e-7


def _fd_check(n, nsrc, nodes, seed, pad):
    from paper_2604_19501_gb300 import helmholtz_solve

    c, q, mask, d = _problem(n, nsrc, seed=seed, pad=pad)
    opts = dict(abc_width=c.abc, alpha3=c.alpha3, stencil="4th", intergrid=c.intergrid, jacobi_w=_weights(c),
                precision="mixed", max_rhs=nsrc)
    qd = torch.from_numpy(q).cuda()
    dd = torch.from_numpy(d).cuda()
    mk = torch.from_numpy(mask).cuda()

    def loss(k2):
        p = helmholtz_solve(k2, qd, n, c.omega, tol=1e-10, maxit=800, **opts)
        r = torch.where(mk, p - dd, torch.zeros_like(p))
        return 0.5 * (r.abs() ** 2).sum()

    k2 = torch.from_numpy(c.kappa2.copy()).cuda().requires_grad_(True)
    loss(k2).backward()
    g = k2.grad.cpu().numpy()
    gmax = np.max(np.abs(g))
    worst = 0.0
    for j in nodes:
        h = 1e-4 * c.kappa2[j]
        kp = c.kappa2.copy()
        km = c.kappa2.copy()
        kp[j] += h
        km[j] -= h
        with torch.no_grad():
            fd = (loss(torch.from_numpy(kp).cuda()).item() - loss(torch.from_numpy(km).cuda()).item()) / (2 * h)
        worst = max(worst, abs(g[j] - fd) / max(abs(fd), 1e-300))
        assert g[j] == pytest.approx(fd, rel=1e-4, abs=1e-5 * gmax), (j, g[j], fd)
    print("largest relative FD difference", worst, "max |g|", gmax)


def test_mixed_gradient_central_differences_2d_full_size():
    """The differentiation workload's 2D size: 512^2 interior cells + a 32-cell layer
    (576^2), 16 surface sources as one block, receivers on the top interior row, 20
    seeded interior nodes."""
    n = (576, 576)
    rng = np.random.default_rng(31)
    nodes = [(int(rng.integers(40, 536)), int(rng.integers(40, 536))) for _ in range(20)]
    _fd_check(n, 16, nodes, seed=31, pad=32)


def test_mixed_gradient_central_differences_3d():
    """3D (19-point stencil, lev-dep transfers): 40^3 cells incl. an 8-cell layer, 4
    surface sources, 20 seeded interior nodes."""
    n = (40, 40, 40)
    rng = np.random.default_rng(33)
    nodes = [tuple(int(v) for v in rng.integers(10, 31, size=3)) for _ in range(20)]
    _fd_check(n, 4, nodes, seed=33, pad=8)
