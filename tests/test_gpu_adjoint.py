"""Adjoint gradient on the CUDA path (helm_adjoint_grad, the torch.autograd backward)
against the oracle's adjoint gradient and against central finite differences of the
misfit (step 1e-4 relative, solves at tol 1e-11)."""
import numpy as np
import pytest

import workloads
from oracle import adjoint as OA
from oracle import grid as OG
from oracle import operators as OO
from tests._cases import Case, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(n, order, ig, nsrc, seed):
    pad = 6
    rng = np.random.default_rng(seed)
    kappa2 = workloads.layered_faulted_2d(n[0] - 2 * pad, pad, seed=seed, sigma=2.0) if len(n) == 2 \
        else workloads.layered_3d([v - 2 * pad for v in n], pad, seed=seed, sigma=2.0)
    c = Case(n, abc=pad, alpha3=1.0045 if ig == "cubic" else 1.117, kappa2=kappa2, G_ppw=12, order=order,
             intergrid=ig)
    q = workloads.surface_sources(n, nsrc, pad, seed=seed)
    mask = np.zeros(c.grid.shape, dtype=bool)
    if len(n) == 2:
        mask[pad, :] = True
    else:
        mask[pad, :, :] = True
    d = (rng.standard_normal(q.shape) + 1j * rng.standard_normal(q.shape)) * 0.01 * mask
    return c, q, mask, d


def _oracle_solve(c, rhs):
    import scipy.sparse.linalg as spla

    lu = spla.splu(c.hier.A[0].tocsc())
    return np.stack([lu.solve(r.ravel()).reshape(r.shape) for r in rhs])


@pytest.mark.parametrize("n,order,ig", [((64, 64), "2nd", "fw"), ((64, 64), "4th", "cubic"),
                                        ((24, 24, 16), "4th", "levdep")])
def test_adjoint_gradient_matches_oracle(n, order, ig):
    c, q, mask, d = _problem(n, order, ig, 3, seed=5)
    s = c.solver(cycle="V", jacobi_w=(0.89, 0.89) if len(n) == 2 else (0.6, 0.4))
    qd = torch.from_numpy(q).cuda()
    p, st = s.solve(qd, tol=1e-11, maxit=500)
    pn = p.cpu().numpy()
    resid = np.where(mask, pn - d, 0.0)
    grad = torch.zeros(c.grid.shape, dtype=torch.float64, device="cuda")
    adj = torch.empty_like(p)
    ast = s.adjoint_grad(p, torch.from_numpy(resid).cuda(), grad, adj, tol=1e-11, maxit=500)
    assert all(a["converged"] for a in ast)
    po = _oracle_solve(c, q)
    mu = _oracle_solve(c, OA.adjoint_rhs(po, d, mask))
    go = OA.gradient(c.grid, c.omega, c.gamma, po, mu, order)
    assert rel(grad.cpu().numpy(), go) < 1e-8
    assert rel(adj.cpu().numpy(), mu) < 1e-8
    s.close()


def test_autograd_gradient_matches_central_differences():
    """The differentiation workload at reduced size: 2D layered medium, 4 surface sources,
    receivers on the top interior row; dL/dkappa2 at 10 seeded interior nodes."""
    from paper_2604_19501_gb300 import helmholtz_solve

    n = (96, 96)
    c, q, mask, d = _problem(n, "4th", "cubic", 4, seed=9)
    opts = dict(abc_width=c.abc, alpha3=c.alpha3, stencil="4th", intergrid="cubic", jacobi_w=(0.89, 0.89))
    qd = torch.from_numpy(q).cuda()
    dd = torch.from_numpy(d).cuda()
    mk = torch.from_numpy(mask).cuda()

    def loss(k2):
        p = helmholtz_solve(k2, qd, n, c.omega, tol=1e-11, maxit=800, **opts)
        r = torch.where(mk, p - dd, torch.zeros_like(p))
        return 0.5 * (r.abs() ** 2).sum()

    k2 = torch.from_numpy(c.kappa2.copy()).cuda().requires_grad_(True)
    L = loss(k2)
    L.backward()
    g = k2.grad.cpu().numpy()
    rng = np.random.default_rng(3)
    nodes = [(int(rng.integers(8, 88)), int(rng.integers(8, 88))) for _ in range(10)]
    for j in nodes:
        h = 1e-4 * c.kappa2[j]
        kp = c.kappa2.copy()
        km = c.kappa2.copy()
        kp[j] += h
        km[j] -= h
        with torch.no_grad():
            fd = (loss(torch.from_numpy(kp).cuda()).item() - loss(torch.from_numpy(km).cuda()).item()) / (2 * h)
        assert g[j] == pytest.approx(fd, rel=1e-4, abs=1e-6 * np.max(np.abs(g)))


def test_recompute_and_source_gradient():
    from paper_2604_19501_gb300 import helmholtz_solve

    n = (48, 48)
    c, q, mask, d = _problem(n, "2nd", "fw", 2, seed=11)
    opts = dict(abc_width=c.abc, alpha3=c.alpha3)
    qd = torch.from_numpy(q).cuda().requires_grad_(True)
    k2 = torch.from_numpy(c.kappa2).cuda().requires_grad_(True)
    grads = []
    for recompute in (False, True):
        p = helmholtz_solve(k2, qd, n, c.omega, tol=1e-11, maxit=500, recompute=recompute, **opts)
        L = 0.5 * (p.abs() ** 2 * torch.from_numpy(mask).cuda()).sum()
        gk, gq = torch.autograd.grad(L, (k2, qd))
        grads.append((gk.cpu().numpy(), gq.cpu().numpy()))
    assert rel(grads[0][0], grads[1][0]) < 1e-9
    # dL/dq = lambda = A^-H (mask p): check with the oracle's direct solves
    po = _oracle_solve(c, q)
    lam = np.conj(_oracle_solve(c, np.conj(mask * po)))
    assert rel(grads[0][1], lam) < 1e-8


def test_reused_context_gives_the_same_gradients():
    """helmholtz_solve(..., reuse_context=True): the second call with the same unmodified
    kappa2 tensor uses the kept context (no new set-up) and gives the same field and
    gradient bit for bit; an in-place change of kappa2 (version counter) or other options
    make a new context, whose gradient matches a context of its own."""
    import paper_2604_19501_gb300 as P
    from paper_2604_19501_gb300 import helmholtz_solve

    n = (48, 48)
    c, q, mask, d = _problem(n, "4th", "cubic", 2, seed=13)
    opts = dict(abc_width=c.abc, alpha3=c.alpha3, stencil="4th", intergrid="cubic", precision="mixed", max_rhs=2)
    qd = torch.from_numpy(q).cuda()
    mk = torch.from_numpy(mask).cuda()
    k2 = torch.from_numpy(c.kappa2.copy()).cuda().requires_grad_(True)

    def grad(reuse, k):
        p = helmholtz_solve(k, qd, n, c.omega, tol=1e-10, maxit=400, reuse_context=reuse, **opts)
        L = 0.5 * ((p.abs() ** 2) * mk).sum()
        (g,) = torch.autograd.grad(L, (k,))
        return p.detach().cpu().numpy(), g.cpu().numpy()

    P.release_reused_context()
    p1, g1 = grad(True, k2)
    kept = P._REUSE["solver"]
    p2, g2 = grad(True, k2)
    assert P._REUSE["solver"] is kept
    assert np.array_equal(p1, p2) and np.array_equal(g1, g2)
    p0, g0 = grad(False, k2)          # a context of its own
    assert rel(g1, g0) < 1e-8 and rel(p1, p0) < 1e-9
    with torch.no_grad():
        k2 *= 1.001                   # bumps the version counter
    p3, g3 = grad(True, k2)
    assert P._REUSE["solver"] is not kept
    p4, g4 = grad(False, k2)
    assert rel(g3, g4) < 1e-8 and rel(p3, p4) < 1e-9
    assert rel(g3, g1) > 1e-6         # a different medium
    P.release_reused_context()
