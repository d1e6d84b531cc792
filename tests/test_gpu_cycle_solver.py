"""RS-CGC as a solver (Sec. 5, the parenthesised iteration counts of Table 3): the
stationary iteration p <- p + M^-1 (q - H p) with one cycle as M^-1 (helm_opts.solver =
HELM_SOLVER_CYCLE), against the oracle's stationary iteration with the oracle cycle.

Tolerances: FP64 runs the oracle's arithmetic up to rounding order, so iteration counts
are equal and iterates agree to 1e-10.  Mixed precision computes levels 1-2 of each
cycle in FP32 (unit roundoff 6e-8); after three cycles the iterate agrees to 1e-5, and a
converged solve takes the oracle's count +-1 with a true residual below tol."""
import numpy as np
import pytest

import workloads
from oracle import cycle as OC
from oracle import krylov as OK
from tests._cases import Case, rand_complex, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = (0.89, 0.89)


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _case(n=(96, 96)):
    return Case(n, abc=12, order="4th", intergrid="cubic", alpha3=1.0045,
                kappa2=workloads.constant_medium(n), G_ppw=10)


# (V, mixed) takes the fused tile passes of the cycle, the others one kernel per step
@pytest.mark.parametrize("cyc,prec", [("W", "fp64"), ("W", "mixed"), ("V", "fp64"), ("V", "mixed")])
def test_cycle_solver_matches_oracle(cyc, prec):
    c = _case()
    q = workloads.point_source(c.n)
    qd = torch.from_numpy(q).cuda()
    s = c.solver(precision=prec, cycle=cyc, jacobi_w=W, solver="cycle")
    cy = OC.Cycle(c.hier, cycle=cyc, weights=W)
    A = lambda v: c.hier.A_outer @ v
    # three iterations, not converged: the iterates themselves
    p3, st3 = s.solve(qd, tol=1e-14, maxit=3)
    x3, info3 = OK.stationary(A, q.ravel(), cy, tol=1e-14, maxit=3)
    assert st3[0]["iterations"] == info3["iterations"] == 3 and not st3[0]["converged"]
    assert rel(_n(p3).ravel(), x3) < (1e-10 if prec == "fp64" else 1e-5)
    assert st3[0]["relres"] == pytest.approx(info3["relres"], rel=1e-8 if prec == "fp64" else 1e-4)
    # to convergence
    p, st = s.solve(qd, tol=1e-6, maxit=80)
    x, info = OK.stationary(A, q.ravel(), cy, tol=1e-6, maxit=80)
    s.close()
    assert st[0]["converged"] and info["converged"]
    assert st[0]["est_relres"] == st[0]["relres"]
    r = q.ravel() - c.hier.A_outer @ _n(p).ravel()
    assert np.linalg.norm(r) / np.linalg.norm(q) < 1e-6
    assert np.linalg.norm(r) / np.linalg.norm(q) == pytest.approx(st[0]["relres"], rel=1e-6)
    if prec == "fp64":
        assert st[0]["iterations"] == info["iterations"]
        assert rel(_n(p).ravel(), x) < 1e-10
    else:
        assert abs(st[0]["iterations"] - info["iterations"]) <= 1


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cycle_solver_block_equals_single(prec):
    """A block of right-hand sides (one cycle for the block per iteration) gives each
    right-hand side its single-solve iterate bit for bit, including a zero right-hand
    side (no iteration) and right-hand sides that stop at different iterations."""
    c = Case((64, 64), abc=6, alpha3=1.0045, G_ppw=12, order="4th", intergrid="cubic", seed=2)
    q = workloads.surface_sources(c.n, 5, c.abc, seed=4)
    q[-1] = rand_complex(c.grid.shape, 4)
    q[1] = 0.0
    qd = torch.from_numpy(q).cuda()
    sb = c.solver(max_rhs=3, precision=prec, cycle="W", jacobi_w=W, solver="cycle")
    pb, stb = sb.solve(qd, tol=1e-8, maxit=100)          # blocks of 3 and 2
    s1 = c.solver(max_rhs=1, precision=prec, cycle="W", jacobi_w=W, solver="cycle")
    p1, st1 = s1.solve(qd, tol=1e-8, maxit=100)
    torch.cuda.synchronize()
    assert [a["iterations"] for a in stb] == [a["iterations"] for a in st1]
    assert stb[1]["iterations"] == 0 and stb[1]["converged"]
    assert len({a["iterations"] for a in stb}) > 1
    assert all(a["converged"] for a in stb)
    assert torch.equal(pb, p1)
    assert not torch.any(pb[1])
    sb.close()
    s1.close()


def test_cycle_solver_graph_replay_equals_plain_launches():
    """helm_opts.graphs with the cycle solver: the captured iteration reads and writes
    only context buffers, so replays serve other right-hand sides and output tensors."""
    c = Case((64, 64), abc=6, alpha3=1.0045, G_ppw=12, order="4th", intergrid="cubic", seed=7)
    qs = [torch.from_numpy(workloads.point_source(c.n)).cuda(),
          torch.from_numpy(workloads.surface_sources(c.n, 1, c.abc, seed=3)[0]).cuda()]
    s0 = c.solver(precision="mixed", jacobi_w=W, cycle="W", solver="cycle")
    ref = [s0.solve(q, tol=1e-8, maxit=100) for q in qs]
    torch.cuda.synchronize()
    sg = c.solver(precision="mixed", jacobi_w=W, cycle="W", solver="cycle", graphs=True)
    for q, (p0, st0) in zip(qs + qs, ref + ref):
        pg, stg = sg.solve(q, tol=1e-8, maxit=100)
        torch.cuda.synchronize()
        assert stg[0]["iterations"] == st0[0]["iterations"]
        assert torch.equal(pg, p0)
    assert sg.info()["graphs"] > 0
    s0.close()
    sg.close()


def test_cycle_solver_adjoint_gradient_agrees_with_fgmres():
    """helm_adjoint_grad with the cycle solver: the same gradient as with FGMRES, to the
    accuracy both solves reach (tol 1e-11)."""
    c = Case((64, 64), abc=6, alpha3=1.0045, G_ppw=12, order="4th", intergrid="cubic", seed=5)
    q = torch.from_numpy(workloads.point_source(c.n)).cuda()
    grads = []
    for solver in ("fgmres", "cycle"):
        s = c.solver(cycle="W", jacobi_w=W, solver=solver)
        p, st = s.solve(q, tol=1e-11, maxit=300)
        assert st[0]["converged"]
        resid = torch.from_numpy(rand_complex(c.grid.shape, 8)).cuda()
        g = torch.zeros(c.grid.shape, dtype=torch.float64, device="cuda")
        sta = s.adjoint_grad(p, resid, g, tol=1e-11, maxit=300)
        assert sta[0]["converged"]
        grads.append(_n(g))
        s.close()
    assert rel(grads[1], grads[0]) < 1e-7


def test_bad_solver_is_rejected():
    from paper_2604_19501_gb300 import HelmError, _ffi

    _ffi.SOLVER["bogus"] = 7
    try:
        with pytest.raises(HelmError):
            _case((16, 16)).solver(solver="bogus")
    finally:
        del _ffi.SOLVER["bogus"]


@pytest.mark.parametrize("model,kmin,prec", [("linear", 0.1, "fp64"), ("wedge", 0.5, "mixed")])
def test_table3_models_match_oracle(model, kmin, prec):
    """The 2D heterogeneous models of Sec. 5.1 (Table 3) at 128^2 cells + 20-cell layer,
    W(1,1): FGMRES and the cycle solver take the oracle's iteration counts (mixed: +-1)."""
    from oracle import grid as OG
    from oracle import hierarchy as OH

    cells, pad = 128, 20
    f = {"linear": workloads.linear_2d, "wedge": workloads.wedge_2d}[model]
    kappa2 = f(cells, pad, kmin)
    N = cells + 2 * pad
    c = Case((N, N), abc=pad, alpha3=1.0045, order="4th", intergrid="cubic", kappa2=kappa2, G_ppw=12)
    q = workloads.point_source(c.n, node=(N // 2, pad))
    qd = torch.from_numpy(q).cuda()
    cy = OC.Cycle(c.hier, cycle="W", weights=W)
    A = lambda v: c.hier.A_outer @ v
    for solver in ("fgmres", "cycle"):
        s = c.solver(precision=prec, cycle="W", jacobi_w=W, solver=solver, restart=40)
        p, st = s.solve(qd, tol=1e-6, maxit=60)
        s.close()
        if solver == "fgmres":
            x, info = OK.fgmres(A, q.ravel(), cy, tol=1e-6, maxit=60, restart=60)
        else:
            x, info = OK.stationary(A, q.ravel(), cy, tol=1e-6, maxit=60)
        assert st[0]["converged"] and info["converged"]
        if prec == "fp64":
            assert st[0]["iterations"] == info["iterations"]
            assert rel(_n(p).ravel(), x) < 1e-9
        else:
            assert abs(st[0]["iterations"] - info["iterations"]) <= 1
