"""Blocks of right-hand sides (max_rhs > 1): the cycle and the coarsest solve run once
per block, each right-hand side keeps its own FGMRES state.  Per right-hand side the
arithmetic is that of a single solve, so results and iteration counts are identical
bit for bit; a ragged last block and right-hand sides that converge at different
iterations are covered."""
import numpy as np
import pytest

import workloads
from tests._cases import Case, rand_complex, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sources(c, count, seed):
    q = workloads.surface_sources(c.n, count, c.abc, seed=seed)
    q[-1] = rand_complex(c.grid.shape, seed)   # a smooth-free right-hand side
    q[1] = 0.0                                  # a zero right-hand side: done before the first iteration
    return q


@pytest.mark.parametrize("order,ig,prec", [("2nd", "fw", "fp64"), ("4th", "cubic", "mixed"),
                                           ("4th", "cubic", "fp64")])
def test_block_equals_single_solves(order, ig, prec):
    c = Case((64, 64), abc=6, alpha3=1.0045 if ig == "cubic" else 1.117, G_ppw=12, order=order, intergrid=ig,
             seed=2)
    q = _sources(c, 6, 4)
    qd = torch.from_numpy(q).cuda()
    sb = c.solver(max_rhs=4, precision=prec, jacobi_w=(0.89, 0.89))
    pb, stb = sb.solve(qd, tol=1e-8, maxit=300)          # blocks of 4 and 2
    s1 = c.solver(max_rhs=1, precision=prec, jacobi_w=(0.89, 0.89))
    p1, st1 = s1.solve(qd, tol=1e-8, maxit=300)
    torch.cuda.synchronize()
    assert [a["iterations"] for a in stb] == [a["iterations"] for a in st1]
    assert len({a["iterations"] for a in stb}) > 1
    assert torch.equal(pb, p1)
    sb.close()
    s1.close()


def test_block_adjoint_equals_single():
    c = Case((48, 48), abc=5, alpha3=1.117, G_ppw=12, seed=3)
    q = _sources(c, 5, 6)
    qd = torch.from_numpy(q).cuda()
    res = torch.from_numpy(rand_complex(q.shape, 7)).cuda()
    out = []
    for B in (5, 2):
        s = c.solver(max_rhs=B)
        p, _ = s.solve(qd, tol=1e-9, maxit=300)
        g = torch.zeros(c.grid.shape, dtype=torch.float64, device="cuda")
        adj = torch.empty_like(p)
        s.adjoint_grad(p, res, g, adj, tol=1e-9, maxit=300)
        torch.cuda.synchronize()
        out.append((p, g, adj))
        s.close()
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    assert torch.equal(out[0][2], out[1][2])


def test_autotune_block_picks_a_candidate_and_keeps_results():
    """The RHS-block autotuner times blocks of 1, 2, 4, ... and keeps the fastest; the
    solves that follow are those of any block size (identical per right-hand side)."""
    c = Case((64, 64), abc=6, alpha3=1.0045, G_ppw=12, order="4th", intergrid="cubic", seed=5)
    q = _sources(c, 6, 8)
    qd = torch.from_numpy(q).cuda()
    s = c.solver(max_rhs=4, precision="mixed", jacobi_w=(0.89, 0.89))
    best, costs = s.autotune_block(qd)
    assert best in (1, 2, 4) and set(costs) == {1, 2, 4}
    assert all(v > 0 for v in costs.values())
    assert costs[best] == min(costs.values())
    pb, stb = s.solve(qd, tol=1e-8, maxit=300)
    s.set_block(1)
    p1, st1 = s.solve(qd, tol=1e-8, maxit=300)
    torch.cuda.synchronize()
    assert [a["iterations"] for a in stb] == [a["iterations"] for a in st1]
    assert torch.equal(pb, p1)
    with pytest.raises(Exception):
        s.set_block(5)
    s.close()


@pytest.mark.parametrize("max_rhs,prec", [(1, "mixed"), (3, "mixed"), (1, "fp64")])
def test_graph_replay_equals_plain_launches(max_rhs, prec):
    """helm_opts.graphs: three solves in a row (plain, capture, replay) give the plain
    solve's result bit for bit; the context reports its graphs, or -1 if the capture
    was refused and it stayed on plain launches."""
    c = Case((64, 64), abc=6, alpha3=1.0045, G_ppw=12, order="4th", intergrid="cubic", seed=7)
    q = _sources(c, 3, 9) if max_rhs > 1 else workloads.point_source(c.n)
    qd = torch.from_numpy(q).cuda()
    s0 = c.solver(max_rhs=max_rhs, precision=prec, jacobi_w=(0.89, 0.89))
    p0, st0 = s0.solve(qd, tol=1e-8, maxit=300)
    torch.cuda.synchronize()
    sg = c.solver(max_rhs=max_rhs, precision=prec, jacobi_w=(0.89, 0.89), graphs=True)
    sg.timer_enable(["coarse", "arnoldi_matvec"])
    for _ in range(3):
        pg, stg = sg.solve(qd, tol=1e-8, maxit=300)
        torch.cuda.synchronize()
        assert [a["iterations"] for a in stg] == [a["iterations"] for a in st0]
        assert torch.equal(pg, p0)
    ng = sg.info()["graphs"]
    print("graphs instantiated:", ng)
    assert ng > 0
    # the launch timer sees every iteration, replayed or not: one coarsest solve per iteration
    prof = sg.timer_read()
    assert prof["coarse"][1] == 3 * max(a["iterations"] for a in st0)
    assert prof["coarse"][0] > 0
    s0.close()
    sg.close()
