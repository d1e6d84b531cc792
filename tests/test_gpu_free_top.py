"""Absorbing layers of different width per face (helm_opts.abc_width per face), as in the
paper's 3D set-up (Sec. 5.2): no layer on the top face (the low end of the depth axis),
the source at the centre of that face.  2D and 3D, lev-dep and cubic transfers, W and V
cycles, against the oracle built with the same per-face profile.  FP64: equal iteration
counts and 1e-10; mixed: +-1 iteration and 1e-5."""
import numpy as np
import pytest

import workloads
from oracle import cycle as OC
from oracle import grid as OG
from oracle import hierarchy as OH
from oracle import krylov as OK
from tests._cases import medium, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (cells, per-face widths x-lo x-hi y-lo y-hi [z-lo z-hi], transfers, alpha3, Jacobi, cycle)
CASES = [
    ((48, 40), (4, 4, 0, 4), "cubic", 1.0045, (0.89, 0.89), "W"),
    ((20, 20, 16), (4, 4, 4, 4, 0, 4), "levdep", 1.012, (0.6, 0.4), "W"),
    ((16, 24, 12), (3, 3, 2, 4, 0, 3), "levdep", 1.012, (0.6, 0.4), "V"),
]


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[0])) + "-" + c[2] + "-" + c[5])
def test_free_top_solve_matches_oracle(case, prec):
    from paper_2604_19501_gb300 import Solver

    n, w, ig, alpha3, jw, cyc = case
    dim = len(n)
    kappa2 = medium(n, seed=5)
    omega = workloads.omega_for_ppw(12, 1.0 / np.sqrt(kappa2.max()))
    grid = OG.Grid(n)
    widths = [(w[2 * a], w[2 * a + 1]) for a in range(dim)]
    gamma = OG.abc_profile(grid, widths, 1.0)
    h = OH.Hierarchy(grid, kappa2, omega, gamma, "4th", ig, alpha3=alpha3)
    node = tuple(v // 2 for v in n[:-1]) + (0,)
    q = workloads.point_source(n, node=node)
    x, info = OK.fgmres(lambda v: h.A_outer @ v, q.ravel(), OC.Cycle(h, cycle=cyc, weights=jw),
                        tol=1e-6, maxit=200, restart=10)
    assert info["converged"]
    s = Solver(torch.from_numpy(kappa2).cuda(), n, omega, abc_width=list(w) + [0] * (6 - len(w)), alpha3=alpha3,
               stencil="4th", intergrid=ig, cycle=cyc, jacobi_w=jw, precision=prec)
    p, st = s.solve(torch.from_numpy(q).cuda(), tol=1e-6, maxit=200)
    s.close()
    assert st[0]["converged"]
    if prec == "fp64":
        assert st[0]["iterations"] == info["iterations"]
        assert rel(_n(p).ravel(), x) < 1e-10
    else:
        assert abs(st[0]["iterations"] - info["iterations"]) <= 1
        assert rel(_n(p).ravel(), x) < 1e-5
