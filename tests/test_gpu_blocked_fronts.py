"""Coarsest-level fronts with at least 128 eliminated nodes (helm_opts.coarse_block_min = 128;
the library's default threshold is 512) are eliminated by blocked Gauss-Jordan steps
(panels of 64 columns, pivot rows by partial pivoting, the rest of the front updated by
complex FP64 matrix products).  These cases put such fronts at the top of the nested-dissection
tree and compare the direct solve with SuperLU on the oracle's level-3
operator (Eq. CoarseRealShifted) and whole solves with the oracle's FGMRES.

Tolerances: on the 3D grid (lev-dep transfers, 19-point stencil, 17^3 coarsest nodes) the
direct solve agrees with SuperLU to 1e-10.  On the 2D grid (181^2 coarsest nodes, a
543-node root separator) the undamped interior makes some separator blocks nearly
singular, and the front-local pivoting amplifies rounding (as the unblocked elimination
does at this depth: residuals of a few 1e-11 with FP64 factors, 1e-9 with double-float
ones), so the unrefined bound there is 1e-9 / 1e-8.  With one refinement step
(helm_opts.coarse_refine) every case must reach 1e-12: a factorisation with an error well
above rounding could not."""
import numpy as np
import pytest

import workloads
from oracle import cycle as OC
from oracle import krylov as OK
from tests._cases import Case, rand_complex, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("n,ig,bound", [((720, 720), "cubic", {"fp64": 1e-9, "mixed": 1e-8}),
                                        ((64, 64, 64), "levdep", {"fp64": 1e-10, "mixed": 1e-10})])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_blocked_coarse_solve_matches_superlu(n, ig, bound, prec):
    c = Case(n, abc=8 if len(n) == 2 else 6, alpha3=1.0045 if ig == "cubic" else 1.012, G_ppw=12, seed=17,
             order="4th", intergrid=ig)
    b = rand_complex((2,) + c.hier.grids[2].shape, 18)
    ref = np.stack([c.hier.coarse_solve(bi.ravel()).reshape(bi.shape) for bi in b])
    for refine in (0, 1):
        s = c.solver(precision=prec, coarse_refine=refine, coarse_block_min=128)
        info = s.info()
        e = _n(s.coarse_solve(torch.from_numpy(b).cuda()))
        s.close()
        res = max(np.linalg.norm(c.hier.A[2] @ e[k].ravel() - b[k].ravel()) / np.linalg.norm(b[k]) for k in range(2))
        print(n, prec, "refine", refine, info["coarse_levels"], "levels;", "rel", rel(e, ref), "res", res)
        lim = bound[prec] if refine == 0 else 1e-12
        assert rel(e, ref) < max(lim, 1e-12) * (10 if refine == 0 and len(n) == 2 else 1)
        assert res < lim


def test_blocked_fronts_solve_3d_matches_oracle():
    """A whole FP64 solve on the 3D grid whose coarsest root front is blocked: iteration
    count equal to the oracle's, solution within 1e-10."""
    n = (64, 64, 64)
    c = Case(n, abc=6, alpha3=1.012, G_ppw=12, seed=19, order="4th", intergrid="levdep")
    w = (0.6, 0.4)
    s = c.solver(cycle="W", jacobi_w=w, coarse_block_min=128)
    q = workloads.point_source(n)
    p, st = s.solve(torch.from_numpy(q).cuda(), tol=1e-6, maxit=200)
    s.close()
    cy = OC.Cycle(c.hier, cycle="W", weights=w)
    xo, info = OK.fgmres(lambda v: c.hier.A[0] @ v, q.ravel(), cy, tol=1e-6, maxit=200, restart=10)
    print("gpu", st[0], "oracle", info["iterations"])
    assert st[0]["converged"] and info["converged"]
    assert st[0]["iterations"] == info["iterations"]
    assert rel(_n(p).ravel(), xo) < 1e-10
