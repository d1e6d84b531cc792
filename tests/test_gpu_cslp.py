"""RS-CGC + CSLP (Sec. 5, second experiment: RS-CGC combined with a complex shift of
0.03 k^2 for 10 points per wavelength): the cycle's operators carry the shift, the outer
FGMRES operator does not.  Parity with the oracle: operators 1e-12, FP64 solves with
equal iteration counts and 1e-10 solutions, mixed solves +-1 iteration and 1e-5."""
import numpy as np
import pytest

from oracle import cycle as OC
from oracle import krylov as OK
from tests._cases import Case, rand_complex, rel, stencil_to_dense

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("n,order,ig", [((32, 24), "2nd", "fw"), ((48, 40), "4th", "cubic"), ((8, 12, 16), "2nd", "fw")])
def test_shifted_cycle_operators(n, order, ig):
    c = Case(n, order=order, intergrid=ig, alpha3=1.05, beta=0.03, seed=11)
    s = c.solver()
    x = rand_complex(c.grid.shape, 3)
    assert rel(_n(s.apply(1, _t(x))), (c.hier.A[0] @ x.ravel()).reshape(x.shape)) < 1e-12
    for level in (2, 3):
        coef, r = s.stencil(level)
        A = stencil_to_dense(coef, r, c.hier.grids[level - 1])
        assert rel(A, c.hier.A[level - 1].toarray()) < 1e-12
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rs_cgc_cslp_solve_matches_oracle(prec):
    import workloads

    n = (96, 96)
    c = Case(n, abc=12, order="4th", intergrid="cubic", alpha3=1.0045, beta=0.03,
             kappa2=workloads.constant_medium(n), G_ppw=10)
    q = workloads.point_source(n)
    s = c.solver(precision=prec, jacobi_w=(0.89, 0.89))
    p, st = s.solve(_t(q), tol=1e-6, maxit=300)
    s.close()
    cy = OC.Cycle(c.hier, weights=(0.89, 0.89))
    xo, info = OK.fgmres(lambda v: c.hier.A_outer @ v, q.ravel(), cy, tol=1e-6, maxit=300, restart=10)
    assert st[0]["converged"] and info["converged"]
    if prec == "fp64":
        assert st[0]["iterations"] == info["iterations"]
        assert rel(_n(p).ravel(), xo) < 1e-10
    else:
        assert abs(st[0]["iterations"] - info["iterations"]) <= 1
        assert rel(_n(p).ravel(), xo) < 1e-5
    # the outer operator is unshifted: the solution satisfies H p = q, not the shifted system
    r = q.ravel() - c.hier.A_outer @ _n(p).ravel()
    assert np.linalg.norm(r) / np.linalg.norm(q) < 1e-6
