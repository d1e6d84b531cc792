"""Parity of the paper's discretisation on the CUDA path: the compact 4th-order
9-point / 19-point stencils (Eqs. disc4thCompact, disc4thCompact3D) with cubic
(Eq. intergrid) or level-dependent (Eq. levdep) transfers, giving 5x5 and 7x7 (2D)
or 5x5x5 (3D) Galerkin stencils, and the real shift of Tables 1-2."""
import numpy as np
import pytest

from oracle import cycle as OC
from oracle import krylov as OK
from oracle import smoothers as OS
from tests._cases import Case, rand_complex, rel, stencil_to_dense

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONFIGS = [((32, 24), "cubic"), ((24, 40), "levdep"), ((12, 12), "cubic"), ((8, 8), "cubic"),
           ((8, 8, 12), "levdep"), ((8, 8, 8), "levdep")]
RADII = {"cubic": (2, 3), "levdep": (2, 2)}


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module")
def cases():
    out = {}
    for n, ig in CONFIGS:
        c = Case(n, abc=2, alpha2=1.01, alpha3=1.0135, seed=len(n) + n[0], order="4th", intergrid=ig)
        out[(n, ig)] = (c, c.solver())
    yield out
    for _, s in out.values():
        s.close()


@pytest.mark.parametrize("key", CONFIGS)
@pytest.mark.parametrize("level", [1, 2, 3])
def test_apply(cases, key, level):
    c, s = cases[key]
    x = rand_complex((2,) + c.hier.grids[level - 1].shape, level)
    y = _n(s.apply(level, _t(x)))
    A = c.hier.A[level - 1]
    ref = np.stack([(A @ xi.ravel()).reshape(xi.shape) for xi in x])
    assert rel(y, ref) < 1e-12
    if level < 3:
        x32 = x[0].astype(np.complex64)
        y32 = _n(s.apply(level, _t(x32)))
        assert rel(y32, (A @ x32.astype(np.complex128).ravel()).reshape(x32.shape)) < 2e-5


@pytest.mark.parametrize("key", CONFIGS)
@pytest.mark.parametrize("level", [2, 3])
def test_stencils(cases, key, level):
    c, s = cases[key]
    coef, r = s.stencil(level)
    assert r == RADII[key[1]][level - 2]
    A = stencil_to_dense(coef, r, c.hier.grids[level - 1])
    assert rel(A, c.hier.A[level - 1].toarray()) < 1e-12


@pytest.mark.parametrize("key", CONFIGS)
def test_coarse_solve_and_transfers(cases, key):
    c, s = cases[key]
    b = rand_complex(c.hier.grids[2].shape, 5)
    e = _n(s.coarse_solve(_t(b)))
    assert rel(e.ravel(), c.hier.coarse_solve(b.ravel())) < 1e-10
    for level in (1, 2):
        gf, gc = c.hier.grids[level - 1], c.hier.grids[level]
        rf = rand_complex(gf.shape, 6)
        assert rel(_n(s.restrict(level, _t(rf))).ravel(), c.hier.R[level - 1] @ rf.ravel()) < 1e-13
        ec, xf = rand_complex(gc.shape, 7), rand_complex(gf.shape, 8)
        out = _n(s.prolong_add(level, _t(ec), _t(xf))).ravel()
        assert rel(out, xf.ravel() + c.hier.P[level - 1] @ ec.ravel()) < 1e-13


@pytest.mark.parametrize("key", CONFIGS)
@pytest.mark.parametrize("smoother", ["jacobi", "rb"])
def test_smoother(key, smoother):
    n, ig = key
    c = Case(n, abc=2, alpha3=1.0135, seed=3, order="4th", intergrid=ig)
    s = c.solver(smoother=smoother, jacobi_w=(0.89, 0.89), rb_w=0.9)
    for level in (1, 2):
        g = c.hier.grids[level - 1]
        b, x = rand_complex(g.shape, 9), rand_complex(g.shape, 10)
        got = _n(s.smooth(level, _t(b), _t(x))).ravel()
        A, d = c.hier.A[level - 1], c.hier.diag[level - 1]
        ref = (OS.jacobi(A, d, x.ravel(), b.ravel(), 0.89) if smoother == "jacobi"
               else OS.red_black(A, d, x.ravel(), b.ravel(), OS.colours(g), 0.9))
        assert rel(got, ref) < 1e-12
    s.close()


@pytest.mark.parametrize("key", CONFIGS)
@pytest.mark.parametrize("cyc", ["V", "W"])
def test_cycle(key, cyc):
    n, ig = key
    c = Case(n, abc=2, alpha3=1.0135, seed=4, order="4th", intergrid=ig)
    s = c.solver(cycle=cyc, jacobi_w=(0.89, 0.89))
    v = rand_complex(c.grid.shape, 11)
    z = _n(s.cycle(_t(v)))
    ref = OC.Cycle(c.hier, cycle=cyc, weights=(0.89, 0.89))(v.ravel())
    assert rel(z.ravel(), ref) < 1e-10
    s.close()
    sm = c.solver(cycle=cyc, jacobi_w=(0.89, 0.89), precision="mixed")
    assert rel(_n(sm.cycle(_t(v))).ravel(), ref) < 1e-5
    sm.close()


@pytest.mark.parametrize("n,ig,alpha,cyc", [((128, 128), "cubic", 1.0045, "W"), ((96, 64), "levdep", 1.0135, "V"),
                                            ((16, 16, 16), "levdep", 1.0120, "V")])
def test_solve_matches_oracle(n, ig, alpha, cyc):
    """The paper's 2D set-up (W(1,1), Jacobi 0.89, Table 1 shift) at 12 ppw."""
    import workloads

    c = Case(n, abc=16 if n[0] == 128 else 4, alpha3=alpha, G_ppw=12, seed=5, order="4th", intergrid=ig,
             kappa2=workloads.constant_medium(n) if n[0] == 128 else None)
    w = (0.89, 0.89) if len(n) == 2 else (0.6, 0.4)
    s = c.solver(cycle=cyc, jacobi_w=w)
    q = workloads.point_source(n)
    p, st = s.solve(_t(q), tol=1e-6, maxit=300)
    cy = OC.Cycle(c.hier, cycle=cyc, weights=w)
    xo, info = OK.fgmres(lambda v: c.hier.A[0] @ v, q.ravel(), cy, tol=1e-6, maxit=300, restart=10)
    assert st[0]["converged"] and info["converged"]
    assert st[0]["iterations"] == info["iterations"]
    assert rel(_n(p).ravel(), xo) < 1e-10
    s.close()
    sm = c.solver(cycle=cyc, jacobi_w=w, precision="mixed")
    pm, stm = sm.solve(_t(q), tol=1e-6, maxit=300)
    assert stm[0]["converged"] and abs(stm[0]["iterations"] - info["iterations"]) <= 1
    assert rel(_n(pm).ravel(), xo) < 1e-5
    sm.close()
