"""The fused 2D mixed-precision cycle (tile passes of Sec. 2's V(1,1) Jacobi cycle) against
the oracle cycle and against the per-step kernels: every discretisation / transfer pair,
ragged grids whose tiles are partly outside, batches, and full FGMRES solves.

Tolerance: 1e-5 relative (FP32 arithmetic of the cycle, as for the per-step c64 path)."""
import numpy as np
import pytest

from oracle import cycle as OC
from oracle import krylov as OK
from tests._cases import Case, rand_complex, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONFIGS = [((32, 24), "2nd", "fw"), ((48, 40), "4th", "cubic"), ((64, 52), "4th", "levdep"),
           ((100, 76), "4th", "cubic"), ((36, 100), "2nd", "cubic"), ((8, 4), "4th", "fw")]


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _n(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("n,order,ig", CONFIGS)
def test_fused_cycle_matches_oracle_and_unfused(n, order, ig):
    c = Case(n, order=order, intergrid=ig, alpha3=1.05, seed=4, abc=2 if min(n) <= 8 else 4)
    v = rand_complex(c.grid.shape, 5)
    ref = OC.Cycle(c.hier)(v.ravel()).reshape(v.shape)
    s = c.solver(precision="mixed")
    z = _n(s.cycle(_t(v)))
    s.close()
    u = c.solver(precision="mixed", fuse_cycle=False)
    zu = _n(u.cycle(_t(v)))
    u.close()
    assert rel(z, ref) < 1e-5
    assert rel(z, zu) < 1e-5


@pytest.mark.parametrize("n,order,ig", CONFIGS)
def test_fine_pass_kernels_agree(n, order, ig):
    """Every kernel kind of the fine passes (shared-memory tiles; one warp per strip with
    segments of 8, 16 and 32 coarse rows) against the oracle cycle and against each other
    (the same operators and sums in the same order: FP32 rounding only), and the autotuner
    picks one of them."""
    from paper_2604_19501_gb300 import _ffi

    c = Case(n, order=order, intergrid=ig, alpha3=1.05, seed=14, abc=2 if min(n) <= 8 else 4)
    v = np.stack([rand_complex(c.grid.shape, 15 + k) for k in range(2)])
    ref = np.stack([OC.Cycle(c.hier)(vk.ravel()).reshape(vk.shape) for vk in v])
    s = c.solver(precision="mixed")
    out = {}
    for kind in _ffi.CYCLE_KERNELS:
        s.set_cycle_kernels(kind)
        out[kind] = _n(s.cycle(_t(v)))
        assert rel(out[kind], ref) < 1e-5, kind
        assert rel(out[kind], out["tiles"]) < 1e-6, kind
    best, ms = s.autotune_cycle(2)
    assert best in _ffi.CYCLE_KERNELS and set(ms) == set(_ffi.CYCLE_KERNELS) and all(t > 0 for t in ms.values())
    assert s.info()["cycle_kernels"] == _ffi.CYCLE_KERNELS.index(best)
    assert rel(_n(s.cycle(_t(v))), ref) < 1e-5
    s.close()


def test_fused_cycle_batch_is_per_rhs():
    c = Case((48, 40), order="4th", intergrid="cubic", alpha3=1.05, seed=6)
    s = c.solver(precision="mixed")
    vs = np.stack([rand_complex(c.grid.shape, 10 + k) for k in range(3)])
    zb = _n(s.cycle(_t(vs)))
    for k in range(3):
        zk = _n(s.cycle(_t(vs[k])))
        assert np.array_equal(zb[k], zk)
    s.close()


@pytest.mark.parametrize("order,ig,alpha3", [("4th", "cubic", 1.0045), ("2nd", "fw", 1.117)])
def test_fused_solve_matches_unfused_and_oracle(order, ig, alpha3):
    import workloads

    n = (128, 128)
    c = Case(n, abc=16, order=order, intergrid=ig, alpha3=alpha3, kappa2=workloads.constant_medium(n), G_ppw=12)
    q = workloads.point_source(n)
    s = c.solver(precision="mixed", jacobi_w=(0.89, 0.89) if order == "4th" else (0.8, 0.8))
    p, st = s.solve(_t(q), tol=1e-6, maxit=400)
    p = _n(p)
    s.close()
    u = c.solver(precision="mixed", fuse_cycle=False, jacobi_w=(0.89, 0.89) if order == "4th" else (0.8, 0.8))
    pu, stu = u.solve(_t(q), tol=1e-6, maxit=400)
    pu = _n(pu)
    u.close()
    cy = OC.Cycle(c.hier, weights=(0.89, 0.89) if order == "4th" else (0.8, 0.8))
    xo, info = OK.fgmres(lambda x: c.hier.A[0] @ x, q.ravel(), cy, tol=1e-6, maxit=400, restart=10)
    assert st[0]["converged"] and stu[0]["converged"] and info["converged"]
    assert abs(st[0]["iterations"] - info["iterations"]) <= 1
    assert abs(st[0]["iterations"] - stu[0]["iterations"]) <= 1
    assert rel(p.ravel(), xo) < 1e-5
    assert rel(p, pu) < 1e-5


@pytest.mark.parametrize("passes", [1, 2])
def test_arnoldi_passes_match_oracle(passes):
    """The mixed-precision Arnoldi step with one double-float Gram-Schmidt pass (norm from
    ||w||^2 - ||h||^2) and with CGS2, on the layered medium with restarts (FGMRES(5)):
    iteration count within one of the oracle's FGMRES, solution within 1e-5."""
    import workloads

    n = (160, 160)
    k2 = workloads.layered_faulted_2d(128, 16, seed=21)
    c = Case(n, abc=16, order="4th", intergrid="cubic", alpha3=1.0045, G_ppw=12, kappa2=k2)
    q = workloads.point_source(n)
    s = c.solver(precision="mixed", jacobi_w=(0.89, 0.89), restart=5, arnoldi_passes=passes)
    p, st = s.solve(_t(q), tol=1e-6, maxit=400)
    p = _n(p)
    s.close()
    cy = OC.Cycle(c.hier, weights=(0.89, 0.89))
    xo, info = OK.fgmres(lambda x: c.hier.A[0] @ x, q.ravel(), cy, tol=1e-6, maxit=400, restart=5)
    assert st[0]["converged"] and info["converged"]
    assert abs(st[0]["iterations"] - info["iterations"]) <= 1, (st[0]["iterations"], info["iterations"])
    assert rel(p.ravel(), xo) < 1e-5
