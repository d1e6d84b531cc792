"""Contexts solving at the same time on their own streams (the uneven-grid batch): every
result equals the same context's solve run alone, bit for bit, whatever share of the
device its coarsest solve runs on (helm_opts.coarse_blocks)."""
import pytest

import workloads
from tests._cases import Case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_concurrent_solves_equal_separate_solves():
    from paper_2604_19501_gb300 import solve_concurrent

    cases = [Case((64, 64), abc=6, alpha3=1.0045, G_ppw=12, order="4th", intergrid="cubic", seed=1),
             Case((96, 80), abc=8, alpha3=1.0045, G_ppw=12, order="4th", intergrid="cubic", seed=2),
             Case((48, 112), abc=6, alpha3=1.0045, G_ppw=12, order="4th", intergrid="cubic", seed=3)]
    qs = [torch.from_numpy(workloads.point_source(c.n)).cuda() for c in cases]
    streams = [torch.cuda.Stream() for _ in cases]
    shared = [c.solver(precision="mixed", jacobi_w=(0.89, 0.89), stream=st.cuda_stream, coarse_blocks=152)
              for c, st in zip(cases, streams)]
    alone = [c.solver(precision="mixed", jacobi_w=(0.89, 0.89)) for c in cases]
    ref = [s.solve(q, tol=1e-8, maxit=300) for s, q in zip(alone, qs)]
    torch.cuda.synchronize()
    for _ in range(2):
        out = solve_concurrent(shared, qs, tol=1e-8, maxit=300)
        torch.cuda.synchronize()
        for (p, st), (p0, st0) in zip(out, ref):
            assert [x["iterations"] for x in st] == [x["iterations"] for x in st0]
            assert st[0]["converged"]
            assert torch.equal(p, p0)
    for s in shared + alone:
        s.close()


def test_coarse_blocks_is_validated():
    from paper_2604_19501_gb300 import HelmError

    with pytest.raises(HelmError):
        Case((16, 16)).solver(coarse_blocks=-1)
