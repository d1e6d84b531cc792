"""Failure detection on the GPU without a fault: the coarsest-solve kernel's dependency
waits are bounded.  helm_coarse_wait_check gives one job of the solve's job list a
completion count that nothing reaches and a short limit (1e6 SM cycles, about half a
millisecond); the next solve must come back with HELM_ECUDA and the wait message, the
error must stay recorded for that context, and the device must stay usable: a freshly
set-up context on the same medium solves correctly right afterwards."""
import ctypes

import numpy as np
import pytest

from tests._cases import Case, rand_complex, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,job", [("fp64", -1), ("mixed", -1), ("fp64", 0)])
def test_dependency_wait_runs_out_and_reports(prec, job):
    from paper_2604_19501_gb300 import _ffi

    lib = _ffi.load()
    c = Case((64, 48), abc=4, alpha3=1.05, seed=13, order="4th", intergrid="cubic")
    b = torch.from_numpy(rand_complex(c.hier.grids[2].shape, 3)).cuda()
    e = torch.empty_like(b)
    s = c.solver(precision=prec)
    st = lib.helm_coarse_wait_check(s._ctx, 1000000, job)
    if job == 0:
        # the first job is a leaf's forward job: nothing to wait for, the call refuses it
        assert st == _ffi.HELM_EINVAL
        s.close()
        return
    assert st == _ffi.HELM_OK, lib.helm_last_error()
    st = lib.helm_coarse_solve(s._ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(e.data_ptr()), 1)
    assert st == _ffi.HELM_ECUDA
    assert b"did not complete in time" in lib.helm_last_error()
    # recorded for the context: a later call through the cycle reports it again
    v = torch.from_numpy(rand_complex(c.grid.shape, 4)).cuda()
    st = lib.helm_cycle(s._ctx, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(torch.empty_like(v).data_ptr()), 1)
    assert st == _ffi.HELM_ECUDA
    s.close()
    torch.cuda.synchronize()   # the CUDA context is intact
    fresh = c.solver(precision=prec)
    got = fresh.coarse_solve(b)
    torch.cuda.synchronize()
    fresh.close()
    ref = c.hier.coarse_solve(b.cpu().numpy().ravel())
    assert rel(got.cpu().numpy().ravel(), ref) < 1e-10


def test_wait_check_rejects_bad_arguments():
    from paper_2604_19501_gb300 import _ffi

    lib = _ffi.load()
    c = Case((16, 16), abc=2, seed=8)
    s = c.solver()
    assert lib.helm_coarse_wait_check(s._ctx, 0, -1) == _ffi.HELM_EINVAL
    assert lib.helm_coarse_wait_check(s._ctx, 1000, 1 << 30) == _ffi.HELM_EINVAL
    assert lib.helm_coarse_wait_check(None, 1000, -1) == _ffi.HELM_EINVAL
    s.close()
