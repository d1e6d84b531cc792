"""The allocation-free coarsest solve (helm_coarse_solve_noalloc) gives the same answer
as helm_coarse_solve.

Some callers cannot allocate device memory while they run, for instance a host framework
that reserves all device memory at start-up, or a latency-sensitive loop that cannot
afford the synchronisation an allocation may cause.  This entry point keeps its scratch
in a fixed-size static device array instead.  The file is named to be collected last,
so a run that stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from tests._cases import Case, rand_complex, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _calls(lib, ctx, b, nrhs):
    e_ref = torch.empty_like(b)
    e_new = torch.empty_like(b)
    st = lib.helm_coarse_solve(ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(e_ref.data_ptr()), nrhs)
    assert st == 0, lib.helm_last_error()
    st = lib.helm_coarse_solve_noalloc(ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(e_new.data_ptr()), nrhs)
    assert st == 0, lib.helm_last_error()
    torch.cuda.synchronize()
    return e_ref.cpu().numpy(), e_new.cpu().numpy()


@pytest.mark.parametrize("n,order,ig", [((32, 24), "2nd", "fw"), ((48, 40), "4th", "cubic"),
                                        ((8, 8, 12), "4th", "levdep")])
def test_noalloc_matches_coarse_solve_twice(n, order, ig):
    from paper_2604_19501_gb300 import _ffi

    lib = _ffi.load()
    c = Case(n, abc=2, alpha3=1.05, seed=7, order=order, intergrid=ig)
    s = c.solver()
    shape3 = c.hier.grids[2].shape
    for call, nrhs in enumerate((1, 2)):   # two calls in a row, the second reuses the array
        b = torch.from_numpy(rand_complex((nrhs,) + shape3, 100 + call)).cuda()
        ref, new = _calls(lib, s._ctx, b, nrhs)
        assert rel(new, ref) < 1e-10
        oracle = np.stack([c.hier.coarse_solve(bi.ravel()).reshape(bi.shape) for bi in b.cpu().numpy()])
        assert rel(new, oracle) < 1e-10
    s.close()


def test_noalloc_rejects_oversize_request():
    from paper_2604_19501_gb300 import _ffi

    lib = _ffi.load()
    c = Case((16, 16), abc=2, seed=8)
    s = c.solver()
    nrhs = 50000   # 50000 x (25 + 25) scratch entries exceed the 2^20 of the static array
    b = torch.zeros((nrhs,) + c.hier.grids[2].shape, dtype=torch.complex128, device="cuda")
    e = torch.empty_like(b)
    st = lib.helm_coarse_solve_noalloc(s._ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(e.data_ptr()), nrhs)
    assert st == _ffi.HELM_EINVAL
    assert b"static array" in lib.helm_last_error()
    s.close()
