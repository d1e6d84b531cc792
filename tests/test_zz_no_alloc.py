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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,order,ig", [((32, 24), "2nd", "fw"), ((48, 40), "4th", "cubic"),
                                        ((8, 8, 12), "4th", "levdep")])
def test_noalloc_matches_coarse_solve_twice(n, order, ig, prec):
    """Calls in a row on the shared array: one right-hand side, then five (a full group of
    four that share each staged factor entry, plus a partial group of one).  A mixed-
    precision context applies its factors in double-float and keeps a double-float copy of
    the result in the array's tail."""
    from paper_2604_19501_gb300 import _ffi

    lib = _ffi.load()
    c = Case(n, abc=2, alpha3=1.05, seed=7, order=order, intergrid=ig)
    s = c.solver(precision=prec)
    shape3 = c.hier.grids[2].shape
    for call, nrhs in enumerate((1, 5)):   # two calls in a row, the second reuses the array
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
    # per right-hand side the solve needs the update vectors of every front, two vectors
    # over the 25 coarsest nodes and at least one 128-entry partial-sum block: more than
    # 178 entries, so 50000 right-hand sides exceed the 2^20 entries of the static array
    nrhs = 50000
    b = torch.zeros((nrhs,) + c.hier.grids[2].shape, dtype=torch.complex128, device="cuda")
    e = torch.empty_like(b)
    st = lib.helm_coarse_solve_noalloc(s._ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(e.data_ptr()), nrhs)
    assert st == _ffi.HELM_EINVAL
    assert b"static array" in lib.helm_last_error()
    s.close()


def test_noalloc_refuses_another_current_device():
    """The array's address is looked up per device, and the context's buffers live on the
    device it was set up on: a call with another device current is refused, not run."""
    from paper_2604_19501_gb300 import _ffi

    if torch.cuda.device_count() < 2:
        pytest.skip("needs two devices")
    lib = _ffi.load()
    c = Case((16, 16), abc=2, seed=8)
    s = c.solver()
    b = torch.from_numpy(rand_complex(c.hier.grids[2].shape, 5)).cuda()
    e = torch.empty_like(b)
    with torch.cuda.device(1):
        st = lib.helm_coarse_solve_noalloc(s._ctx, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(e.data_ptr()), 1)
    assert st == _ffi.HELM_EINVAL
    s.close()
