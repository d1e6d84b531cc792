"""The C-ABI library loads and exports every entry point that include/helm.h
declares; host-only calls behave as documented (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "helm.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|long long|const char\*)\s+(helm_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("helm_setup", "helm_solve", "helm_adjoint_grad", "helm_destroy", "helm_cycle",
              "helm_coarse_solve", "helm_apply", "helm_smooth", "helm_restrict", "helm_prolong_add"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2604_19501_gb300 import _ffi

    assert sorted(_ffi.SIGNATURES) == _declared()


def test_host_only_calls(lib):
    from paper_2604_19501_gb300 import _ffi

    l = _ffi.load()
    o = _ffi.HelmOpts()
    assert l.helm_default_opts(ctypes.byref(o)) == 0
    assert o.restart == 10 and o.nu1 == 1 and o.jacobi_w[0] == 0.8 and o.alpha3 == 1.0
    assert l.helm_strerror(_ffi.HELM_NOT_CONVERGED) == b"not converged"
    ctx = ctypes.c_void_p()
    k = (ctypes.c_double * 4)()
    o.dim = 5
    assert l.helm_setup(ctypes.byref(o), ctypes.cast(k, ctypes.c_void_p), ctypes.byref(ctx)) == _ffi.HELM_EINVAL
    assert b"dim" in l.helm_last_error()
    o.dim, o.n[0], o.n[1] = 2, 6, 8
    assert l.helm_setup(ctypes.byref(o), ctypes.cast(k, ctypes.c_void_p), ctypes.byref(ctx)) == _ffi.HELM_EINVAL
    assert l.helm_destroy(None) == 0


def _header_opts_fields():
    src = open(HEADER).read()
    body = re.search(r"typedef struct \{(.*?)\} helm_opts;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(",") if "," in decl else [decl]:
            m = re.search(r"(\w+)\s*(\[\d+\])?\s*$", part.strip())
            names.append(m.group(1))
    return names


def test_binding_opts_layout_follows_header():
    from paper_2604_19501_gb300 import _ffi

    assert [f[0] for f in _ffi.HelmOpts._fields_] == _header_opts_fields()


def test_solver_option_defaults_and_validation(lib):
    from paper_2604_19501_gb300 import _ffi

    l = _ffi.load()
    o = _ffi.HelmOpts()
    assert l.helm_default_opts(ctypes.byref(o)) == 0
    assert o.solver == _ffi.SOLVER["fgmres"] and o.fuse_cycle == 1 and o.graphs == 0 and o.cslp_beta == 0.0
    ctx = ctypes.c_void_p()
    k = (ctypes.c_double * 81)()
    o.dim, o.n[0], o.n[1] = 2, 8, 8
    o.solver = 7
    assert l.helm_setup(ctypes.byref(o), ctypes.cast(k, ctypes.c_void_p), ctypes.byref(ctx)) == _ffi.HELM_EINVAL
    assert b"solver" in l.helm_last_error()
    assert not ctx.value


@pytest.mark.parametrize("field,bad,word", [("coarse_refine", -1, b"coarse_refine"), ("coarse_refine", 9, b"coarse_refine"),
                                            ("coarse_block_min", -5, b"coarse_block_min"),
                                            ("arnoldi_passes", 3, b"arnoldi_passes"),
                                            ("arnoldi_passes", -1, b"arnoldi_passes")])
def test_new_option_defaults_and_ranges(lib, field, bad, word):
    """Defaults of the coarsest-solve refinement, the blocked-elimination threshold and the
    Arnoldi passes (0 = the library's choice), and their range checks before any device call."""
    from paper_2604_19501_gb300 import _ffi

    l = _ffi.load()
    o = _ffi.HelmOpts()
    assert l.helm_default_opts(ctypes.byref(o)) == 0
    assert o.coarse_refine == 0 and o.coarse_block_min == 0 and o.arnoldi_passes == 0
    ctx = ctypes.c_void_p()
    k = (ctypes.c_double * 81)()
    o.dim, o.n[0], o.n[1] = 2, 8, 8
    setattr(o, field, bad)
    assert l.helm_setup(ctypes.byref(o), ctypes.cast(k, ctypes.c_void_p), ctypes.byref(ctx)) == _ffi.HELM_EINVAL
    assert word in l.helm_last_error()
    assert not ctx.value
