"""ctypes declarations of the C ABI in include/helm.h (argument marshalling only)."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libhelm.so")

HELM_OK, HELM_EINVAL, HELM_ENOMEM, HELM_NOT_CONVERGED, HELM_ECUDA, HELM_ENUMERIC = range(6)
STENCIL = {"2nd": 0, "4th": 1}
INTERGRID = {"fw": 0, "cubic": 1, "levdep": 2}
CYCLE = {"V": 0, "W": 1}
SMOOTHER = {"jacobi": 0, "redblack": 1, "rb": 1}
PRECISION = {"fp64": 0, "mixed": 1}
DTYPE = {"c128": 0, "c64": 1}
SOLVER = {"fgmres": 0, "cycle": 1}
INFO_KEYS = ["nodes1", "nodes2", "nodes3", "radius2", "radius3", "coarse_entries", "coarse_fronts",
             "coarse_levels", "coarse_bwd_entries", "double_float", "graphs", "cycle_kernels"]
CYCLE_KERNELS = ["tiles", "rows8", "rows16", "rows32"]
KERNEL_CLASSES = ["fine", "stencil", "transfer", "coarse", "arnoldi_matvec", "arnoldi_update",
                  "arnoldi_norm", "krylov_other", "setup"]


class HelmOpts(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("h", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("abc_width", ctypes.c_int * 6),
        ("abc_gamma_max", ctypes.c_double),
        ("alpha2", ctypes.c_double),
        ("alpha3", ctypes.c_double),
        ("stencil", ctypes.c_int),
        ("intergrid", ctypes.c_int),
        ("cycle", ctypes.c_int),
        ("nu1", ctypes.c_int),
        ("nu2", ctypes.c_int),
        ("smoother", ctypes.c_int),
        ("jacobi_w", ctypes.c_double * 2),
        ("rb_w", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("restart", ctypes.c_int),
        ("max_rhs", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("fuse_cycle", ctypes.c_int),
        ("graphs", ctypes.c_int),
        ("cslp_beta", ctypes.c_double),
        ("solver", ctypes.c_int),
        ("coarse_blocks", ctypes.c_int),
        ("coarse_refine", ctypes.c_int),
        ("coarse_block_min", ctypes.c_int),
        ("arnoldi_passes", ctypes.c_int),
    ]


class HelmStats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("relres", ctypes.c_double),
        ("est_relres", ctypes.c_double),
    ]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

# name -> (restype, argtypes); every entry point of include/helm.h
SIGNATURES = {
    "helm_default_opts": (_I, [ctypes.POINTER(HelmOpts)]),
    "helm_setup": (_I, [ctypes.POINTER(HelmOpts), _P, ctypes.POINTER(_P)]),
    "helm_destroy": (_I, [_P]),
    "helm_solve": (_I, [_P, _P, _P, _I, _D, _I, ctypes.POINTER(HelmStats)]),
    "helm_adjoint_grad": (_I, [_P, _P, _P, _I, _D, _I, _P, _P, ctypes.POINTER(HelmStats)]),
    "helm_apply": (_I, [_P, _I, _I, _P, _P, _I]),
    "helm_smooth": (_I, [_P, _I, _I, _P, _P, _I]),
    "helm_residual": (_I, [_P, _I, _I, _P, _P, _P, _I]),
    "helm_restrict": (_I, [_P, _I, _I, _P, _P, _I]),
    "helm_prolong_add": (_I, [_P, _I, _I, _P, _P, _I]),
    "helm_get_stencil": (_I, [_P, _I, _P, ctypes.POINTER(_I)]),
    "helm_coarse_solve": (_I, [_P, _P, _P, _I]),
    "helm_coarse_solve_noalloc": (_I, [_P, _P, _P, _I]),
    "helm_coarse_wait_check": (_I, [_P, ctypes.c_longlong, _I]),
    "helm_cycle": (_I, [_P, _P, _P, _I]),
    "helm_set_block": (_I, [_P, _I]),
    "helm_autotune_block": (_I, [_P, _P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "helm_set_cycle_kernels": (_I, [_P, _I]),
    "helm_autotune_cycle": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "helm_coarse_plan": (_I, [_I, ctypes.POINTER(_I), _I, _I, _I, _I, ctypes.POINTER(ctypes.c_longlong)]),
    "helm_launch_count": (ctypes.c_longlong, [_P]),
    "helm_info": (_I, [_P, _I, ctypes.POINTER(ctypes.c_longlong)]),
    "helm_timer_enable": (_I, [_P, ctypes.c_uint]),
    "helm_timer_read": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong)]),
    "helm_strerror": (ctypes.c_char_p, [_I]),
    "helm_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load():
    """Load libhelm.so (built in-tree); raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python paper_2604_19501_gb300/build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class HelmError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.helm_last_error().decode() or lib.helm_strerror(status).decode()
        super().__init__(f"{where}: {lib.helm_strerror(status).decode()} ({msg})")
        self.status = status


def check(status, where):
    if status != HELM_OK:
        raise HelmError(status, where)
    return status
