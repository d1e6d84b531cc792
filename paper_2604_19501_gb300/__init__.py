"""GB300 RS-CGC Helmholtz solver: Python binding of the C ABI (include/helm.h).

The binding only marshals arguments: every step of the method runs in the CUDA
library ``lib/libhelm.so`` (built by :mod:`paper_2604_19501_gb300.build`).  Vectors are
torch tensors on the GPU (complex128, or complex64 for the FP32 component calls) or
host numpy arrays where an entry point accepts host memory.  Importing this package
fails if the library has not been built.
"""
import ctypes

from . import _ffi
from ._ffi import HelmError, HelmOpts, HelmStats, check

__all__ = ["Solver", "HelmError", "level_shape", "helmholtz_solve", "release_reused_context", "coarse_plan",
           "solve_concurrent"]

_lib = _ffi.load()


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def level_shape(n, level):
    """Array shape (z, y, x order) of the nodes of level ``level`` (1 = fine)."""
    f = 2 ** (level - 1)
    return tuple(v // f + 1 for v in reversed(tuple(n)))


class Solver:
    """A set-up RS-CGC context (helm_setup) for one medium and frequency.

    ``kappa2``: slowness squared on the fine nodes (float64 torch CUDA tensor or
    numpy array), ``n``: cells per axis (x, y[, z]), ``omega``: angular frequency,
    ``abc_width``: absorbing-layer width (int for every face, or 6 per-face ints).
    Remaining keywords mirror ``helm_opts``.
    """

    def __init__(self, kappa2, n, omega, h=1.0, abc_width=0, abc_gamma_max=1.0, alpha2=1.0,
                 alpha3=1.0, stencil="2nd", intergrid="fw", cycle="V", nu=(1, 1),
                 smoother="jacobi", jacobi_w=(0.8, 0.8), rb_w=1.0, precision="fp64", restart=10,
                 max_rhs=1, stream=None, fuse_cycle=True, graphs=False, cslp_beta=0.0,
                 solver="fgmres", coarse_blocks=0, coarse_refine=0,
                 coarse_block_min=0, arnoldi_passes=0):
        self.n = tuple(int(v) for v in n)
        self.dim = len(self.n)
        o = HelmOpts()
        check(_lib.helm_default_opts(ctypes.byref(o)), "helm_default_opts")
        o.dim = self.dim
        for a, v in enumerate(self.n):
            o.n[a] = v
        o.h, o.omega = float(h), float(omega)
        widths = [int(abc_width)] * 6 if isinstance(abc_width, int) else [int(v) for v in abc_width]
        for f in range(6):
            o.abc_width[f] = widths[f] if f < 2 * self.dim else 0
        o.abc_gamma_max = float(abc_gamma_max)
        o.alpha2, o.alpha3 = float(alpha2), float(alpha3)
        o.stencil = _ffi.STENCIL[stencil]
        o.intergrid = _ffi.INTERGRID[intergrid]
        o.cycle = _ffi.CYCLE[cycle]
        o.nu1, o.nu2 = int(nu[0]), int(nu[1])
        o.smoother = _ffi.SMOOTHER[smoother]
        o.jacobi_w[0], o.jacobi_w[1] = float(jacobi_w[0]), float(jacobi_w[1])
        o.rb_w = float(rb_w)
        o.precision = _ffi.PRECISION[precision]
        o.restart = int(restart)
        o.max_rhs = int(max_rhs)
        self.max_rhs = int(max_rhs)
        o.fuse_cycle = int(bool(fuse_cycle))
        o.graphs = int(bool(graphs))
        o.cslp_beta = float(cslp_beta)
        o.solver = _ffi.SOLVER[solver]
        o.coarse_blocks = int(coarse_blocks)
        o.coarse_refine = int(coarse_refine)
        o.coarse_block_min = int(coarse_block_min)
        o.arnoldi_passes = int(arnoldi_passes)
        if stream is None:
            import torch

            stream = torch.cuda.current_stream().cuda_stream
        o.stream = ctypes.c_void_p(int(stream))
        self.opts = o
        self.precision = precision
        self._ctx = ctypes.c_void_p()
        check(_lib.helm_setup(ctypes.byref(o), _ptr(kappa2), ctypes.byref(self._ctx)), "helm_setup")

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            _lib.helm_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def shape(self, level=1):
        return level_shape(self.n, level)

    @property
    def launches(self):
        """Kernel launches issued by this context so far."""
        return int(_lib.helm_launch_count(self._ctx))

    def info(self):
        """Context facts (node counts, stencil radii, coarsest-factor size)."""
        out = {}
        for i, key in enumerate(_ffi.INFO_KEYS):
            v = ctypes.c_longlong()
            check(_lib.helm_info(self._ctx, i, ctypes.byref(v)), "helm_info")
            out[key] = v.value
        return out

    def timer_enable(self, classes=None):
        """Time every launch of the named kernel classes (all when None)."""
        names = _ffi.KERNEL_CLASSES if classes is None else classes
        mask = 0
        for nme in names:
            mask |= 1 << _ffi.KERNEL_CLASSES.index(nme)
        check(_lib.helm_timer_enable(self._ctx, mask), "helm_timer_enable")

    def timer_read(self):
        """{class: (total device ms, launches)} of the timed launches."""
        out = {}
        for i, nme in enumerate(_ffi.KERNEL_CLASSES):
            ms, cnt = ctypes.c_double(), ctypes.c_longlong()
            check(_lib.helm_timer_read(self._ctx, i, ctypes.byref(ms), ctypes.byref(cnt)), "helm_timer_read")
            out[nme] = (ms.value, cnt.value)
        return out

    # ------------------------------------------------------------------ solves
    def _nrhs(self, x, level=1):
        return x.numel() // _numel(self.shape(level)) if hasattr(x, "numel") else x.size // _numel(self.shape(level))

    def solve(self, q, p=None, tol=1e-6, maxit=500, raise_on_nonconvergence=False):
        """p = H^-1 q by FGMRES + RS-CGC (helm_solve).  q: complex128, shape
        (n_rhs,) + grid or grid; device tensor or host array.  Returns (p, stats)."""
        nrhs = self._nrhs(q)
        if p is None:
            p = _empty_like(q)
        stats = (HelmStats * nrhs)()
        st = _lib.helm_solve(self._ctx, _ptr(q), _ptr(p), nrhs, float(tol), int(maxit), stats)
        if st not in (_ffi.HELM_OK, _ffi.HELM_NOT_CONVERGED) or (st and raise_on_nonconvergence):
            check(st, "helm_solve")
        return p, [dict(iterations=s.iterations, converged=bool(s.converged), relres=s.relres,
                        est_relres=s.est_relres) for s in stats]

    def adjoint_grad(self, p, resid, grad, adj=None, tol=1e-6, maxit=500):
        """Accumulates dL/dkappa^2 into ``grad`` (helm_adjoint_grad); ``adj`` optionally
        receives the adjoint fields mu = conj(lambda).  Returns the adjoint-solve stats."""
        nrhs = self._nrhs(p)
        stats = (HelmStats * nrhs)()
        st = _lib.helm_adjoint_grad(self._ctx, _ptr(p), _ptr(resid), nrhs, float(tol), int(maxit),
                                    _ptr(grad), _ptr(adj), stats)
        if st not in (_ffi.HELM_OK, _ffi.HELM_NOT_CONVERGED):
            check(st, "helm_adjoint_grad")
        return [dict(iterations=s.iterations, converged=bool(s.converged), relres=s.relres) for s in stats]

    # ------------------------------------------------------------------ components
    @staticmethod
    def _dt(x):
        return _ffi.DTYPE["c64"] if str(x.dtype).endswith("complex64") else _ffi.DTYPE["c128"]

    def apply(self, level, x, y=None):
        y = _empty_like(x) if y is None else y
        check(_lib.helm_apply(self._ctx, level, self._dt(x), _ptr(x), _ptr(y), self._nrhs(x, level)), "helm_apply")
        return y

    def residual(self, level, b, x, r=None):
        r = _empty_like(x) if r is None else r
        check(_lib.helm_residual(self._ctx, level, self._dt(x), _ptr(b), _ptr(x), _ptr(r),
                                 self._nrhs(x, level)), "helm_residual")
        return r

    def smooth(self, level, b, x):
        """One smoothing sweep in place on x."""
        check(_lib.helm_smooth(self._ctx, level, self._dt(x), _ptr(b), _ptr(x), self._nrhs(x, level)),
              "helm_smooth")
        return x

    def restrict(self, level, rf, rc=None):
        import torch

        nrhs = self._nrhs(rf, level)
        if rc is None:
            rc = torch.empty((nrhs,) + self.shape(level + 1), dtype=rf.dtype, device=rf.device)
        check(_lib.helm_restrict(self._ctx, level, self._dt(rf), _ptr(rf), _ptr(rc), nrhs), "helm_restrict")
        return rc

    def prolong_add(self, level, ec, xf):
        check(_lib.helm_prolong_add(self._ctx, level, self._dt(ec), _ptr(ec), _ptr(xf),
                                    self._nrhs(xf, level)), "helm_prolong_add")
        return xf

    def stencil(self, level):
        """Assembled stencil of level 2 or 3 as a numpy complex128 array
        [ncoef, nodes] and its radius."""
        import numpy as np

        r = ctypes.c_int()
        check(_lib.helm_get_stencil(self._ctx, level, None, ctypes.byref(r)), "helm_get_stencil")
        ncoef = (2 * r.value + 1) ** self.dim
        out = np.empty((ncoef, _numel(self.shape(level))), dtype=np.complex128)
        check(_lib.helm_get_stencil(self._ctx, level, ctypes.c_void_p(out.ctypes.data), ctypes.byref(r)),
              "helm_get_stencil")
        return out, r.value

    def set_block(self, block):
        """Solve in FGMRES blocks of ``block`` right-hand sides (<= max_rhs)."""
        check(_lib.helm_set_block(self._ctx, int(block)), "helm_set_block")

    def autotune_block(self, q, probe_iters=0):
        """Time one FGMRES restart cycle for blocks of 1, 2, 4, ... right-hand sides of
        ``q`` (device tensor [n_rhs, ...]) and keep the fastest per right-hand side.
        Returns (block, {block: ms per right-hand side and iteration})."""
        n_rhs = self._nrhs(q)
        best = ctypes.c_int(0)
        costs = (ctypes.c_double * 7)()
        check(_lib.helm_autotune_block(self._ctx, _ptr(q), n_rhs, int(probe_iters), ctypes.byref(best), costs),
              "helm_autotune_block")
        cap = min(self.max_rhs, n_rhs)
        cands = []
        b = 1
        while b < cap:
            cands.append(b)
            b *= 2
        cands.append(cap)
        return best.value, {c: costs[i] for i, c in enumerate(cands[:7])}

    def set_cycle_kernels(self, kind):
        """Kernels of the fused cycle's fine passes: "tiles", "rows8", "rows16" or "rows32"."""
        check(_lib.helm_set_cycle_kernels(self._ctx, _ffi.CYCLE_KERNELS.index(kind)), "helm_set_cycle_kernels")

    def autotune_cycle(self, n_rhs=1):
        """Time the fused cycle's fine passes with every kernel kind and keep the fastest.
        Returns (kind, {kind: ms per down + up pair})."""
        best = ctypes.c_int(0)
        ms = (ctypes.c_double * 4)()
        check(_lib.helm_autotune_cycle(self._ctx, int(n_rhs), ctypes.byref(best), ms), "helm_autotune_cycle")
        return _ffi.CYCLE_KERNELS[best.value], {k: ms[i] for i, k in enumerate(_ffi.CYCLE_KERNELS)}

    def coarse_solve(self, b, e=None):
        e = _empty_like(b) if e is None else e
        check(_lib.helm_coarse_solve(self._ctx, _ptr(b), _ptr(e), self._nrhs(b, 3)), "helm_coarse_solve")
        return e

    def cycle(self, v, z=None):
        z = _empty_like(v) if z is None else z
        check(_lib.helm_cycle(self._ctx, _ptr(v), _ptr(z), self._nrhs(v)), "helm_cycle")
        return z


PLAN_KEYS = ("fronts", "levels", "jobs", "factor_entries", "bwd_entries", "part_blocks", "split_outputs",
             "max_boundary")


def solve_concurrent(solvers, qs, ps=None, tol=1e-6, maxit=500, executor=None):
    """Solves one problem per context at the same time (grids of different sizes, for
    instance): each helm_solve runs from its own host thread on its context's stream (the
    library is called with the interpreter lock released), so the kernels of different
    contexts overlap on the GPU.  Give the contexts distinct streams and, so that their
    coarsest solves can run side by side, a share of the device each (``coarse_blocks``).
    ``ps``: optional output tensors; ``executor``: an optional thread pool to reuse.
    Returns ``[(p, stats)]`` in the order of ``solvers``."""
    from concurrent.futures import ThreadPoolExecutor

    ps = list(ps) if ps is not None else [None] * len(solvers)
    own = executor is None
    ex = ThreadPoolExecutor(max_workers=max(1, len(solvers))) if own else executor
    try:
        futs = [ex.submit(s.solve, q, p, tol, maxit) for s, q, p in zip(solvers, qs, ps)]
        return [f.result() for f in futs]
    finally:
        if own:
            ex.shutdown()


def coarse_plan(n_nodes, radius, leaf_max=64, symmetric=True, grid=304):
    """Host-only plan of the coarsest-level direct solve (helm_coarse_plan): the
    nested-dissection tree and the solve kernel's job list for a level-3 grid of
    ``n_nodes`` nodes per axis (x first), checked against the kernel's extents."""
    dim = len(n_nodes)
    nn = (ctypes.c_int * 3)(*(list(n_nodes) + [1] * (3 - dim)))
    st = (ctypes.c_longlong * 8)()
    check(_lib.helm_coarse_plan(dim, nn, int(radius), int(leaf_max), int(bool(symmetric)), int(grid), st),
          "helm_coarse_plan")
    return dict(zip(PLAN_KEYS, list(st)))


def _numel(shape):
    n = 1
    for v in shape:
        n *= v
    return n


def _empty_like(x):
    if hasattr(x, "data_ptr"):
        import torch

        return torch.empty_like(x)
    import numpy as np

    return np.empty_like(x)


def _autograd_function():
    import torch

    class HelmholtzSolve(torch.autograd.Function):
        """p = H(kappa2)^-1 q with the adjoint-state backward.

        forward: set-up for kappa2, then helm_solve.  backward: helm_adjoint_grad with
        the incoming gradient as residual, giving dL/dkappa2 and, as conj(mu), dL/dq.
        ``recompute=True`` keeps only q and solves for p again in the backward (less
        memory, one more forward solve)."""

        @staticmethod
        def forward(ctx, kappa2, q, opts, tol, maxit, recompute, reuse):
            solver = _context_for(kappa2, opts) if reuse else Solver(kappa2.detach().contiguous(), **opts)
            qd = q.detach().contiguous()
            p, _ = solver.solve(qd, tol=tol, maxit=maxit)
            ctx.solver, ctx.tol, ctx.maxit, ctx.recompute = solver, tol, maxit, recompute
            ctx.save_for_backward(qd if recompute else p)
            return p

        @staticmethod
        def backward(ctx, grad_p):
            (saved,) = ctx.saved_tensors
            solver = ctx.solver
            p = solver.solve(saved, tol=ctx.tol, maxit=ctx.maxit)[0] if ctx.recompute else saved
            grad_k = torch.zeros(solver.shape(1), dtype=torch.float64, device=p.device)
            adj = torch.empty_like(p)
            solver.adjoint_grad(p, grad_p.contiguous(), grad_k, adj, tol=ctx.tol, maxit=ctx.maxit)
            grad_q = adj.conj() if ctx.needs_input_grad[1] else None
            ctx.solver = None   # a context of its own is freed here, a reused one stays in the cache
            return grad_k, grad_q, None, None, None, None, None

    return HelmholtzSolve


_HELMHOLTZ_SOLVE = None
# the context kept for reuse: the kappa2 tensor it was set up from (weak reference), that
# tensor's version counter at set-up, the options, and the context
_REUSE = {"ref": None, "version": None, "key": None, "solver": None}


def _context_for(kappa2, opts):
    """A context for kappa2 and opts: the kept one when it was set up from this very tensor
    object, unmodified since (same autograd version counter), with the same options;
    otherwise a new one, which replaces it (the old one is freed once no backward pass
    holds it)."""
    import weakref

    key = repr(sorted(opts.items()))
    r = _REUSE
    if (r["solver"] is not None and r["ref"] is not None and r["ref"]() is kappa2
            and r["version"] == kappa2._version and r["key"] == key):
        return r["solver"]
    solver = Solver(kappa2.detach().contiguous(), **opts)
    r.update(ref=weakref.ref(kappa2), version=kappa2._version, key=key, solver=solver)
    return solver


def release_reused_context():
    """Frees the context helmholtz_solve(..., reuse_context=True) keeps (once no backward
    pass still holds it)."""
    _REUSE.update(ref=None, version=None, key=None, solver=None)


def helmholtz_solve(kappa2, q, n, omega, tol=1e-6, maxit=500, recompute=False, reuse_context=False, **opts):
    """Differentiable p = H(kappa2)^-1 q (torch.autograd): the backward pass is the
    adjoint solve of helm_adjoint_grad.  ``opts`` are Solver keywords.

    By default every call sets up a context for kappa2 (the medium usually changes from one
    call to the next).  ``reuse_context=True`` keeps the last context and uses it again
    while the same kappa2 tensor object, unmodified (its autograd version counter
    unchanged), comes with the same options: several sources or data sets for one medium
    then pay for one set-up.  Changes made through ``.data`` bypass the version counter; call
    release_reused_context() after such a change.  The kept context is one context: calls
    that reuse it, and their backward passes, must not run at the same time from several
    host threads."""
    global _HELMHOLTZ_SOLVE
    if _HELMHOLTZ_SOLVE is None:
        _HELMHOLTZ_SOLVE = _autograd_function()
    o = dict(opts, n=n, omega=omega)
    return _HELMHOLTZ_SOLVE.apply(kappa2, q, o, tol, maxit, recompute, bool(reuse_context))
