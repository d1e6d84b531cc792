"""The 3-level RS-CGC cycle used as a preconditioner (Algorithm TwoGrid applied
recursively, Sec. 2; cycle settings of Sec. 5).

Oracle module (test infrastructure only).

cycle(l, b, x):
    l = 3: return the exact solution of H_4h^alpha e = b
    x <- Relax^nu1(x);  r_c = R (b - H x)
    e = 0;  repeat g times: e <- cycle(l + 1, r_c, e)
    x <- x + P e;  x <- Relax^nu2(x)

g = 1 for a V-cycle and 2 for a W-cycle, except that the coarsest level is
always visited once per visit of level 2 (reading: the standard convention that
the coarsest "recursion" is one exact solve).  The preconditioner starts from
x = 0 on every level.
"""
import numpy as np

from . import smoothers


class Cycle:
    def __init__(self, hier, cycle="V", nu1=1, nu2=1, smoother="jacobi",
                 weights=(0.8, 0.8), rb_weight=1.0):
        self.h = hier
        self.kind = cycle
        self.nu1, self.nu2 = nu1, nu2
        self.smoother = smoother
        self.weights = tuple(weights)
        self.rb_weight = rb_weight
        self.colour = [smoothers.colours(g) for g in hier.grids[:2]]

    def relax(self, level, x, b):
        A, d = self.h.A[level], self.h.diag[level]
        if self.smoother == "jacobi":
            return smoothers.jacobi(A, d, x, b, self.weights[level])
        return smoothers.red_black(A, d, x, b, self.colour[level], self.rb_weight)

    def run(self, level, b, x=None):
        if level == 2:
            return self.h.coarse_solve(b)
        x = np.zeros_like(b) if x is None else np.array(x, copy=True)
        for _ in range(self.nu1):
            x = self.relax(level, x, b)
        rc = self.h.R[level] @ (b - self.h.A[level] @ x)
        g = 1 if (self.kind == "V" or level + 1 == 2) else 2
        e = None
        for _ in range(g):
            e = self.run(level + 1, rc, e)
        x = x + self.h.P[level] @ e
        for _ in range(self.nu2):
            x = self.relax(level, x, b)
        return x

    def __call__(self, b):
        """Apply the preconditioner: approximate H_h^-1 b."""
        return self.run(0, np.asarray(b, dtype=np.complex128))
