"""Host-only checks of the coarsest solve plan (no GPU): the nested-dissection tree and
the persistent solve kernel's job list, validated by the library against every extent
the kernel indexes and the job order its schedule relies on (a job's dependencies are
listed before it)."""
import pytest

pytest.importorskip("numpy")

from paper_2604_19501_gb300 import HelmError, coarse_plan


def _nd_entries(n, r, leaf_max):
    """Reference count of the stored factor entries: re-derive the nested-dissection
    tree in Python (the same bisection rule) and sum |S| x (|S| + |B|) per front."""
    import itertools

    dim = len(n)

    def ring(lo, hi):
        a = [max(0, lo[d] - r) for d in range(dim)]
        b = [min(n[d], hi[d] + r) for d in range(dim)]
        vol = 1
        for d in range(dim):
            vol *= b[d] - a[d]
        inner = 1
        for d in range(dim):
            inner *= hi[d] - lo[d]
        return vol - inner

    total = 0
    stack = [(tuple([0] * dim), tuple(n))]
    while stack:
        lo, hi = stack.pop()
        ext = [hi[d] - lo[d] for d in range(dim)]
        vol = 1
        for e in ext:
            vol *= e
        axis = max(range(dim), key=lambda d: (ext[d], -d))
        nB = ring(lo, hi)
        if vol <= leaf_max or ext[axis] < r + 2:
            nS = vol
        else:
            mid = lo[axis] + (ext[axis] - r) // 2
            nS = vol // ext[axis] * r
            left_hi = list(hi)
            left_hi[axis] = mid
            right_lo = list(lo)
            right_lo[axis] = mid + r
            stack.append((lo, tuple(left_hi)))
            if hi[axis] > right_lo[axis]:
                stack.append((tuple(right_lo), hi))
        total += nS * (nS + nB)
    return total


@pytest.mark.parametrize("n,r,sym,grid", [
    ((33, 33), 1, True, 304),       # 128^2 cells, 5-point / full weighting
    ((33, 33), 3, True, 304),       # 128^2 cells, 9-point / cubic
    ((273, 273), 3, True, 304),     # 1088^2 cells
    ((529, 529), 3, True, 304),     # 2112^2 cells
    ((529, 529), 3, True, 152),
    ((41, 23), 2, False, 7),        # ragged, unsymmetric storage, tiny grid
    ((17, 19, 13), 2, False, 304),  # 3D lev-dep (unsymmetric)
    ((17, 17, 17), 1, True, 64),
    ((49, 49, 19), 2, False, 608),  # 192 x 192 x 72 cells, lev-dep
    ((75, 75, 75), 2, False, 608),  # 296^3 cells (256^3 + 20-cell layer): fronts of up to 11,400 boundary nodes
])
def test_plan_valid(n, r, sym, grid):
    st = coarse_plan(n, r, symmetric=sym, grid=grid)
    assert st["fronts"] >= 1 and st["levels"] >= 1 and st["jobs"] >= 2 * st["fronts"]
    entries = _nd_entries(n, r, 64)
    # M [nS][nF] per front for the forward sweep, G^T [nB][nS] for the backward sweep
    assert st["factor_entries"] == entries + st["bwd_entries"]
    assert st["bwd_entries"] <= st["factor_entries"]


def test_plan_grid_independent_factors():
    a = coarse_plan((273, 273), 3, grid=152)
    b = coarse_plan((273, 273), 3, grid=608)
    assert a["factor_entries"] == b["factor_entries"] and a["fronts"] == b["fronts"]
    assert b["jobs"] >= a["jobs"]


def test_plan_rejects_bad_arguments():
    with pytest.raises(HelmError):
        coarse_plan((33, 33), 0)
    with pytest.raises(HelmError):
        coarse_plan((33, 33), 1, grid=0)


def test_plan_valid_on_seeded_random_grids():
    """Seeded random 2D and 3D coarsest grids (ragged sizes, radii 1-3, both storage
    forms, small and large resident grids): every plan passes the library's checks and
    stores the nested-dissection entry count re-derived above."""
    import numpy as np

    rng = np.random.default_rng(2604)
    for _ in range(24):
        dim = int(rng.integers(2, 4))
        n = tuple(int(v) for v in (rng.integers(5, 90, 2) if dim == 2 else rng.integers(5, 22, 3)))
        r = int(rng.integers(1, 4))
        sym = bool(rng.integers(0, 2))
        grid = int(rng.choice([1, 7, 152, 608]))
        st = coarse_plan(n, r, symmetric=sym, grid=grid)
        assert st["factor_entries"] == _nd_entries(n, r, 64) + st["bwd_entries"], (n, r)
        assert st["jobs"] >= 2 * st["fronts"]
