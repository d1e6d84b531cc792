"""Writes ``shifts.json``: the real shifts handed to the solver for each
discretisation and ppw.

* 4th-order stencils with cubic / lev-dep transfers: the paper's Tables 1 and 2.
* 2nd-order stencil with full weighting / bilinear transfers (no published
  value): the min-max search of the grid-to-grid dispersion analysis (Sec. 4),
  run by the oracle, for the level-3 shift alpha3 and for the optional level-2
  shift alpha2.

Run: ``python -m workloads.make_shifts`` from the repository root.
"""
import json
import os

import numpy as np


def main():
    from oracle import dispersion as D

    out = {
        "source": {
            "4th": "Yovel & Treister, Table 1 (2D) and Table 2 (3D)",
            "2nd/fw": "oracle.dispersion.optimal_shift, min-max of Eq. minmax, bisection radius",
        },
        "2d": {"4th": {"cubic": {"10": 1.0140, "11": 1.0075, "12": 1.0045},
                        "levdep": {"10": 1.0290, "11": 1.0190, "12": 1.0135}},
               "2nd": {"fw": {}}},
        "3d": {"4th": {"cubic": {"10": 1.0130, "11": 1.0065, "12": 1.0045},
                        "levdep": {"10": 1.0245, "11": 1.0165, "12": 1.0120}},
               "2nd": {"fw": {}}},
    }
    alphas = np.round(np.arange(1.0, 1.25 + 1e-9, 5e-4), 6)
    for dim in (2, 3):
        for G in (10, 11, 12):
            a3, e3 = D.optimal_shift(dim, "2nd", G, "fw", alphas=alphas)
            a2, e2 = D.optimal_shift(dim, "2nd", G, "fw", alphas=alphas, level=2)
            out[f"{dim}d"]["2nd"]["fw"][str(G)] = {"alpha3": a3, "e_g3": e3, "alpha2": a2, "e_g2": e2}
            print(dim, G, a3, e3, a2, e2, flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "shifts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
