"""Brute-force dense constructions from the definitions, by explicit loops over
nodes.  Used only to pin the oracle on tiny grids; shares no code with it."""
import itertools

import numpy as np


def nodes(n):
    """All node index tuples (x first) of a grid with ``n`` cells per axis, in
    flat order (x fastest)."""
    axes = [range(v + 1) for v in reversed(n)]
    for rev in itertools.product(*axes):
        yield tuple(reversed(rev))


def flat(node, n):
    f, s = 0, 1
    for k, v in enumerate(node):
        f += v * s
        s *= n[k] + 1
    return f


def inside(node, n):
    return all(0 <= v <= n[k] for k, v in enumerate(node))


def dense_operator(n, h, lap, mass, c):
    """Dense H with H[i, i+o] = lap[o] - mass[o] (c_i + c_{i+o}) / 2 for in-grid
    pairs; ``lap`` / ``mass`` are dicts offset -> weight, ``c`` a flat array."""
    N = int(np.prod([v + 1 for v in n]))
    A = np.zeros((N, N), dtype=np.complex128)
    for node in nodes(n):
        i = flat(node, n)
        for off in set(lap) | set(mass):
            nb = tuple(a + b for a, b in zip(node, off))
            if not inside(nb, n):
                continue
            j = flat(nb, n)
            A[i, j] += lap.get(off, 0.0) - mass.get(off, 0.0) * 0.5 * (c[i] + c[j])
    return A


def dense_restriction(n, w1):
    """Dense tensor-product restriction with 1D weights w1 (dict offset->w)."""
    nc = tuple(v // 2 for v in n)
    Nf = int(np.prod([v + 1 for v in n]))
    Nc = int(np.prod([v + 1 for v in nc]))
    R = np.zeros((Nc, Nf))
    for I in nodes(nc):
        for offs in itertools.product(sorted(w1), repeat=len(n)):
            i = tuple(2 * a + o for a, o in zip(I, offs))
            if inside(i, n):
                R[flat(I, nc), flat(i, n)] += np.prod([w1[o] for o in offs])
    return R
