"""Mesh checks used by the tests (plain numpy; no polygonization arithmetic)."""
from collections import Counter

import numpy as np


def area(pos):
    """pos [T,3,3] -> total triangle area."""
    n = np.cross(pos[:, 1] - pos[:, 0], pos[:, 2] - pos[:, 0])
    return 0.5 * np.linalg.norm(n, axis=1).sum()


def signed_volume(pos):
    """Divergence theorem over oriented triangles: sum v0.(v1 x v2) / 6."""
    return np.einsum("ij,ij->i", pos[:, 0], np.cross(pos[:, 1], pos[:, 2])).sum() / 6.0


def directed_edges(keys):
    """keys [T,3] vertex ids -> Counter of directed edges."""
    e = Counter()
    for a, b, c in keys.tolist():
        e[(a, b)] += 1
        e[(b, c)] += 1
        e[(c, a)] += 1
    return e


def closed_oriented(keys):
    """True when every directed edge occurs once and its reverse occurs once:
    closed 2-manifold with consistent orientation (vertices deduplicated by key)."""
    e = directed_edges(keys)
    return all(c == 1 and e.get((b, a), 0) == 1 for (a, b), c in e.items())


def boundary_edges(keys):
    e = directed_edges(keys)
    return [(a, b) for (a, b), c in e.items() if e.get((b, a), 0) == 0]


def euler(keys):
    V = np.unique(keys).size
    e = directed_edges(keys)
    E = len({(min(a, b), max(a, b)) for (a, b) in e})
    return V - E + keys.shape[0]


def canonical_tris(keys):
    """Rotate each key triple so its smallest key comes first (orientation
    kept) and return a sorted structured view for multiset comparison."""
    k = np.asarray(keys, np.int64).reshape(-1, 3)
    r = np.argmin(k, axis=1)
    idx = (r[:, None] + np.arange(3)[None, :]) % 3
    rk = np.take_along_axis(k, idx, axis=1)
    order = np.lexsort((rk[:, 2], rk[:, 1], rk[:, 0]))
    return rk[order]


def vertex_table(keys, pos):
    """edge key -> position (first occurrence); keys [T,3], pos [T,3,3]."""
    k = keys.reshape(-1)
    p = pos.reshape(-1, 3)
    uk, first = np.unique(k, return_index=True)
    return uk, p[first]
