"""The oracle's continuation method (Sec. 2: crawl the surface from a seed
cell) against its enumeration: on a closed surface of one component the
crawl finds exactly the sign-change cells and the same triangles; one seed
finds one component and never another; a seed whose search line has no sign
change finds nothing."""
import numpy as np

import meshutil
import oracle
from paper_2111_05778_gb300 import synth


def _same_mesh(a, b):
    assert np.array_equal(np.sort(a.cells[(a.cases > 0) & (a.cases < 255)]), np.sort(b.cells))
    assert np.array_equal(meshutil.canonical_tris(a.tri_keys), meshutil.canonical_tris(b.tri_keys))


def test_one_component_equals_enumeration():
    scenes = [synth.sphere_prims(0.5, (0.03, -0.02, 0.01)),
              synth.prim_row(synth.TORUS, synth.UNION, [0.0, 0.1, 0.0], [0.5, 0.15], synth._quat_rot([1, 0.3, 0.2, 0.1]))[None],
              synth.primitive_scene(0)[:1]]
    for prims in scenes:
        o = oracle.csg(prims)
        for N in (33, 64):
            c = prims[0, 2:5]
            seed = c + np.array([0.0, 0.0, 0.0])
            r = oracle.cont(o, N, [seed])
            assert r.col_evals[0] >= 0
            e = oracle.enum(o, N)
            _same_mesh(r, e)
            # only surface cells are visited: the crawl is O(N^2)
            assert ((r.cases > 0) & (r.cases < 255)).all()


def test_one_seed_one_component():
    a = synth.sphere_prims(0.3, (-0.45, 0.0, 0.0))
    b = synth.sphere_prims(0.3, (0.45, 0.0, 0.0))
    both = np.concatenate([a, b])
    N = 48
    o = oracle.csg(both)
    r = oracle.cont(o, N, [[-0.45, 0.0, 0.0]])  # inside the left sphere
    ea = oracle.enum(oracle.csg(a), N)
    _same_mesh(r, ea)
    r2 = oracle.cont(o, N, [[-0.45, 0.0, 0.0], [0.45, 0.0, 0.0]])
    _same_mesh(r2, oracle.enum(o, N))
    # the second seed of the same component adds nothing
    r3 = oracle.cont(o, N, [[-0.45, 0.0, 0.0], [-0.5, 0.05, 0.0]])
    _same_mesh(r3, ea)


def test_seed_without_crossing():
    o = oracle.csg(synth.sphere_prims(0.3, (-0.5, 0.0, 0.0)))
    r = oracle.cont(o, 32, [[0.5, 0.9, 0.9]])  # the +x line from here misses the sphere
    assert r.col_evals[0] == -1
    assert r.cells.size == 0 and r.tri_keys.shape[0] == 0


def _components(o, N, lo=-1.0, hi=1.0):
    """Brute force: f at all lattice points, the sign-change cells, and their
    connected components under "the shared face has both signs" (scipy
    connected_components) -> (cell ids, component label per cell)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    h = (hi - lo) / N
    g = np.arange(N + 1) * h + lo
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    neg = (o.eval(np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)) < 0).reshape(N + 1, N + 1, N + 1)
    cnt = sum(neg[di:di + N, dj:dj + N, dk:dk + N].astype(int) for di in (0, 1) for dj in (0, 1) for dk in (0, 1))
    surf = (cnt > 0) & (cnt < 8)
    ids = np.arange(N ** 3).reshape(N, N, N)
    rows, cols = [], []
    for ax in range(3):
        # the face between cell c and c + e_ax is the lattice square at index c[ax] + 1 on that axis
        sl = [slice(None)] * 3
        sl[ax] = slice(1, N + 1)
        fneg = neg[tuple(sl)]
        other = [a for a in range(3) if a != ax]
        fc = 0
        for d0 in (0, 1):
            for d1 in (0, 1):
                sl2 = [slice(0, N)] * 3
                sl2[ax] = slice(0, N)
                sl2[other[0]] = slice(d0, d0 + N)
                sl2[other[1]] = slice(d1, d1 + N)
                fc = fc + fneg[tuple(sl2)].astype(int)
        mixed = (fc > 0) & (fc < 4)
        sa = [slice(0, N)] * 3
        sa[ax] = slice(0, N - 1)
        sb = [slice(0, N)] * 3
        sb[ax] = slice(1, N)
        m = mixed[tuple(sa)]
        rows.append(ids[tuple(sa)][m])
        cols.append(ids[tuple(sb)][m])
    r, c = np.concatenate(rows), np.concatenate(cols)
    A = coo_matrix((np.ones(r.size), (r, c)), shape=(N ** 3, N ** 3))
    _, lab = connected_components(A, directed=False)
    cells = ids[surf]
    return cells, lab[cells]


def test_seeded_components_equal_brute_force_components():
    """The analytic scene of the benchmark (24 spheres, 8 tori, 4 boxes, several
    separate components): the crawl from seeds near every primitive finds
    exactly the union of the brute-force components of its seed cells."""
    prims = synth.csg_prims(0)
    o = oracle.csg(prims)
    N = 48
    seeds = prims[:, 2:5].copy()
    seeds[:, 0] -= 0.3
    r = oracle.cont(o, N, seeds)
    cells, lab = _components(o, N)
    seed_cells = r.col_evals[r.col_evals >= 0]
    assert seed_cells.size >= 20 and np.isin(seed_cells, cells).all()
    want = cells[np.isin(lab, lab[np.isin(cells, seed_cells)])]
    got = r.cells
    assert np.array_equal(np.sort(got), np.sort(want))
    assert np.unique(lab).size > 1  # the scene has more than one component
