"""Pins for the oracle's Marching Cubes table (the paper polygonizes cells
with Marching Cubes, Sec. 3 and Sec. 5, but prints no table).

Checked against facts that do not come from the table generator itself:
cube symmetry, the classical triangle counts of unambiguous configurations,
edge usage, face-boundary structure, and closed, consistently oriented
meshes on random fields that exercise most of the 256 cases."""
import itertools

import numpy as np
import pytest

import oracle
import meshutil

CORNERS = np.array([[b & 1, (b >> 1) & 1, (b >> 2) & 1] for b in range(8)])


def _edges():
    out = []
    for e in range(12):
        ax, u, v = e // 4, e & 1, (e >> 1) & 1
        o = [a for a in range(3) if a != ax]
        c = [0, 0, 0]
        c[o[0]], c[o[1]] = u, v
        lo = c[0] + 2 * c[1] + 4 * c[2]
        out.append((lo, lo + (1 << ax), ax))
    return out


EDGES = _edges()


def _symmetries():
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product([1, -1], repeat=3):
            M = np.zeros((3, 3), int)
            for r, (p, s) in enumerate(zip(perm, signs)):
                M[r, p] = s
            mats.append(M)
    perms = []
    for M in mats:
        x = (2 * CORNERS - 1) @ M.T
        y = (x + 1) // 2
        idx = y[:, 0] + 2 * y[:, 1] + 4 * y[:, 2]
        perms.append(idx)
    return perms  # 48 corner permutations


def _map_case(c, perm):
    out = 0
    for b in range(8):
        if (c >> b) & 1:
            out |= 1 << int(perm[b])
    return out


def _ambiguous_face(c):
    for ax in range(3):
        for sd in range(2):
            fc = [b for b in range(8) if ((b >> ax) & 1) == sd]
            # diagonal pairs: corners differing in both other coordinates
            s = [(c >> b) & 1 for b in fc]
            a, b_, c_, d = fc  # ordered by index: (0,0),(1,0),(0,1),(1,1) in the face's axes
            if s[0] == s[3] and s[1] == s[2] and s[0] != s[1]:
                return True
    return False


@pytest.fixture(scope="module")
def table():
    return oracle.mc_table(16)


def test_table_size_and_trivial_cases(table):
    ntri, edges, mx = table
    assert ntri[0] == 0 and ntri[255] == 0
    assert mx <= 5  # at most 5 triangles per cell, as in classical Marching Cubes
    assert (ntri[1:255] >= 1).all()


def test_classical_counts(table):
    ntri, _, _ = table
    assert ntri[0b00000001] == 1  # one corner
    assert ntri[0b00000011] == 2  # two corners on one edge
    assert ntri[0b00000111] == 3  # three corners of a face
    assert ntri[0b00001111] == 2  # a whole face
    assert ntri[0b00010111] == 4  # a corner and its three neighbours (hexagon)
    assert ntri[0b10000001] == 2  # two opposite cube corners: two separate caps
    assert ntri[0b00001001] == 2  # face diagonal, negatives kept apart: two caps


def test_symmetry_invariance(table):
    ntri, _, _ = table
    perms = _symmetries()
    assert len(perms) == 48
    for c in range(256):
        for p in perms:
            assert ntri[_map_case(c, p)] == ntri[c]


def test_complement_of_unambiguous_cases(table):
    ntri, _, _ = table
    for c in range(256):
        if not _ambiguous_face(c):
            assert ntri[c] == ntri[255 - c], c


def test_edges_used_are_exactly_the_crossing_edges(table):
    ntri, edges, _ = table
    for c in range(256):
        crossing = {e for e, (a, b, _) in enumerate(EDGES) if ((c >> a) & 1) != ((c >> b) & 1)}
        used = set(edges[c, : ntri[c]].ravel().tolist())
        assert used == crossing, c


def test_case_boundary_lies_on_faces(table):
    """The open boundary of each cell's triangle fan is made of segments that
    each join two edges of one face; there are (crossings on faces)/2 of them."""
    ntri, edges, _ = table
    for c in range(1, 255):
        keys = edges[c, : ntri[c]]
        bnd = meshutil.boundary_edges(keys)
        nface_cross = 0
        for ax in range(3):
            for sd in range(2):
                fe = [e for e, (a, b, eax) in enumerate(EDGES)
                      if eax != ax and ((a >> ax) & 1) == sd and ((c >> a) & 1) != ((c >> b) & 1)]
                nface_cross += len(fe)
        assert len(bnd) * 2 == nface_cross, c
        for a, b in bnd:
            la, ha, axa = EDGES[a]
            lb, hb, axb = EDGES[b]
            common = [ax for ax in range(3)
                      if axa != ax and axb != ax and ((la >> ax) & 1) == ((lb >> ax) & 1)]
            assert common, (c, a, b)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_random_fields_closed_and_oriented(seed):
    N = 8
    rng = np.random.default_rng(seed)
    vals = rng.uniform(-1, 1, (N + 1,) * 3)
    for ax in range(3):
        idx = [slice(None)] * 3
        idx[ax] = 0
        vals[tuple(idx)] = 1.0
        idx[ax] = -1
        vals[tuple(idx)] = 1.0
    # oracle index a + (N+1)(b + (N+1)c) for vals[a, b, c]
    s = oracle.lattice(N, vals.transpose(2, 1, 0).ravel())
    r = oracle.enum(s, N)
    keys, pos = r.tri_keys, r.tri_pos
    assert keys.shape[0] > 500
    assert meshutil.closed_oriented(keys)
    # the enclosed (negative) region has positive volume when normals point to f > 0
    assert meshutil.signed_volume(pos) > 0
    n = np.cross(pos[:, 1] - pos[:, 0], pos[:, 2] - pos[:, 0])
    ln = np.linalg.norm(n, axis=1)
    ok = ln > 1e-12
    g = pos.mean(1)[ok]
    u = n[ok] / ln[ok, None]
    d = 1e-4
    frac = np.mean(s.eval(g + d * u) > s.eval(g - d * u))
    assert frac > 0.97
    assert len(set(r.cases.tolist())) > 120
