"""Geometric pins for the oracle's meshes: sphere area and volume converge
to 4 pi r^2 and 4/3 pi r^3 at O(h^2); closed shapes give closed, consistently
oriented meshes with the right Euler characteristic; and brute-force counts
of sign-change cells and crossing lattice edges, done here in numpy without
the oracle, agree with the oracle's mesh."""
import numpy as np
import pytest

import oracle
import meshutil
from paper_2111_05778_gb300 import synth


def _sphere_lattice(N, r=0.5):
    g = -1.0 + np.arange(N + 1) * (2.0 / N)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    return np.sqrt(X * X + Y * Y + Z * Z) - r


@pytest.mark.parametrize("N", [16, 32, 64, 128])
def test_sphere_brute_force_counts(N):
    F = _sphere_lattice(N)
    neg = F < 0
    cnt = np.zeros((N, N, N), np.int32)
    for b in range(8):
        x, y, z = b & 1, (b >> 1) & 1, (b >> 2) & 1
        cnt += neg[x : x + N, y : y + N, z : z + N]
    sign_change = int(((cnt > 0) & (cnt < 8)).sum())
    V = int((neg[1:] != neg[:-1]).sum() + (neg[:, 1:] != neg[:, :-1]).sum() + (neg[:, :, 1:] != neg[:, :, :-1]).sum())
    s = oracle.csg(synth.sphere_prims(0.5))
    hr, mr = oracle.polygonize(s, N)
    surf = mr.cells[(mr.cases > 0) & (mr.cases < 255)]
    assert surf.size == sign_change
    keys = mr.tri_keys
    assert np.unique(keys).size == V
    assert keys.shape[0] == 2 * V - 4  # Euler: a genus-0 surface, V - E + F = 2 with E = 3F/2
    assert meshutil.closed_oriented(keys)
    assert meshutil.euler(keys) == 2


def test_sphere_area_volume_converge_quadratically():
    s = oracle.csg(synth.sphere_prims(0.5))
    Ns = np.array([32, 64, 128, 256, 512])
    ea, ev = [], []
    for N in Ns:
        _, mr = oracle.polygonize(s, int(N))
        pos = mr.tri_pos
        ea.append(abs(meshutil.area(pos) - np.pi))
        ev.append(abs(meshutil.signed_volume(pos) - np.pi / 6))
        # normals point outwards (towards f > 0)
        n = np.cross(pos[:, 1] - pos[:, 0], pos[:, 2] - pos[:, 0])
        nz = np.linalg.norm(n, axis=1) > 1e-14
        assert (np.einsum("ij,ij->i", n[nz], pos.mean(1)[nz]) > 0).all()
    h = 2.0 / Ns
    sa = np.polyfit(np.log(h), np.log(ea), 1)[0]
    sv = np.polyfit(np.log(h), np.log(ev), 1)[0]
    assert sa >= 1.8 and sv >= 1.8, (sa, sv)


def test_csg_closed_where_inside_domain():
    s = oracle.csg(synth.csg_prims(0))
    N = 128
    _, mr = oracle.polygonize(s, N)
    keys = mr.tri_keys
    # boundary edges may only come from surfaces cut by the domain faces
    N1 = N + 1
    for a, b in meshutil.boundary_edges(keys):
        for k in (a, b):
            r = k % N1**3
            ax = k // N1**3
            coords = [r % N1, (r // N1) % N1, r // N1**2]
            on_face = any(c in (0, N) for i, c in enumerate(coords) if i != ax)
            assert on_face
    e = meshutil.directed_edges(keys)
    assert all(c == 1 for c in e.values())


def test_torus_euler_zero():
    rot = np.eye(3)
    prims = synth.prim_row(synth.TORUS, synth.UNION, [0.05, -0.02, 0.01], [0.5, 0.17], rot)[None, :]
    s = oracle.csg(prims)
    _, mr = oracle.polygonize(s, 64)
    assert meshutil.closed_oriented(mr.tri_keys)
    assert meshutil.euler(mr.tri_keys) == 0


def test_tie_convention_zero_is_outside():
    """C0 has six lattice corners with f == 0 exactly ((+-0.5,0,0) and
    permutations); they count as outside, giving t in [0, 1]."""
    s = oracle.csg(synth.sphere_prims(0.5))
    N = 64
    _, mr = oracle.polygonize(s, N)
    assert mr.min_abs_f == 0.0
    pos = mr.tri_pos.reshape(-1, 3)
    for p in ([0.5, 0, 0], [-0.5, 0, 0], [0, 0.5, 0], [0, -0.5, 0], [0, 0, 0.5], [0, 0, -0.5]):
        assert (np.abs(pos - np.array(p)).max(axis=1) < 1e-15).any()


def _golden_rows():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sphere_r05_counts.txt")
    rows = [list(map(int, l.split())) for l in open(path) if l.strip() and not l.startswith("#")]
    return np.array(rows, np.int64)


def test_golden_sphere_counts_consistent():
    rows = _golden_rows()
    N, ev, md, mh, surf, V, T = rows.T
    assert (T == 2 * V - 4).all()  # genus 0 at every N
    assert (surf <= mh).all() and (mh <= md).all()
    s = oracle.csg(synth.sphere_prims(0.5))
    for r in rows[N <= 128]:
        hr = oracle.hop(s, int(r[0]))
        assert hr.col_evals.sum() == r[1] and hr.marks.size == r[2]


def test_csg_adjoint_matches_implicit_fd():
    """Adjoint of the analytic scene w.r.t. centres and size parameters
    against central differences of the implicit loss (FP64, oracle evaluator
    only): L(theta') with v(theta') = v - (f(v;theta') - f(v;theta)) grad f/|grad f|^2."""
    prims = synth.csg_prims(5)
    s = oracle.csg(prims)
    N = 48
    _, mr = oracle.polygonize(s, N)
    keys, pos = mr.tri_keys.ravel(), mr.tri_pos.reshape(-1, 3)
    _, first = np.unique(keys, return_index=True)
    V = pos[first]
    c = np.array([0.03, -0.02, 0.01])
    r = np.linalg.norm(V - c, axis=1)
    dldv = (2 * (r - 0.4) / r)[:, None] * (V - c) / V.shape[0]
    g = s.adjoint(V, dldv)
    f0 = s.eval(V)
    h = 1e-7
    gx = np.stack([(s.eval(V + h * e) - s.eval(V - h * e)) / (2 * h) for e in np.eye(3)], 1)
    n2 = (gx * gx).sum(1)

    def implicit_loss(pp):
        f1 = oracle.csg(pp).eval(V)
        v = V - ((f1 - f0) / n2)[:, None] * gx
        return np.mean((np.linalg.norm(v - c, axis=1) - 0.4) ** 2)

    d = 1e-7
    checked = 0
    for i in range(prims.shape[0]):
        for slot in [2, 3, 4, 5, 6]:
            if prims[i, 0] == synth.SPHERE and slot == 6:
                continue
            hi = prims.copy()
            lo = prims.copy()
            hi[i, slot] += d
            lo[i, slot] -= d
            fd = (implicit_loss(hi) - implicit_loss(lo)) / (2 * d)
            assert abs(g[i, slot] - fd) <= 1e-5 * abs(fd) + 1e-6 * np.abs(g).max(), (i, slot, g[i, slot], fd)
            checked += 1
    assert checked > 100 and np.abs(g[:, 2:8]).max() > 0
