"""Pins for the oracle's capsule, capped cylinder, hexagonal prism and cone
(the primitives of the paper's first scene, Sec. 5.1, besides the sphere,
box and torus pinned elsewhere).

* The distance is checked against brute force: the distance to a dense set
  of points sampled on the primitive's surface, with the sampling's covering
  radius as the tolerance; the sign against an inside test written from the
  solid's inequalities.  For the solids of revolution the nearest surface
  point lies in the query's half-plane through the axis, so sampling the
  profile curve in that half-plane is enough and is tight; the prism is
  sampled in 3-D.
* Each primitive is an exact distance, hence 1-Lipschitz.
* Polygonized alone, each is a closed oriented genus-0 mesh whose volume
  converges to the closed form.
* The adjoint of a scene of all seven primitives matches central
  differences of the implicit loss (as for the sphere / torus / box scene).
"""
import numpy as np
import pytest

import meshutil
import oracle
from paper_2111_05778_gb300 import synth



def _rot(seed):
    q = np.random.default_rng(seed).standard_normal(4)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
        ]
    )


def _local(row, p):
    R = row[8:17].reshape(3, 3)
    return (p - row[2:5]) @ R.T


def _profile(kind, a, b, step=2e-5):
    """Dense points (rho, y) on the boundary of the half-plane profile of a
    solid of revolution (the axis itself excluded)."""
    if kind == synth.CAPSULE:  # a = H, b = r
        side = np.stack([np.full(int(2 * a / step) + 1, b), np.linspace(-a, a, int(2 * a / step) + 1)], 1)
        t = np.linspace(0, np.pi / 2, int(np.pi / 2 * b / step) + 1)
        top = np.stack([b * np.cos(t), a + b * np.sin(t)], 1)
        bot = np.stack([b * np.cos(t), -a - b * np.sin(t)], 1)
        return np.concatenate([side, top, bot])
    if kind == synth.CYLINDER:  # a = r, b = H
        side = np.stack([np.full(int(2 * b / step) + 1, a), np.linspace(-b, b, int(2 * b / step) + 1)], 1)
        r = np.linspace(0, a, int(a / step) + 1)
        return np.concatenate([side, np.stack([r, np.full_like(r, b)], 1), np.stack([r, np.full_like(r, -b)], 1)])
    if kind == synth.CONE:  # a = R, b = H
        r = np.linspace(0, a, int(a / step) + 1)
        base = np.stack([r, np.full_like(r, -b)], 1)
        n = int(np.hypot(a, 2 * b) / step) + 1
        t = np.linspace(0, 1, n)
        slant = np.stack([a * (1 - t), -b + 2 * b * t], 1)
        return np.concatenate([base, slant])
    raise ValueError(kind)


def _inside_revolution(kind, a, b, rho, y):
    if kind == synth.CAPSULE:
        return ((np.abs(y) <= a) & (rho < b)) | (np.hypot(rho, y - a) < b) | (np.hypot(rho, y + a) < b)
    if kind == synth.CYLINDER:
        return (rho < a) & (np.abs(y) < b)
    if kind == synth.CONE:
        return (y > -b) & (y < b) & (rho < a * (b - y) / (2 * b))
    raise ValueError(kind)


def _queries(seed, n, extent):
    return np.random.default_rng(seed).uniform(-extent, extent, (n, 3))


@pytest.mark.parametrize(
    "kind,a,b", [(synth.CAPSULE, 0.21, 0.13), (synth.CYLINDER, 0.17, 0.26), (synth.CONE, 0.23, 0.19), (synth.CONE, 0.3, 0.05)]
)
def test_revolution_distance_brute_force(kind, a, b):
    centre = np.array([0.11, -0.07, 0.05])
    row = synth.prim_row(kind, synth.UNION, centre, [a, b], _rot(kind))
    s = oracle.csg(row[None, :])
    prof = _profile(kind, row[5], row[6])
    P = _queries(7 + kind, 3000, 0.35) + row[2:5]
    q = _local(row, P)
    rho, y = np.hypot(q[:, 0], q[:, 2]), q[:, 1]
    best = np.full(P.shape[0], np.inf)
    for c in range(0, prof.shape[0], 4096):
        pr = prof[c : c + 4096]
        d = np.hypot(rho[:, None] - pr[None, :, 0], y[:, None] - pr[None, :, 1])
        best = np.minimum(best, d.min(1))
    f = s.eval(P)
    # the samples are at most 2e-5 apart along the profile
    assert np.abs(np.abs(f) - best).max() < 2e-5
    inside = _inside_revolution(kind, row[5], row[6], rho, y)
    assert ((f < 0) == inside).all()
    assert 0.02 < inside.mean() < 0.95


def _hexprism_surface(a, H, step):
    """Points covering the prism's surface: the six side rectangles and the
    two hexagonal caps, with spacing about ``step``."""
    pts = []
    half = a / np.sqrt(3.0)  # half the edge length
    u = np.linspace(-half, half, int(np.ceil(2 * half / step)) + 1)
    v = np.linspace(-H, H, int(np.ceil(2 * H / step)) + 1)
    U, Vv = np.meshgrid(u, v, indexing="ij")
    for k in range(6):
        th = k * np.pi / 3
        n = np.array([np.cos(th), np.sin(th)])  # (x, z) outward normal
        t = np.array([-n[1], n[0]])
        x = a * n[0] + U * t[0]
        z = a * n[1] + U * t[1]
        pts.append(np.stack([x.ravel(), Vv.ravel(), z.ravel()], 1))
    g = np.arange(-a * 2 / np.sqrt(3), a * 2 / np.sqrt(3) + step / 2, step)
    X, Z = np.meshgrid(g, g, indexing="ij")
    X, Z = X.ravel(), Z.ravel()
    keep = np.ones(X.shape, bool)
    for k in range(6):
        th = k * np.pi / 3
        keep &= X * np.cos(th) + Z * np.sin(th) <= a
    X, Z = X[keep], Z[keep]
    for yy in (-H, H):
        pts.append(np.stack([X, np.full_like(X, yy), Z], 1))
    # the hexagon's boundary ring at each cap, so the rims are covered exactly
    for yy in (-H, H):
        for k in range(6):
            th = k * np.pi / 3
            n = np.array([np.cos(th), np.sin(th)])
            t = np.array([-n[1], n[0]])
            pts.append(np.stack([a * n[0] + u * t[0], np.full_like(u, yy), a * n[1] + u * t[1]], 1))
    return np.concatenate(pts)


def test_hexprism_distance_brute_force():
    a, H = 0.19, 0.14
    row = synth.prim_row(synth.HEXPRISM, synth.UNION, [-0.05, 0.08, 0.02], [a, H], _rot(5))
    s = oracle.csg(row[None, :])
    step = 2.5e-3
    S = _hexprism_surface(row[5], row[6], step)
    P = _queries(11, 600, 0.4) + row[2:5]
    q = _local(row, P)
    best = np.full(P.shape[0], np.inf)
    for c in range(0, S.shape[0], 8192):
        d = np.linalg.norm(q[:, None, :] - S[None, c : c + 8192, :], axis=2)
        best = np.minimum(best, d.min(1))
    f = s.eval(P)
    # covering radius of a square grid of spacing `step`: step / sqrt(2)
    assert (np.abs(f) <= best + 1e-12).all()
    assert (np.abs(f) >= best - step / np.sqrt(2)).all()
    inside = np.abs(q[:, 1]) < row[6]
    for k in range(6):
        th = k * np.pi / 3
        inside &= q[:, 0] * np.cos(th) + q[:, 2] * np.sin(th) < row[5]
    assert ((f < 0) == inside).all()
    assert 0.05 < inside.mean() < 0.95


@pytest.mark.parametrize("kind", [synth.CAPSULE, synth.CYLINDER, synth.HEXPRISM, synth.CONE])
def test_new_primitives_are_one_lipschitz(kind):
    row = synth.prim_row(kind, synth.UNION, [0.02, 0.01, -0.03], [0.2, 0.15], _rot(kind + 20))
    s = oracle.csg(row[None, :])
    rng = np.random.default_rng(kind)
    P = rng.uniform(-0.5, 0.5, (4000, 3))
    Q = P + rng.normal(0, 0.05, P.shape)
    lip = np.abs(s.eval(P) - s.eval(Q)) / np.linalg.norm(P - Q, axis=1)
    assert lip.max() <= 1 + 1e-9
    assert lip.max() > 0.9  # an exact distance attains slope 1 along normals


def _closed_form_volume(kind, a, b):
    if kind == synth.CAPSULE:
        return np.pi * b * b * 2 * a + 4 / 3 * np.pi * b**3
    if kind == synth.CYLINDER:
        return np.pi * a * a * 2 * b
    if kind == synth.HEXPRISM:
        return 2 * np.sqrt(3) * a * a * 2 * b
    if kind == synth.CONE:
        return np.pi * a * a * 2 * b / 3
    raise ValueError(kind)


@pytest.mark.parametrize("kind", [synth.CAPSULE, synth.CYLINDER, synth.HEXPRISM, synth.CONE])
def test_new_primitives_mesh_closed_and_volume_converges(kind):
    row = synth.prim_row(kind, synth.UNION, [0.031, -0.017, 0.023], [0.37, 0.29], _rot(kind + 40))
    s = oracle.csg(row[None, :])
    exact = _closed_form_volume(kind, row[5], row[6])
    errs = []
    for N in (48, 96, 192):
        _, mr = oracle.polygonize(s, N)
        keys = mr.tri_keys
        assert meshutil.closed_oriented(keys)
        assert meshutil.euler(keys) == 2
        errs.append(abs(meshutil.signed_volume(mr.tri_pos) - exact) / exact)
    assert errs[2] < 0.01
    assert errs[1] < errs[0] and errs[2] < errs[1]


def test_primitive_scene_adjoint_matches_implicit_fd():
    """All seven primitives in one union; adjoint w.r.t. every centre and
    size parameter against central differences of the implicit loss."""
    prims = synth.primitive_scene(3)
    s = oracle.csg(prims)
    N = 48
    _, mr = oracle.polygonize(s, N)
    keys, pos = mr.tri_keys.ravel(), mr.tri_pos.reshape(-1, 3)
    _, first = np.unique(keys, return_index=True)
    V = pos[first]
    c = np.array([0.02, 0.01, -0.03])
    r = np.linalg.norm(V - c, axis=1)
    dldv = (2 * (r - 0.5) / r)[:, None] * (V - c) / V.shape[0]
    g = s.adjoint(V, dldv)
    f0 = s.eval(V)
    h = 1e-7
    gx = np.stack([(s.eval(V + h * e) - s.eval(V - h * e)) / (2 * h) for e in np.eye(3)], 1)
    n2 = (gx * gx).sum(1)

    def implicit_loss(pp):
        f1 = oracle.csg(pp).eval(V)
        v = V - ((f1 - f0) / n2)[:, None] * gx
        return np.mean((np.linalg.norm(v - c, axis=1) - 0.5) ** 2)

    d = 1e-6
    nparam = {synth.SPHERE: 1, synth.TORUS: 2, synth.BOX: 3}
    for i in range(prims.shape[0]):
        for slot in range(2, 5 + nparam.get(int(prims[i, 0]), 2)):
            hi = prims.copy()
            lo = prims.copy()
            hi[i, slot] += d
            lo[i, slot] -= d
            fd = (implicit_loss(hi) - implicit_loss(lo)) / (2 * d)
            assert abs(g[i, slot] - fd) <= 1e-4 * abs(fd) + 1e-5 * np.abs(g).max(), (i, slot, g[i, slot], fd)
    assert np.abs(g[:, 5:8]).max() > 0
