"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no polygonization arithmetic: it only draws the parameters
of the shapes the benchmarks and tests polygonize, with numpy's PCG64
``default_rng``.  Every value is rounded to float32 once, so the CUDA path
(float32) and the FP64 oracle see exactly the same function.

Shapes (the paper's learned SDBs and scenes are not available, Sec. 5):

* ``sphere_prims``: one sphere, f = |p - c| - r.
* ``csg_prims(seed)``: the union (min, Sec. 4.3) of 24 spheres and 8 randomly
  rotated tori, minus 4 axis-aligned boxes (max with -d_box).
* ``mlp_params(seed, width)``: f(p) = (|p| - 0.6 + 0.1 g(p)) / 1.1 where g is
  a ReLU MLP 3 -> W -> ... -> W -> 1 (six W-wide layers) with Gaussian weights,
  each matrix divided by its largest singular value (so g and f are
  1-Lipschitz, i.e. signed distance bounds, Sec. 1) and N(0, 0.01^2) biases.
* ``batch_items()``: 64 (kind, seed, N, width) items mixing both generators.
* ``paper_network(seed)``: the paper's own network architecture (Sec. 5.2:
  3 -> 64, six 64 -> 64, 64 -> 1, ReLU, batch normalisation after every layer
  but the last) trained with Adam on point-distance samples of a seeded
  shape (a union of four spheres; the paper's Thingi10K shapes are not
  available), normalisation folded into the weights; SDB = network / 1.5.
* ``primitive_scene(seed)``: the seven basic primitives of the paper's first
  scene (Sec. 5.1: sphere, cube, cone, cylinder, torus, hexagonal prism and
  capsule), one of each, randomly rotated, in a union.

Primitive rows are 17 float64 numbers:
``type, op, cx, cy, cz, p0, p1, p2, rot[9]`` with type 0 sphere (p0 = r),
1 torus around the local y axis (p0 = R, p1 = r), 2 box (half sizes p0..p2),
3 capsule (segment (0,-p0,0)-(0,p0,0), radius p1), 4 capped cylinder around
the local y axis (radius p0, half height p1), 5 hexagonal prism (apothem p0 in
the local xz-plane, half height p1), 6 cone (base radius p0 at y = -p1, apex
at y = +p1);
op 0 union, 1 subtract, 2 intersect, applied as a left fold; ``rot`` maps
world offsets to the primitive's local frame (row-major).
"""
from __future__ import annotations

import numpy as np

PRIM_STRIDE = 17
SPHERE, TORUS, BOX, CAPSULE, CYLINDER, HEXPRISM, CONE = 0, 1, 2, 3, 4, 5, 6
UNION, SUBTRACT, INTERSECT = 0, 1, 2

MLP_R0, MLP_ALPHA, MLP_BETA = 0.6, 0.1, 1.1
MLP_NMID = 5  # W x W layers between the 3 -> W input layer and the W -> 1 output


def _f32(a):
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def prim_row(kind, op, centre, params, rot=None) -> np.ndarray:
    r = np.zeros(PRIM_STRIDE, np.float64)
    r[0], r[1] = kind, op
    r[2:5] = centre
    p = np.zeros(3)
    p[: len(params)] = params
    r[5:8] = p
    r[8:17] = (np.eye(3) if rot is None else np.asarray(rot, np.float64)).ravel()
    return _f32(r)


def sphere_prims(r=0.5, centre=(0.0, 0.0, 0.0)) -> np.ndarray:
    return prim_row(SPHERE, UNION, centre, [r])[None, :]


def half_space_prims(normal, offset, big=64.0) -> np.ndarray:
    """The half-space n.p <= offset as a huge box whose one face is the plane
    n.p = offset (the exact box distance then equals the plane distance of
    Eq. 5 everywhere inside the polygonization volume)."""
    n = np.asarray(normal, np.float64)
    n = n / np.linalg.norm(n)
    # build a rotation whose first row is n (local x axis = plane normal)
    a = np.eye(3)[np.argmin(np.abs(n))]
    u = np.cross(n, a)
    u /= np.linalg.norm(u)
    v = np.cross(n, u)
    rot = np.stack([n, u, v])
    centre = n * (offset - big)
    return prim_row(BOX, UNION, centre, [big, big, big], rot)[None, :]


def _quat_rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
        ]
    )


def csg_prims(seed: int, n_sphere=24, n_torus=8, n_box=4) -> np.ndarray:
    """CSG scene: draw order spheres (centre U[-0.7,0.7]^3, r U[0.05,0.2]),
    tori (centre, R U[0.1,0.3], r U[0.02,0.06], rotation from a normalised
    4-D Gaussian quaternion), boxes (centre, half sizes U[0.05,0.15] each,
    axis-aligned, subtracted)."""
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n_sphere):
        c = rng.uniform(-0.7, 0.7, 3)
        r = rng.uniform(0.05, 0.2)
        rows.append(prim_row(SPHERE, UNION, c, [r]))
    for _ in range(n_torus):
        c = rng.uniform(-0.7, 0.7, 3)
        R = rng.uniform(0.1, 0.3)
        r = rng.uniform(0.02, 0.06)
        rot = _quat_rot(rng.standard_normal(4))
        rows.append(prim_row(TORUS, UNION, c, [R, r], rot))
    for _ in range(n_box):
        c = rng.uniform(-0.7, 0.7, 3)
        hs = rng.uniform(0.05, 0.15, 3)
        rows.append(prim_row(BOX, SUBTRACT, c, hs))
    return np.stack(rows)


def primitive_scene(seed: int = 0) -> np.ndarray:
    """One of each of the seven primitives, centres at the middle and on a
    hexagon of radius 0.55 in the xy-plane (z U[-0.15,0.15]), each under a
    rotation from a normalised 4-D Gaussian quaternion, sizes drawn in the
    order sphere r U[0.18,0.25]; box half sizes U[0.12,0.2]; cone R
    U[0.15,0.22], H U[0.15,0.22]; cylinder r U[0.1,0.18], H U[0.12,0.2];
    torus R U[0.14,0.2], r U[0.04,0.07]; prism a U[0.1,0.18], H U[0.1,0.18];
    capsule H U[0.08,0.15], r U[0.06,0.1]."""
    rng = np.random.default_rng(seed)
    ang = np.arange(6) * (np.pi / 3)
    centres = [np.zeros(2)] + [0.55 * np.array([np.cos(a), np.sin(a)]) for a in ang]
    kinds = [SPHERE, BOX, CONE, CYLINDER, TORUS, HEXPRISM, CAPSULE]
    rows = []
    for kind, cxy in zip(kinds, centres):
        c = np.array([cxy[0], cxy[1], rng.uniform(-0.15, 0.15)])
        rot = _quat_rot(rng.standard_normal(4))
        if kind == SPHERE:
            prm = [rng.uniform(0.18, 0.25)]
        elif kind == BOX:
            prm = rng.uniform(0.12, 0.2, 3)
        elif kind == CONE:
            prm = [rng.uniform(0.15, 0.22), rng.uniform(0.15, 0.22)]
        elif kind == CYLINDER:
            prm = [rng.uniform(0.1, 0.18), rng.uniform(0.12, 0.2)]
        elif kind == TORUS:
            prm = [rng.uniform(0.14, 0.2), rng.uniform(0.04, 0.07)]
        elif kind == HEXPRISM:
            prm = [rng.uniform(0.1, 0.18), rng.uniform(0.1, 0.18)]
        else:
            prm = [rng.uniform(0.08, 0.15), rng.uniform(0.06, 0.1)]
        rows.append(prim_row(kind, UNION, c, prm, rot))
    return np.stack(rows)


def mixed_prims(seed: int, n: int = 96) -> np.ndarray:
    """Many-primitive CSG scene of all seven kinds: draw order per primitive
    kind U{0..6}, centre U[-0.7,0.7]^3, rotation from a normalised 4-D
    Gaussian quaternion, sizes U[0.04,0.16] (a, b, c in the kind's parameter
    order), op union (first primitive, then with probability 0.8) else
    subtract; the fold ends with an intersection with a box of half sizes
    U[0.6,0.8]^3 at the origin."""
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(n):
        kind = int(rng.integers(0, 7))
        c = rng.uniform(-0.7, 0.7, 3)
        rot = _quat_rot(rng.standard_normal(4))
        prm = rng.uniform(0.04, 0.16, 3)
        op = UNION if i == 0 or rng.uniform() < 0.8 else SUBTRACT
        rows.append(prim_row(kind, op, c, prm if kind == BOX else prm[:2], rot))
    rows.append(prim_row(BOX, INTERSECT, np.zeros(3), rng.uniform(0.6, 0.8, 3), _quat_rot(rng.standard_normal(4))))
    return np.stack(rows)


PAPER_WIDTH, PAPER_NMID, PAPER_LAMBDA = 64, 6, 1.5


def _blob_shape(rng):
    """four spheres: centres U[-0.35, 0.35]^3, radii U[0.2, 0.35]"""
    return rng.uniform(-0.35, 0.35, (4, 3)), rng.uniform(0.2, 0.35, 4)


def _blob_distance(C, R, P):
    # training labels: distance to the union of the spheres (exact outside)
    return (np.linalg.norm(P[:, None, :] - C[None], axis=2) - R[None]).min(1)


def paper_network(seed: int = 0, steps: int = 1500, batch: int = 4096, cache: bool = True):
    """(params float32 packed like pack_layers, width, n_mid, lambda, (linears,
    norms)) of the paper's network architecture trained on a seeded shape.

    Samples per step (drawn from the seed): half near the surface (points of
    the sphere union jittered by N(0, 0.02^2)), half uniform in [-1, 1]^3;
    labels are distances to the union; L1 loss, Adam (lr 1e-3), batch
    normalisation in training mode; the running statistics are then folded
    into the weights (bn.fold_batchnorm).  Trained once per (seed, steps) and
    cached in the temporary directory."""
    import os
    import tempfile

    from .bn import fold_batchnorm

    path = os.path.join(tempfile.gettempdir(), "gh_paper_network_%d_%d_%d.npz" % (seed, steps, batch))
    if cache and os.path.exists(path):
        z = np.load(path, allow_pickle=False)
        n = int(z["n"])
        linears = [(z["W%d" % i], z["b%d" % i]) for i in range(n)]
        norms = [(z["g%d" % i], z["be%d" % i], z["m%d" % i], z["v%d" % i]) if ("g%d" % i) in z else None
                 for i in range(n)]
    else:
        import torch

        rng = np.random.default_rng(seed)
        C, R = _blob_shape(rng)
        torch.manual_seed(seed)
        W = PAPER_WIDTH
        mods = []
        dims = [3] + [W] * (PAPER_NMID + 1)
        for i in range(PAPER_NMID + 1):
            mods += [torch.nn.Linear(dims[i], W), torch.nn.BatchNorm1d(W), torch.nn.ReLU()]
        mods.append(torch.nn.Linear(W, 1))
        net = torch.nn.Sequential(*mods).double()
        opt = torch.optim.Adam(net.parameters(), lr=1e-3)
        for _ in range(steps):
            k = rng.integers(0, 4, batch // 2)
            d = rng.standard_normal((batch // 2, 3))
            d /= np.linalg.norm(d, axis=1, keepdims=True)
            near = C[k] + R[k, None] * d + rng.normal(0.0, 0.02, (batch // 2, 3))
            P = np.concatenate([near, rng.uniform(-1.0, 1.0, (batch - batch // 2, 3))])
            y = _blob_distance(C, R, P)
            pred = net(torch.from_numpy(P))[:, 0]
            loss = (pred - torch.from_numpy(y)).abs().mean()
            opt.zero_grad()
            loss.backward()
            opt.step()
        net.eval()
        lins = [m for m in mods if isinstance(m, torch.nn.Linear)]
        bns = [m for m in mods if isinstance(m, torch.nn.BatchNorm1d)]
        linears = [(m.weight.detach().numpy().copy(), m.bias.detach().numpy().copy()) for m in lins]
        norms = [(b.weight.detach().numpy().copy(), b.bias.detach().numpy().copy(), b.running_mean.numpy().copy(),
                  b.running_var.numpy().copy()) for b in bns] + [None]
        if cache:
            arrs = {"n": np.array(len(linears))}
            for i, (Wl, bl) in enumerate(linears):
                arrs["W%d" % i], arrs["b%d" % i] = Wl, bl
            for i, bn in enumerate(norms):
                if bn is not None:
                    arrs["g%d" % i], arrs["be%d" % i], arrs["m%d" % i], arrs["v%d" % i] = bn
            tmp = path + ".%d.tmp" % os.getpid()
            np.savez(tmp, **arrs)
            os.replace(tmp + ".npz" if not tmp.endswith(".npz") else tmp, path)
    folded = fold_batchnorm(linears, norms)
    layers = [(Wl.astype(np.float32), bl.astype(np.float32)) for Wl, bl in folded]
    return pack_layers(layers), PAPER_WIDTH, PAPER_NMID, PAPER_LAMBDA, (linears, norms)


def mlp_param_count(width: int, nmid: int = MLP_NMID) -> int:
    return 3 * width + width + nmid * (width * width + width) + width + 1


def mlp_layers(seed: int, width: int = 256, nmid: int = MLP_NMID):
    """[(W_l, b_l)] float32, shapes (W,3),(W,W)*nmid,(1,W)."""
    rng = np.random.default_rng(seed)
    shapes = [(width, 3)] + [(width, width)] * nmid + [(1, width)]
    layers = []
    for out_d, in_d in shapes:
        W = rng.standard_normal((out_d, in_d))
        b = rng.normal(0.0, 0.01, out_d)
        sig = np.linalg.svd(W, compute_uv=False)[0]
        layers.append(((W / sig).astype(np.float32), b.astype(np.float32)))
    return layers


def pack_layers(layers) -> np.ndarray:
    """Flat float32 vector W0 b0 {W b}*nmid wout bout (row-major)."""
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers]).astype(np.float32)


def unpack_layers(vec, width: int, nmid: int = MLP_NMID):
    vec = np.asarray(vec)
    shapes = [(width, 3)] + [(width, width)] * nmid + [(1, width)]
    out, o = [], 0
    for od, id_ in shapes:
        W = vec[o : o + od * id_].reshape(od, id_)
        o += od * id_
        b = vec[o : o + od]
        o += od
        out.append((W, b))
    return out


def mlp_params(seed: int, width: int = 256, nmid: int = MLP_NMID) -> np.ndarray:
    return pack_layers(mlp_layers(seed, width, nmid))


BATCH_NS = (128, 256, 384, 512, 768, 1024)
BATCH_WIDTHS = (64, 128, 256)


def batch_items(n: int = 64):
    """(kind, seed, N, width) for seeds 0..n-1: even seeds CSG, odd seeds MLP;
    N and width drawn from default_rng(10000 + seed)."""
    items = []
    for s in range(n):
        rng = np.random.default_rng(10000 + s)
        N = int(rng.choice(BATCH_NS))
        W = int(rng.choice(BATCH_WIDTHS))
        items.append(("csg" if s % 2 == 0 else "mlp", s, N, W))
    return items


def uniform_points(seed: int, n: int, lo=-1.0, hi=1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (n, 3)).astype(np.float32)
