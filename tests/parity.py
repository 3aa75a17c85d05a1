"""GPU-vs-oracle mesh comparison used by the GPU parity tests.

The FP32 path against the FP64 oracle:
* Excluded cells.  A cell is left out of the exact comparison only when one
  of its corners (a) is a zero of f up to FP64 rounding (|f64| < 1e-13, the
  tie rule's own case), or (b) has a GPU FP32 value whose sign differs from
  the FP64 sign.  (b) is measured, not assumed: the GPU's own FP32 evaluator
  (gh_eval, the evaluator the hopper and the vertex pass use, bit for bit) is
  run at the corner positions the GPU uses -- the float32 lattice points
  fma(a, h32, lo32) -- and compared with the FP64 value at the exact lattice
  point.  This is stricter than the tie band the workloads state (corners
  with |f| < 1e-6 h): band cells whose FP32 signs agree are compared too;
  their number is returned as "tie_cells", with "exact_zero_cells" and
  "sign_flip_cells"; flips inside the band are the stated ties, flips outside
  it ("sign_flip_outside_band") are bounded (max_excluded).
* delta32 = 2 max |f32 - f64| over the corners of every compared cell
  (measured per call, returned).
* Vertices: |v_gpu - v_oracle| <= 1e-4 h + h delta32 / |fA - fB|, the second
  term being the propagated evaluation error of t = fA / (fA - fB) on a nearly
  tangent edge; the share within the bare 1e-4 h is returned and bounded
  (min_bare), the largest error is returned as max_err_over_h.
Outside the excluded cells the surface-cell set, every case index and the
triangle edge-key multiset must be identical; triangles are compared as
multisets (GPU order is not deterministic) with each key triple rotated to
start at its smallest key.
"""
import numpy as np

import meshutil

TIE_H = 1e-6  # the tie band, in units of h
# Point-wise evaluation tests (the same float32 input point on both sides):
# a bound on |f32 - f64| for the scenes and networks of the tests, about 16
# float32 roundings of values of magnitude <= 2.
EVAL32 = 2e-6


def grid32(N, lo, hi):
    """The float32 grid constants of the library (gh_polygonize's check):
    lo32, h32 = (hi32 - lo32) / N in single precision."""
    lo32 = np.float32(lo)
    ext = np.float32(np.float32(hi) - lo32)
    return lo32, np.float32(ext / np.float32(N))


def lattice32(ijk, N, lo, hi):
    """Float32 positions fma(a, h32, lo32) of lattice coordinates (exact in
    float64 before the one rounding to float32, like the device's fmaf)."""
    lo32, h32 = grid32(N, lo, hi)
    v = np.asarray(ijk, np.float64) * np.float64(h32) + np.float64(lo32)
    return v.astype(np.float32)


def corner_ijk(cells, N):
    c = np.asarray(cells, np.int64)
    k = c % N
    j = (c // N) % N
    i = c // (N * N)
    off = np.array([[b & 1, (b >> 1) & 1, (b >> 2) & 1] for b in range(8)], np.int64)
    return np.stack([i, j, k], 1)[:, None, :] + off[None]


def cell_corner_points(cells, N, lo, h):
    return lo + corner_ijk(cells, N).astype(np.float64) * h


def cell_edge_keys(cells, N):
    """the 12 edge keys of each cell, [n, 12]"""
    c = np.asarray(cells, np.int64)
    k = c % N
    j = (c // N) % N
    i = c // (N * N)
    N1 = N + 1
    out = []
    for e in range(12):
        ax, u, v = e // 4, e & 1, (e >> 1) & 1
        o = [0, 0, 0]
        others = [a for a in range(3) if a != ax]
        o[others[0]], o[others[1]] = u, v
        a, b, cc = i + o[0], j + o[1], k + o[2]
        out.append(ax * N1**3 + a + N1 * (b + N1 * cc))
    return np.stack(out, 1)


def tri_cells(keys, N):
    """Cell of each triangle from its three edge keys: the one cell whose
    edges contain all three (unique: no table triangle lies in one face)."""
    keys = np.asarray(keys, np.int64)
    N1 = N + 1
    ax = keys // N1**3
    r = keys % N1**3
    a, b, c = r % N1, (r // N1) % N1, r // N1**2
    out = np.full(keys.shape[0], -1, np.int64)
    sets = []
    for v in range(3):
        cells = []
        for du in (0, 1):
            for dv in (0, 1):
                ii, jj, kk = a[:, v].copy(), b[:, v].copy(), c[:, v].copy()
                axv = ax[:, v]
                ii = ii - np.where(axv == 0, 0, du)
                jj = jj - np.where(axv == 1, 0, np.where(axv == 0, du, dv))
                kk = kk - np.where(axv == 2, 0, dv)
                ok = (ii >= 0) & (jj >= 0) & (kk >= 0) & (ii < N) & (jj < N) & (kk < N)
                cells.append(np.where(ok, (ii * N + jj) * N + kk, -1 - v))
        sets.append(np.stack(cells, 1))
    for q in range(4):
        cq = sets[0][:, q]
        hit = (sets[1] == cq[:, None]).any(1) & (sets[2] == cq[:, None]).any(1) & (cq >= 0)
        out = np.where(hit & (out < 0), cq, out)
    return out


def gpu_fp32(gsdb, precision="fp32"):
    """Callable: float32 points [n,3] -> the GPU's values (float64) from the
    evaluator that produced the mesh's corner values: FP32 (plain and BF16 +
    FP32 refinement) or the split-BF16 engine ("bf16x6" refinement)."""
    import torch

    from paper_2111_05778_gb300 import gh

    def f(p32):
        p = torch.from_numpy(np.ascontiguousarray(p32, np.float32).reshape(-1, 3)).cuda()
        return gh.eval_points(gsdb, p, precision).cpu().numpy().astype(np.float64)

    return f


def _rows(a):
    a = np.ascontiguousarray(a, np.int64)
    return a.view(np.dtype((np.void, a.dtype.itemsize * a.shape[1]))).ravel()


def compare(gpu, osdb, N, lo=-1.0, hi=1.0, ref=None, restrict_cells=None, gsdb=None, min_bare=0.999,
            max_excluded=None, check=True, f32=None, gprec="fp32"):
    """gpu: gh.Mesh with keys and cells; osdb: the oracle SDB; ref: oracle
    Result with the oracle's sign-change cells (cells/cases) and triangles;
    gsdb: the GPU SDB (its FP32 evaluator decides (b) above and delta32;
    gprec="bf16x6" takes its split-BF16 evaluator instead, the one that
    refines the corners of that precision's meshes).
    restrict_cells: optional predicate (cell ids -> bool mask) limiting the
    comparison to a sampled region.  max_excluded: bound on the sign-flip
    cells outside the band (default max(32, 0.2 % of the compared cells)).  Returns a dict of
    statistics; check=True asserts every bound, check=False only reports
    (mismatch counts included).  f32: optional callable standing in for the
    GPU's FP32 evaluator (float32 points -> values), for CPU self-tests."""
    assert gsdb is not None or f32 is not None, "compare() needs the GPU SDB for its FP32 corner values"
    f32_eval = f32 if f32 is not None else gpu_fp32(gsdb, "bf16x6" if gprec == "bf16x6" else "fp32")
    h = (hi - lo) / N
    tie = TIE_H * h
    gc = gpu.cell_ids.cpu().numpy().astype(np.int64)
    gk = gpu.cell_cases.cpu().numpy().astype(np.int32)
    gkeys = gpu.tri_keys.cpu().numpy().astype(np.int64)
    gpos = gpu.tri_xyz.cpu().numpy().astype(np.float64)
    oc = ref.cells
    ok_ = ref.cases
    sel = (ok_ > 0) & (ok_ < 255)
    oc, ok_ = oc[sel], ok_[sel]
    okeys, opos = ref.tri_keys, ref.tri_pos
    if restrict_cells is not None:
        gm = restrict_cells(gc)
        om = restrict_cells(oc)
        # triangles follow their cells
        gsel = restrict_cells(tri_cells(gkeys, N))
        osel = restrict_cells(ref.tri_cell)
        gc, gk, oc, ok_ = gc[gm], gk[gm], oc[om], ok_[om]
        gkeys, gpos, okeys, opos = gkeys[gsel], gpos[gsel], okeys[osel], opos[osel]
    allc = np.union1d(gc, oc)
    ijk = corner_ijk(allc, N).reshape(-1, 3)
    f64 = osdb.eval_many(lo + ijk.astype(np.float64) * h).reshape(-1, 8)
    f32 = f32_eval(lattice32(ijk, N, lo, hi)).reshape(-1, 8)
    delta32 = 2.0 * float(np.abs(f32 - f64).max()) if f64.size else 0.0
    in_band = (np.abs(f64) < tie).any(1)
    # corners where f is zero up to FP64 rounding: the tie rule's own cases
    # (f = 0 counts as outside), where even the FP64 sign is not meaningful;
    # a lattice aligned with the scene can produce them by the hundred
    exact = (np.abs(f64) < 1e-13).any(1)
    flipped = ((f32 < 0) != (f64 < 0)).any(1) & ~exact
    excl = allc[exact | flipped]
    n_bounded = int((flipped & ~in_band).sum())  # flips inside the band are the stated ties
    limit = max_excluded if max_excluded is not None else max(32, int(0.002 * allc.size))
    gset = np.setdiff1d(gc, excl)
    oset = np.setdiff1d(oc, excl)
    common = np.intersect1d(gset, oset)
    gmap = dict(zip(gc.tolist(), gk.tolist()))
    omap = dict(zip(oc.tolist(), ok_.tolist()))
    bad_case = [c for c in common.tolist() if gmap[c] != omap[c]]
    # triangles, excluding those touching an edge of an excluded cell
    ex_keys = np.unique(cell_edge_keys(excl, N)) if excl.size else np.zeros(0, np.int64)
    gtk = ~np.isin(gkeys, ex_keys).any(1)
    otk = ~np.isin(okeys, ex_keys).any(1)
    ct_g = meshutil.canonical_tris(gkeys[gtk])
    ct_o = meshutil.canonical_tris(okeys[otk])
    rg, ro = _rows(ct_g), _rows(ct_o)
    tri_mismatch = int(np.setdiff1d(rg, ro).size + np.setdiff1d(ro, rg).size)
    # vertices on the edges both sides have
    uk_g, p_g = meshutil.vertex_table(gkeys[gtk], gpos[gtk])
    uk_o, p_o = meshutil.vertex_table(okeys[otk], opos[otk])
    kk, ig, io = np.intersect1d(uk_g, uk_o, return_indices=True)
    N1 = N + 1
    ax = kk // N1**3
    r = kk % N1**3
    A = np.stack([r % N1, (r // N1) % N1, r // N1**2], 1).astype(np.float64)
    B = A.copy()
    B[np.arange(B.shape[0]), ax] += 1
    fA = osdb.eval_many(lo + A * h)
    fB = osdb.eval_many(lo + B * h)
    err = np.abs(p_g[ig] - p_o[io]).max(1) if kk.size else np.zeros(0)
    tol = 1e-4 * h + h * delta32 / np.maximum(np.abs(fA - fB), 1e-300)
    bare = float(np.mean(err <= 1e-4 * h)) if err.size else 1.0
    st = {"cells": int(gset.size), "tie_cells": int(in_band.sum()), "exact_zero_cells": int(exact.sum()),
          "sign_flip_cells": int(flipped.sum()), "sign_flip_outside_band": n_bounded,
          "mismatched_cells": int(np.setdiff1d(gset, oset).size + np.setdiff1d(oset, gset).size + len(bad_case)),
          "mismatched_tris": tri_mismatch, "delta32": delta32, "tris": int(ct_g.shape[0]), "verts": int(kk.size),
          "vertices_over_tol": int((err > tol).sum()),
          "max_err_over_h": float(err.max() / h) if err.size else 0.0, "bare_frac": bare}
    if check:
        try:
            assert n_bounded <= limit, "%d cells with an FP32 sign flip outside the 1e-6 h band > %d" % (
                n_bounded, limit)
            assert gset.size == oset.size and (gset == oset).all(), (
                "surface cells differ: %d only on GPU, %d only in oracle" % (np.setdiff1d(gset, oset).size,
                                                                             np.setdiff1d(oset, gset).size))
            assert not bad_case, "case index differs in %d cells, e.g. %d: gpu %d oracle %d" % (
                len(bad_case), bad_case[0], gmap[bad_case[0]], omap[bad_case[0]])
            assert ct_g.shape == ct_o.shape, "triangle counts differ: gpu %d oracle %d" % (ct_g.shape[0],
                                                                                           ct_o.shape[0])
            assert tri_mismatch == 0, "triangle edge-key multisets differ"
            assert uk_g.size == uk_o.size == kk.size
            worst = np.argmax(err - tol) if err.size else 0
            assert (err <= tol).all(), "vertex error %.3g > tol %.3g (h = %.3g, delta32 = %.3g)" % (
                err[worst], tol[worst], h, delta32)
            assert bare >= min_bare, "only %.5f of vertices within 1e-4 h" % bare
        except AssertionError as e:
            raise AssertionError("%s | stats: %r" % (e, st)) from None
    return st


def silhouette_columns(osdb, N, lo=-1.0, hi=1.0, n_angles=64, r0=0.45, r1=0.75, band=(-3.0, 2.0)):
    """Columns whose ray passes within a few cells of the surface's
    silhouette as seen along z, found with the oracle alone: for each of
    n_angles directions in the xy-plane, the oracle's hopper runs on the
    columns at radii r0..r1 (step 2h) and the outermost one with a marked
    cell gives the silhouette radius r_s; the columns nearest to the radii
    r_s + band (step h/2) along that direction are returned.  Grazing rays
    are where a hop could skip a cell."""
    import oracle

    h = (hi - lo) / N

    def col_at(r, phi):
        x, y = r * np.cos(phi), r * np.sin(phi)
        i = np.clip(np.floor((x - lo) / h).astype(np.int64), 0, N - 1)
        j = np.clip(np.floor((y - lo) / h).astype(np.int64), 0, N - 1)
        return i * N + j

    phis = 2 * np.pi * (np.arange(n_angles) + 0.5) / n_angles
    rs = np.arange(r0, r1, 2 * h)
    coarse = np.stack([col_at(rs, p) for p in phis])  # [angles, radii]
    hr = oracle.hop(osdb, N, lo, hi, cols=np.unique(coarse))
    marked_cols = np.unique(hr.marks // N)
    out = []
    for a, p in enumerate(phis):
        hit = np.nonzero(np.isin(coarse[a], marked_cols))[0]
        if hit.size == 0:
            continue
        rsil = rs[hit.max()]
        out.append(col_at(np.arange(rsil + band[0] * h, rsil + band[1] * h + 1e-12, 0.5 * h), p))
    return np.unique(np.concatenate(out)) if out else np.zeros(0, np.int64)


def slab_reference(osdb, N, k0, lo=-1.0, hi=1.0):
    """Enumeration (Sec. 2) restricted to the z-slab of cells k = k0: f at
    the (N+1)^2 x 2 lattice points of the slab (FP64, oracle.eval_many), the
    case of every one of its N^2 cells, and the oracle's Marching Cubes on
    the sign-change cells.  Returns the oracle Result of those cells."""
    import oracle

    h = (hi - lo) / N
    N1 = N + 1
    a, b = np.meshgrid(np.arange(N1), np.arange(N1), indexing="ij")
    vals = []
    for c in (k0, k0 + 1):
        P = np.stack([lo + a.ravel() * h, lo + b.ravel() * h, np.full(a.size, lo + c * h)], 1)
        vals.append(osdb.eval_many(P).reshape(N1, N1))
    neg = [v < 0 for v in vals]
    cnt = np.zeros((N, N), np.int32)
    for q in (0, 1):
        for di in (0, 1):
            for dj in (0, 1):
                cnt += neg[q][di:di + N, dj:dj + N]
    i, j = np.nonzero((cnt > 0) & (cnt < 8))
    cells = (i.astype(np.int64) * N + j) * N + k0
    return oracle.mc(osdb, N, cells, lo, hi)
