"""GPU-vs-oracle mesh comparison used by the GPU parity tests.

Tolerances (the FP32 path against the FP64 oracle):
* TIE: a cell with a corner |f64| < TIE may legitimately differ in case index
  (the FP32 evaluation error decides the sign there).  TIE = max(1e-6 h,
  DELTA32) with DELTA32 = 2e-6 a bound on |f32 - f64| for the inputs used
  (about 16 float32 roundings of values of magnitude <= 2).
* vertices: |v_gpu - v_oracle| <= 1e-4 h + h DELTA32 / |fA - fB|, the second
  term being the propagated evaluation error of t = fA/(fA - fB) on a badly
  conditioned (nearly tangent) edge; the share of vertices within the bare
  1e-4 h is checked separately.
Cells, case indices and triangle edge-key triples are compared exactly
outside the tie cells; triangles are compared as multisets (GPU order is not
deterministic) with each key triple rotated to start at its smallest key.
"""
import numpy as np

import meshutil
import oracle

DELTA32 = 2e-6


def cell_corner_points(cells, N, lo, h):
    c = np.asarray(cells, np.int64)
    k = c % N
    j = (c // N) % N
    i = c // (N * N)
    off = np.array([[b & 1, (b >> 1) & 1, (b >> 2) & 1] for b in range(8)], np.int64)
    ijk = np.stack([i, j, k], 1)[:, None, :] + off[None]
    return lo + ijk.astype(np.float64) * h


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


def compare(gpu, osdb, N, lo=-1.0, hi=1.0, ref=None, restrict_cells=None, delta32=DELTA32, min_bare=0.999):
    """gpu: gh.Mesh with keys and cells; ref: oracle Result with the oracle's
    sign-change cells (cells/cases) and triangles.  restrict_cells: optional
    predicate (np array of cell ids -> bool mask) limiting the comparison to
    a sampled region.  Returns a dict of statistics."""
    h = (hi - lo) / N
    tie = max(1e-6 * h, delta32)
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
    fc = osdb.eval(cell_corner_points(allc, N, lo, h).reshape(-1, 3)).reshape(-1, 8)
    tie_cells = allc[(np.abs(fc) < tie).any(1)]
    gset = np.setdiff1d(gc, tie_cells)
    oset = np.setdiff1d(oc, tie_cells)
    assert gset.size == oset.size and (gset == oset).all(), (
        "surface cells differ: %d only on GPU, %d only in oracle" % (np.setdiff1d(gset, oset).size,
                                                                     np.setdiff1d(oset, gset).size))
    gmap = dict(zip(gc.tolist(), gk.tolist()))
    omap = dict(zip(oc.tolist(), ok_.tolist()))
    bad = [c for c in gset.tolist() if gmap[c] != omap[c]]
    assert not bad, "case index differs in %d cells, e.g. %d: gpu %d oracle %d" % (len(bad), bad[0], gmap[bad[0]],
                                                                                  omap[bad[0]])
    # triangles, excluding those touching an edge of a tie cell
    tie_keys = np.unique(cell_edge_keys(tie_cells, N)) if tie_cells.size else np.zeros(0, np.int64)
    gtk = ~np.isin(gkeys, tie_keys).any(1)
    otk = ~np.isin(okeys, tie_keys).any(1)
    ct_g = meshutil.canonical_tris(gkeys[gtk])
    ct_o = meshutil.canonical_tris(okeys[otk])
    assert ct_g.shape == ct_o.shape, "triangle counts differ: gpu %d oracle %d" % (ct_g.shape[0], ct_o.shape[0])
    assert (ct_g == ct_o).all(), "triangle edge-key multisets differ"
    # vertices
    uk_g, p_g = meshutil.vertex_table(gkeys[gtk], gpos[gtk])
    uk_o, p_o = meshutil.vertex_table(okeys[otk], opos[otk])
    assert (uk_g == uk_o).all()
    N1 = N + 1
    ax = uk_o // N1**3
    r = uk_o % N1**3
    A = np.stack([r % N1, (r // N1) % N1, r // N1**2], 1).astype(np.float64)
    B = A.copy()
    B[np.arange(B.shape[0]), ax] += 1
    fA = osdb.eval(lo + A * h)
    fB = osdb.eval(lo + B * h)
    err = np.abs(p_g - p_o).max(1)
    tol = 1e-4 * h + h * delta32 / np.maximum(np.abs(fA - fB), 1e-300)
    worst = np.argmax(err - tol) if err.size else 0
    assert (err <= tol).all(), "vertex error %.3g > tol %.3g (h = %.3g)" % (err[worst], tol[worst], h)
    bare = float(np.mean(err <= 1e-4 * h)) if err.size else 1.0
    assert bare >= min_bare, "only %.5f of vertices within 1e-4 h" % bare
    return {"cells": int(gset.size), "tie_cells": int(tie_cells.size), "tris": int(ct_g.shape[0]),
            "verts": int(uk_g.size), "max_err_over_h": float(err.max() / h) if err.size else 0.0,
            "bare_frac": bare}
