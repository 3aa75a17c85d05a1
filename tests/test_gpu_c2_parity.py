"""The neural workload at full size -- the width-256 network of seed 1
(f = (|p| - 0.6 + 0.1 g(p)) / 1.1, Sec. 5.2) on the N = 1024 grid -- against
the FP64 oracle, in plain FP32 and in BF16 with FP32 refinement:

* every sign-change cell of 300 uniformly random columns and of the columns
  whose rays graze the surface's silhouette (found by the oracle's own
  hopper), checked cell by cell, case by case, triangle by triangle;
* one full z-slab through the equator against the oracle's enumeration of
  that slab (Sec. 2);
* the BF16 + refinement mesh equal to the FP32 mesh over the whole grid,
  triangle for triangle and vertex for vertex (bit-identical positions);
* the same network at N = 256 against the oracle on every column;
and the same for BF16 hopping refined with split-BF16 products ("bf16x6"),
whose corner values are compared as its own evaluator gives them.
"""
import numpy as np
import pytest

import meshutil
import oracle
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth  # noqa: E402

N = 1024
W = 256


@pytest.fixture(scope="module")
def c2():
    p = synth.mlp_params(1, W)
    sdb = gh.MlpSdb(p, W)
    o = oracle.mlp(W, synth.MLP_NMID, p.astype(np.float64))
    eps = sdb.calibrate(N)
    meshes = {"fp32": gh.polygonize(sdb, N, keys=True, cells=True),
              "bf16": gh.polygonize(sdb, N, precision="bf16", eps=eps, keys=True, cells=True),
              "bf16x6": gh.polygonize(sdb, N, precision="bf16x6", eps=eps, keys=True, cells=True)}
    return sdb, o, eps, meshes


@pytest.fixture(scope="module")
def column_ref(c2):
    _, o, _, _ = c2
    rng = np.random.default_rng(17)
    uniform = rng.choice(N * N, 300, replace=False)
    sil = parity.silhouette_columns(o, N)
    cols = np.unique(np.concatenate([uniform, sil]))
    _, ref = oracle.polygonize(o, N, cols=cols)
    return cols, sil, ref


@pytest.fixture(scope="module")
def slab_ref(c2):
    _, o, _, _ = c2
    k0 = N // 2  # z in [0, h]: the equator of the perturbed sphere
    return k0, parity.slab_reference(o, N, k0)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "bf16x6"])
def test_c2_uniform_and_silhouette_columns(c2, column_ref, precision):
    sdb, o, _, meshes = c2
    cols, sil, ref = column_ref
    assert sil.size >= 200
    m = meshes[precision]
    # grazing rays cross the surface on nearly tangent z-edges, where the FP32
    # evaluation error divided by |fA - fB| exceeds the bare 1e-4 h for ~5 %
    # of the vertices (every vertex meets the propagated bound)
    st = parity.compare(m, o, N, ref=ref, restrict_cells=lambda c: np.isin(c // N, cols), gsdb=sdb, min_bare=0.9,
                        gprec=precision)
    print("C2 N=1024 %s columns: %s" % (precision, st))
    assert st["cells"] > 8000
    # the grazing columns alone hold most of those cells: they are compared too
    sil_cells = np.isin(ref.cells[(ref.cases > 0) & (ref.cases < 255)] // N, sil).sum()
    assert sil_cells > 5000
    assert st["sign_flip_outside_band"] <= 0.002 * st["cells"] + 8


@pytest.mark.parametrize("precision", ["fp32", "bf16", "bf16x6"])
def test_c2_equatorial_slab_against_enumeration(c2, slab_ref, precision):
    sdb, o, _, meshes = c2
    k0, ref = slab_ref
    st = parity.compare(meshes[precision], o, N, ref=ref, restrict_cells=lambda c: (c % N) == k0, gsdb=sdb,
                        min_bare=0.9, gprec=precision)
    print("C2 N=1024 %s slab k=%d: %s" % (precision, k0, st))
    assert st["cells"] > 2000
    assert st["sign_flip_outside_band"] <= 0.002 * st["cells"] + 8


def test_c2_bf16_mesh_equals_fp32_mesh(c2):
    """Refinement re-evaluates in FP32 every corner whose sign or value the
    mesh uses, so the two meshes are the same: same triangles (as edge-key
    triples, orientation kept) and bit-identical vertex positions."""
    _, _, _, meshes = c2
    a, b = meshes["fp32"], meshes["bf16"]
    assert a.n_tris == b.n_tris > 3_000_000
    ka, kb = a.tri_keys.cpu().numpy(), b.tri_keys.cpu().numpy()
    assert np.array_equal(meshutil.canonical_tris(ka), meshutil.canonical_tris(kb))
    ua, pa = meshutil.vertex_table(ka, a.tri_xyz.cpu().numpy())
    ub, pb = meshutil.vertex_table(kb, b.tri_xyz.cpu().numpy())
    assert np.array_equal(ua, ub)
    assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
    assert np.array_equal(np.sort(a.cell_ids.cpu().numpy()), np.sort(b.cell_ids.cpu().numpy()))
    # hops shrink by eps but stay O(N^2 log N): within a few percent of FP32
    assert a.stats["hop_evals"] < b.stats["hop_evals"] < 1.1 * a.stats["hop_evals"]


@pytest.mark.parametrize("precision", ["fp32", "bf16", "bf16x6"])
def test_width256_every_column_n256(precision):
    """The same network at N = 256: every column against the oracle's hopper
    followed by Marching Cubes (whose surface-cell set equals enumeration's,
    a property the oracle's own tests pin)."""
    n = 256
    p = synth.mlp_params(1, W)
    sdb = gh.MlpSdb(p, W)
    o = oracle.mlp(W, synth.MLP_NMID, p.astype(np.float64))
    eps = sdb.calibrate(n) if precision != "fp32" else None
    m = gh.polygonize(sdb, n, precision=precision, eps=eps, keys=True, cells=True)
    ref = _full_ref(o, n)
    st = parity.compare(m, o, n, ref=ref, gsdb=sdb, min_bare=0.99, gprec=precision)
    print("width 256 N=256 %s: %s" % (precision, st))
    assert st["cells"] > 100000
    assert st["sign_flip_outside_band"] <= 0.002 * st["cells"] + 8


_FULL = {}


def _full_ref(o, n):
    if n not in _FULL:
        _FULL[n] = oracle.polygonize(o, n)[1]
    return _FULL[n]
