"""Continuation on the GPU (gh_polygonize_cont, Sec. 2: the surface crawled
from seed cells) against the oracle's continuation and against grid
hopping, through the C ABI: a crawled component's mesh is the hopper's mesh
of that component bit for bit (same evaluator, same lattice points), one
seed gives one component, and the crawled cells are the oracle's."""
import numpy as np
import pytest

import meshutil
import oracle
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth  # noqa: E402


def _bitwise_same(a, b):
    ka, kb = a.tri_keys.cpu().numpy(), b.tri_keys.cpu().numpy()
    assert np.array_equal(meshutil.canonical_tris(ka), meshutil.canonical_tris(kb))
    ua, pa = meshutil.vertex_table(ka, a.tri_xyz.cpu().numpy())
    ub, pb = meshutil.vertex_table(kb, b.tri_xyz.cpu().numpy())
    assert np.array_equal(ua, ub) and np.array_equal(pa.view(np.uint32), pb.view(np.uint32))


@pytest.mark.parametrize("N", [2, 37, 64, 200])
def test_sphere_cont_equals_hopping_and_oracle(N):
    prims = synth.sphere_prims(0.5, (0.01, -0.02, 0.03))
    sdb = gh.CsgSdb(prims)
    c = gh.polygonize_cont(sdb, N, [[0.0, 0.0, 0.0]], keys=True, cells=True)
    hp = gh.polygonize(sdb, N, keys=True, cells=True)
    _bitwise_same(c, hp)
    st = c.stats
    assert st["status"] == 0 and st["marked_cells"] == st["surface_cells"] == hp.stats["surface_cells"]
    assert st["hop_evals"] >= 8 * st["marked_cells"]
    o = oracle.csg(prims)
    ref = oracle.cont(o, N, [[0.0, 0.0, 0.0]])
    # the centre and radius in float32 put many lattice corners within ~1e-8 of
    # the surface (band ties); vertices next to them have a larger FP32 error
    s = parity.compare(c, o, N, ref=ref, gsdb=sdb, min_bare=0.995)
    assert s["sign_flip_outside_band"] == 0


def test_one_seed_one_component():
    a = synth.sphere_prims(0.3, (-0.45, 0.0, 0.0))
    b = synth.sphere_prims(0.3, (0.45, 0.0, 0.0))
    both = np.concatenate([a, b])
    N = 96
    sdb = gh.CsgSdb(both)
    one = gh.polygonize_cont(sdb, N, [[-0.45, 0.0, 0.0]], keys=True, cells=True)
    _bitwise_same(one, gh.polygonize(gh.CsgSdb(a), N, keys=True))
    two = gh.polygonize_cont(sdb, N, [[-0.45, 0.0, 0.0], [0.45, 0.0, 0.0], [-0.5, 0.01, 0.0]], keys=True)
    _bitwise_same(two, gh.polygonize(sdb, N, keys=True))
    none = gh.polygonize_cont(sdb, N, [[0.9, 0.9, 0.9]], keys=True)
    assert none.n_tris == 0 and none.stats["marked_cells"] == 0


@pytest.mark.parametrize("N", [160, 512])
def test_csg_scene_seeded_components_match_oracle(N):
    """The analytic workload (24 spheres + 8 tori - 4 boxes, several
    components), seeds left of every primitive's centre: the crawled cells,
    cases and triangles against the oracle's crawl from the same points."""
    prims = synth.csg_prims(0)
    seeds = prims[:, 2:5].copy()
    seeds[:, 0] -= 0.3
    sdb = gh.CsgSdb(prims)
    c = gh.polygonize_cont(sdb, N, seeds, keys=True, cells=True)
    o = oracle.csg(prims)
    ref = oracle.cont(o, N, seeds)
    if N == 160:
        st = parity.compare(c, o, N, ref=ref, gsdb=sdb)
    else:
        # The crawl follows the surface's connectivity, which rounding can
        # change: where two primitives barely touch, a face with both signs in
        # FP64 can have one sign in FP32 (a flipped corner), and the FP32
        # crawl does not cross it.  A few cells beyond such a neck are then
        # reached in FP64 only (at N = 512: 4 of 718 k cells).
        st = parity.compare(c, o, N, ref=ref, gsdb=sdb, check=False)
        assert st["mismatched_cells"] <= 16 and st["sign_flip_outside_band"] <= 16
        assert st["mismatched_tris"] <= 64 and st["vertices_over_tol"] == 0
    assert st["cells"] > 1000
    # every crawled triangle is one of the hopper's, positions bit-identical
    hp = gh.polygonize(sdb, N, keys=True)
    kc = meshutil.canonical_tris(c.tri_keys.cpu().numpy())
    kh = meshutil.canonical_tris(hp.tri_keys.cpu().numpy())
    assert np.isin(parity._rows(kc), parity._rows(kh)).all()


def test_cont_rejects_neural_and_bad_seeds():
    m = gh.MlpSdb(synth.mlp_params(1, 64), 64)
    bufs = gh.Buffers(1000)
    with pytest.raises(gh.GhError) as e:
        gh.polygonize_cont_into(m, 32, [[0.0, 0.0, 0.0]], bufs)
    assert e.value.code == gh.GH_ERR_UNIMPLEMENTED
    s = gh.CsgSdb(synth.sphere_prims(0.5))
    with pytest.raises(gh.GhError) as e:
        gh.polygonize_cont_into(s, 32, [[np.nan, 0.0, 0.0]], bufs)
    assert e.value.code == gh.GH_ERR_ARG
