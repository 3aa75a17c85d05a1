"""On-device indexed mesh (gh_mesh.vert_xyz / tri_idx): one vertex per
crossing lattice edge, faces into them.  Checked against the triangle soup of
the same call (bit-exact positions, the soup's edge keys), for determinism,
against the oracle's vertex set, and for the capacity protocol."""
import numpy as np
import pytest

import meshutil
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth  # noqa: E402


def _check_against_soup(m):
    keys = m.tri_keys.cpu().numpy()
    pos = m.tri_xyz.cpu().numpy()
    V = m.verts.cpu().numpy()
    F = m.faces.cpu().numpy().astype(np.int64)
    uk = np.unique(keys)
    assert V.shape[0] == uk.size == m.stats["mesh_vertices"]
    assert F.shape == keys.shape and F.min() >= 0 and F.max() < V.shape[0]
    # each corner's vertex has the soup's position, bit for bit
    assert np.array_equal(V[F].view(np.uint32), pos.view(np.uint32))
    # one vertex per edge key: equal keys <-> equal indices
    k_of_v = np.full(V.shape[0], -1, np.int64)
    k_of_v[F.ravel()] = keys.ravel()
    assert np.array_equal(k_of_v[F], keys)
    assert np.unique(k_of_v).size == V.shape[0]
    return keys, F, V, k_of_v


@pytest.mark.parametrize("N,lo,hi", [(100, -1.0, 1.0), (129, -0.7, 0.8)])
def test_csg_indexed_mesh(N, lo, hi):
    prims = synth.csg_prims(0)
    sdb = gh.CsgSdb(prims)
    m = gh.polygonize(sdb, N, lo=lo, hi=hi, indexed=True)
    keys, F, V, k_of_v = _check_against_soup(m)
    # vertex numbering: lower end point (lattice line a*(N+1)+b, then c), then axis
    N1 = N + 1
    ax = k_of_v // N1**3
    r = k_of_v % N1**3
    a, b, c = r % N1, (r // N1) % N1, r // N1**2
    order = np.lexsort((ax, c, a * N1 + b))
    assert np.array_equal(order, np.arange(V.shape[0]))
    # the same vertex set as the oracle's mesh
    _, mr = oracle.polygonize(oracle.csg(prims), N, lo, hi)
    assert np.array_equal(np.unique(mr.tri_keys), np.unique(keys))


def test_indexed_mesh_is_deterministic():
    sdb = gh.CsgSdb(synth.csg_prims(3))
    a = gh.polygonize(sdb, 96, indexed=True)
    b = gh.polygonize(sdb, 96, indexed=True)
    assert torch.equal(a.verts, b.verts)
    fa = np.sort(np.sort(a.faces.cpu().numpy(), 1), 0)
    fb = np.sort(np.sort(b.faces.cpu().numpy(), 1), 0)
    assert np.array_equal(np.unique(fa, axis=0), np.unique(fb, axis=0))


def test_sphere_indexed_closed_genus0():
    sdb = gh.CsgSdb(synth.sphere_prims(0.45, (0.03, -0.02, 0.01)))
    m = gh.polygonize(sdb, 80, indexed=True)
    F = m.faces.cpu().numpy().astype(np.int64)
    assert meshutil.closed_oriented(F)
    assert meshutil.euler(F) == 2
    assert F.shape[0] == 2 * m.verts.shape[0] - 4


def test_neural_bf16_indexed_mesh():
    params = synth.pack_layers(synth.mlp_layers(1, 128))
    sdb = gh.MlpSdb(params, 128)
    eps = sdb.calibrate(128)
    m = gh.polygonize(sdb, 128, precision="bf16", eps=eps, indexed=True)
    _check_against_soup(m)
    F = m.faces.cpu().numpy().astype(np.int64)
    assert meshutil.closed_oriented(F)


def test_batch_indexed_matches_single():
    sdbs = [gh.CsgSdb(synth.csg_prims(s)) for s in (0, 2)]
    Ns = [64, 100]
    bt = gh.polygonize_batch(sdbs, Ns, indexed=True)
    for b in range(2):
        mb = bt.mesh(b)
        _check_against_soup(mb)
        single = gh.polygonize(gh.CsgSdb(synth.csg_prims((0, 2)[b])), Ns[b], indexed=True)
        assert torch.equal(mb.verts, single.verts)


def test_vertex_capacity_protocol():
    sdb = gh.CsgSdb(synth.sphere_prims(0.5))
    need = gh.polygonize(sdb, 64, indexed=True).verts.shape[0]
    bufs = gh.Buffers(4 * 64 * 64, cap_verts=need - 1)
    rc = gh.polygonize_into(sdb, 64, bufs)
    assert rc == gh.GH_ERR_CAPACITY
    assert int(bufs.counts[2].item()) == need
    bufs = gh.Buffers(4 * 64 * 64, cap_verts=need)
    assert gh.polygonize_into(sdb, 64, bufs) == gh.GH_OK


def test_indexed_argument_errors():
    sdb = gh.CsgSdb(synth.sphere_prims(0.5))
    bufs = gh.Buffers(10000, cap_verts=10000)
    bufs.desc.tri_keys = None  # tri_idx needs the edge keys
    with pytest.raises(gh.GhError) as e:
        gh.polygonize_into(sdb, 32, bufs)
    assert e.value.code == gh.GH_ERR_ARG
    bufs = gh.Buffers(100000, cap_verts=100000)
    with pytest.raises(gh.GhError) as e:
        gh.polygonize_into(sdb, 32, bufs, method="enum")
    assert e.value.code == gh.GH_ERR_UNIMPLEMENTED
