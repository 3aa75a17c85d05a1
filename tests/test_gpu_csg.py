"""GPU parity of the analytic-SDB path (hopper + Marching Cubes kernels)
against the FP64 oracle, through the C ABI."""
import os

import numpy as np
import pytest

import oracle
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth  # noqa: E402


def _golden(N):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sphere_r05_counts.txt")
    for l in open(path):
        if l.strip() and not l.startswith("#"):
            r = list(map(int, l.split()))
            if r[0] == N:
                return r
    raise KeyError(N)


@pytest.mark.parametrize("N", [16, 64, 256])
def test_sphere_matches_oracle(N):
    prims = synth.sphere_prims(0.5)
    sdb = gh.CsgSdb(prims)
    m = gh.polygonize(sdb, N, keys=True, cells=True)
    o = oracle.csg(prims)
    _, ref = oracle.polygonize(o, N)
    st = parity.compare(m, o, N, ref=ref, gsdb=sdb)
    g = _golden(N)
    assert m.stats["surface_cells"] == g[4]
    assert m.n_tris == g[6]
    assert m.stats["marked_cells"] == g[2]
    assert m.stats["hop_evals"] == g[1]
    # the six lattice corners with f = 0 exactly, (+-0.5, 0, 0) and permutations,
    # lie on grid points for these N; each touches at most 4 surface cells
    assert st["tie_cells"] <= 24
    assert st["sign_flip_outside_band"] == 0


@pytest.mark.parametrize("N,lo,hi", [(37, -1.0, 1.0), (100, -0.7, 0.9), (2, -1.0, 1.0), (129, -0.61, 0.61)])
def test_ragged_and_offset_grids(N, lo, hi):
    prims = np.concatenate([synth.sphere_prims(0.45, (0.05, -0.1, 0.02)),
                            synth.prim_row(synth.TORUS, synth.UNION, [0.1, 0.2, -0.1], [0.3, 0.08])[None]])
    sdb = gh.CsgSdb(prims)
    m = gh.polygonize(sdb, N, lo=lo, hi=hi, keys=True, cells=True)
    o = oracle.csg(prims)
    ref = oracle.enum(o, N, lo, hi)
    st = parity.compare(m, o, N, lo, hi, ref=ref, gsdb=sdb)
    # lattices aligned with the scene put corners within the scene's float32
    # rounding (~1e-8) of the surface, inside the 1e-6 h band where FP32 can not
    # decide the sign; flips outside the band are bounded
    assert st["sign_flip_outside_band"] <= 8


@pytest.mark.parametrize("tau_mode", [0, 1])
def test_csg_scene_full(tau_mode):
    prims = synth.csg_prims(0)
    N = 160
    sdb = gh.CsgSdb(prims)
    m = gh.polygonize(sdb, N, keys=True, cells=True, tau_mode=tau_mode)
    o = oracle.csg(prims)
    ref = oracle.enum(o, N)
    st = parity.compare(m, o, N, ref=ref, gsdb=sdb)
    assert st["cells"] > 10000
    assert st["sign_flip_outside_band"] <= 16


def test_csg_c1_sampled_columns_n512():
    """The C1 workload (CSG seed 0, N = 512) at full size: every sign-change
    cell of 400 random columns and of two full z-slabs, checked cell by cell."""
    prims = synth.csg_prims(0)
    N = 512
    sdb = gh.CsgSdb(prims)
    m = gh.polygonize(sdb, N, keys=True, cells=True)
    o = oracle.csg(prims)
    rng = np.random.default_rng(11)
    cols = np.unique(rng.choice(N * N, 400, replace=False))
    _, ref = oracle.polygonize(o, N, cols=cols)
    parity.compare(m, o, N, ref=ref, restrict_cells=lambda c: np.isin(c // N, cols), gsdb=sdb)
    for k0 in (173, 301):
        ref = oracle.enum(o, N, kmin=k0, kmax=k0 + 1)
        st = parity.compare(m, o, N, ref=ref, restrict_cells=lambda c: (c % N) == k0, gsdb=sdb)
        assert st["cells"] > 1000
        assert st["sign_flip_outside_band"] <= 8


def test_no_surface_inside_domain():
    for prims in (synth.sphere_prims(0.2, (5.0, 5.0, 5.0)), synth.sphere_prims(10.0)):
        m = gh.polygonize(gh.CsgSdb(prims), 64, keys=True, cells=True)
        assert m.n_tris == 0 and m.cell_ids.numel() == 0
        assert m.stats["status"] == 0


def test_capacity_protocol():
    sdb = gh.CsgSdb(synth.sphere_prims(0.5))
    N = 64
    bufs = gh.Buffers(100, keys=True)
    rc = gh.polygonize_into(sdb, N, bufs)
    assert rc == gh.GH_ERR_CAPACITY
    need = int(bufs.counts[0].item())
    assert need == _golden(N)[6]
    bufs = gh.Buffers(need, keys=True)
    assert gh.polygonize_into(sdb, N, bufs) == gh.GH_OK
    assert int(bufs.counts[0].item()) == need


def test_invalid_arguments():
    sdb = gh.CsgSdb(synth.sphere_prims(0.5))
    bufs = gh.Buffers(1000)
    for N in (1, 4096):
        with pytest.raises(gh.GhError) as e:
            gh.polygonize_into(sdb, N, bufs)
        assert e.value.code == gh.GH_ERR_ARG
    with pytest.raises(gh.GhError):
        gh.polygonize_into(sdb, 32, bufs, lo=[-1, -1, -1], hi=[1, 1, 2])
    with pytest.raises(gh.GhError) as e:
        gh.polygonize_into(sdb, 32, bufs, precision="bf16")
    assert e.value.code == gh.GH_ERR_ARG
    bad = synth.sphere_prims(0.5).copy()
    bad[0, 0] = 7
    with pytest.raises(gh.GhError):
        gh.CsgSdb(bad)
    flat = synth.prim_row(synth.CONE, synth.UNION, [0, 0, 0], [0.2, 0.0])[None]
    with pytest.raises(gh.GhError) as e:
        gh.CsgSdb(flat)
    assert e.value.code == gh.GH_ERR_ARG


def test_repeat_calls_are_identical():
    sdb = gh.CsgSdb(synth.csg_prims(2))
    a = gh.polygonize(sdb, 96, keys=True)
    b = gh.polygonize(sdb, 96, keys=True)
    import meshutil
    ka = meshutil.canonical_tris(a.tri_keys.cpu().numpy())
    kb = meshutil.canonical_tris(b.tri_keys.cpu().numpy())
    assert (ka == kb).all()


def test_eval_points_matches_oracle():
    prims = synth.csg_prims(0)
    sdb = gh.CsgSdb(prims)
    P = synth.uniform_points(3, 100000)
    f = gh.eval_points(sdb, torch.from_numpy(P).cuda()).cpu().numpy()
    ref = oracle.csg(prims).eval(P.astype(np.float64))
    assert np.abs(f - ref).max() < parity.EVAL32


@pytest.mark.parametrize("N", [2, 63, 100])
def test_enumeration_equals_hopping_and_oracle(N):
    """Sec. 2 enumeration on the GPU (f at all lattice points, Marching Cubes
    on every cell) gives the grid hopper's mesh bit for bit (same evaluator at
    the same points), and matches the oracle's enumeration."""
    import meshutil
    prims = synth.csg_prims(1)
    sdb = gh.CsgSdb(prims)
    e = gh.polygonize(sdb, N, keys=True, cells=True, method="enum")
    hp = gh.polygonize(sdb, N, keys=True, cells=True)
    assert e.stats["hop_evals"] == (N + 1) ** 3
    assert sorted(e.cell_ids.cpu().tolist()) == sorted(hp.cell_ids.cpu().tolist())
    ke, pe = meshutil.vertex_table(e.tri_keys.cpu().numpy(), e.tri_xyz.cpu().numpy())
    kh, ph = meshutil.vertex_table(hp.tri_keys.cpu().numpy(), hp.tri_xyz.cpu().numpy())
    assert (ke == kh).all() and np.array_equal(pe, ph)
    assert (meshutil.canonical_tris(e.tri_keys.cpu().numpy()) ==
            meshutil.canonical_tris(hp.tri_keys.cpu().numpy())).all()
    o = oracle.csg(prims)
    parity.compare(e, o, N, ref=oracle.enum(o, N), gsdb=sdb)


@pytest.mark.parametrize("N,lo,hi", [(141, -1.0, 1.0), (200, -0.8, 0.8)])
def test_primitive_scene_matches_oracle(N, lo, hi):
    """The seven primitives of the paper's first scene (Sec. 5.1), rotated, in
    a union: every cell against the oracle's enumeration."""
    prims = synth.primitive_scene(0)
    sdb = gh.CsgSdb(prims)
    m = gh.polygonize(sdb, N, lo=lo, hi=hi, keys=True, cells=True)
    o = oracle.csg(prims)
    ref = oracle.enum(o, N, lo, hi)
    # every vertex meets the propagated bound 1e-4 h + h delta32 / |fA - fB|;
    # the rotated flat faces (box, prism, cylinder caps, cone base) put more
    # lattice edges nearly tangent to the surface than curved shapes do, so
    # the share within the bare 1e-4 h is checked at 0.995
    st = parity.compare(m, o, N, lo, hi, ref=ref, min_bare=0.995, gsdb=sdb)
    assert st["cells"] > 5000


def test_primitive_distances_match_oracle():
    """Each new primitive alone, evaluated at points around it (edges, caps
    and apex included), against the FP64 closed forms."""
    rng = np.random.default_rng(4)
    for kind in (synth.CAPSULE, synth.CYLINDER, synth.HEXPRISM, synth.CONE):
        q = rng.standard_normal(4)
        prims = synth.prim_row(kind, synth.UNION, rng.uniform(-0.2, 0.2, 3), rng.uniform(0.1, 0.3, 2),
                               synth._quat_rot(q))[None]
        P = rng.uniform(-0.6, 0.6, (20000, 3)).astype(np.float32)
        got = gh.eval_points(gh.CsgSdb(prims), torch.tensor(P, device="cuda")).cpu().numpy().astype(np.float64)
        ref = oracle.csg(prims).eval(P.astype(np.float64))
        assert np.abs(got - ref).max() < parity.EVAL32, kind


def test_mixed_scene_eval_matches_oracle():
    """97 primitives of all kinds under union, subtraction and a final
    intersection: most primitives are far from a given point, so the
    evaluator skips them by their bounding radius; the result must still be
    the full fold's."""
    prims = synth.mixed_prims(7)
    rng = np.random.default_rng(11)
    P = rng.uniform(-1.0, 1.0, (200000, 3)).astype(np.float32)
    got = gh.eval_points(gh.CsgSdb(prims), torch.tensor(P, device="cuda")).cpu().numpy().astype(np.float64)
    ref = oracle.csg(prims).eval(P.astype(np.float64))
    assert np.abs(got - ref).max() < parity.EVAL32


def test_scaled_rotation_rejected():
    """A scaled rotation would make a primitive's value exceed its distance
    (no longer a bound, Sec. 1): rejected at creation."""
    prims = synth.mixed_prims(7)
    prims[3, 8:17] = synth._f32(prims[3, 8:17] * 1.25)
    with pytest.raises(gh.GhError) as e:
        gh.CsgSdb(prims)
    assert e.value.code == gh.GH_ERR_ARG and "orthonormal" in str(e.value)


def test_mixed_scene_polygonize_matches_oracle():
    """The 97-primitive scene polygonised (hopper, vertex evaluation and
    Marching Cubes all take the skipping evaluator): every cell against the
    oracle's enumeration."""
    prims = synth.mixed_prims(7)
    N = 150
    sdb = gh.CsgSdb(prims)
    m = gh.polygonize(sdb, N, keys=True, cells=True)
    o = oracle.csg(prims)
    st = parity.compare(m, o, N, ref=oracle.enum(o, N), min_bare=0.995, gsdb=sdb)
    assert st["cells"] > 5000
