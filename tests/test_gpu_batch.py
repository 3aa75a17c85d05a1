"""GPU batch path (gh_polygonize_batch): one persistent hopping launch per
evaluator family over device work queues, batched vertex evaluation, per-item
lists and Marching Cubes, CUDA-graph capture and replay, and the autotuner.
Every item must equal the single-call result (itself checked against the
oracle elsewhere), and one item is checked against the oracle directly."""
import os

import numpy as np
import pytest

import meshutil
import oracle
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth, tune  # noqa: E402


def _sdb(kind, seed, width):
    if kind == "csg":
        return gh.CsgSdb(synth.csg_prims(seed))
    return gh.MlpSdb(synth.mlp_params(seed, width), width)


def _same(a, b, N):
    ka = meshutil.canonical_tris(a.tri_keys.cpu().numpy())
    kb = meshutil.canonical_tris(b.tri_keys.cpu().numpy())
    assert ka.shape == kb.shape and (ka == kb).all()
    ua, pa = meshutil.vertex_table(a.tri_keys.cpu().numpy(), a.tri_xyz.cpu().numpy())
    ub, pb = meshutil.vertex_table(b.tri_keys.cpu().numpy(), b.tri_xyz.cpu().numpy())
    assert (ua == ub).all() and np.array_equal(pa, pb)


def test_mixed_batch_fp32_equals_single_calls():
    spec = [("csg", 0, 0, 160), ("mlp", 1, 64, 96), ("csg", 2, 0, 37), ("mlp", 3, 128, 128),
            ("csg", 4, 0, 200), ("mlp", 5, 64, 2)]
    sdbs = [_sdb(k, s, w) for k, s, w, _ in spec]
    Ns = [n for *_, n in spec]
    bt = gh.polygonize_batch(sdbs, Ns, keys=True)
    for b, (k, s, w, N) in enumerate(spec):
        single = gh.polygonize(_sdb(k, s, w), N, keys=True)
        _same(bt.mesh(b), single, N)
        assert bt.mesh(b).stats["surface_cells"] == single.stats["surface_cells"]
    # one item straight against the oracle (enumeration)
    o = oracle.csg(synth.csg_prims(0))
    ref = oracle.enum(o, 160)
    m = bt.mesh(0)
    cells = np.asarray(parity.tri_cells(m.tri_keys.cpu().numpy(), 160))
    assert cells.min() >= 0
    ct = meshutil.canonical_tris(m.tri_keys.cpu().numpy())
    co = meshutil.canonical_tris(ref.tri_keys)
    assert ct.shape[0] == co.shape[0]


def test_bf16_batch_equals_single_calls_and_graph_replay():
    spec = [(1, 64, 128), (3, 128, 96), (5, 256, 160), (7, 64, 64)]
    sdbs, Ns = [], []
    for seed, w, N in spec:
        s = gh.MlpSdb(synth.mlp_params(seed, w), w)
        s.calibrate(N)
        sdbs.append(s)
        Ns.append(N)
    for tiles in (1, 2):
        bt = gh.polygonize_batch(sdbs, Ns, precision="bf16", keys=True, mlp_tiles=tiles)
        for b, s in enumerate(sdbs):
            single = gh.polygonize(s, Ns[b], precision="bf16", eps=s.eps, keys=True)
            _same(bt.mesh(b), single, Ns[b])
            f32 = gh.polygonize(s, Ns[b], precision="fp32", keys=True)
            _same(bt.mesh(b), f32, Ns[b])
    # graph: capture, wipe the outputs, replay, compare
    caps = [int(c) + 4096 for c in bt.counts()]
    g = gh.Batch(sdbs, Ns, caps, precision="bf16", keys=True)
    g.capture()
    ref = [g.mesh(b) for b in range(len(sdbs))]
    ref = [(m.tri_keys.clone(), m.tri_xyz.clone()) for m in ref]
    for bb in g.bufs:
        bb.tri_keys.zero_()
        bb.tri_xyz.zero_()
        bb.counts.zero_()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for b in range(len(sdbs)):
        m = g.mesh(b)
        assert m.n_tris == ref[b][0].shape[0]
        a = meshutil.canonical_tris(m.tri_keys.cpu().numpy())
        c = meshutil.canonical_tris(ref[b][0].cpu().numpy())
        assert (a == c).all()
    g.close()


def test_autotuner_picks_a_candidate(tmp_path):
    os.environ["GH_TUNE_CACHE"] = str(tmp_path / "tune.json")
    sdbs = [_sdb("csg", 0, 0), _sdb("mlp", 1, 64)]
    for s in sdbs[1:]:
        s.calibrate(96)
    rb, mt, t = tune.tune_batch(sdbs, [128, 96], precision="bf16")
    assert (rb, mt) in tune.CANDIDATES
    assert len(t) >= 2
    rb2, mt2, _ = tune.tune_batch(sdbs, [128, 96], precision="bf16")
    assert (rb2, mt2) == (rb, mt)
    assert os.path.exists(tmp_path / "tune.json")


@pytest.mark.parametrize("precision", ["bf16", "bf16x6"])
def test_full_batch_config_64_items(precision):
    """The 64-item batch (seeds 0..63: even CSG, odd neural of width 64/128/256,
    N from {128,...,1024}): every item equals its single-call result mesh for
    mesh (same triangles, bit-identical vertices), and the items with N <= 256
    match the oracle -- every column for the analytic items and the N = 128
    neural ones, 256 random columns for the N = 256 neural ones."""
    items = synth.batch_items(64)
    sdbs, Ns = [], []
    for kind, seed, N, W in items:
        s = _sdb(kind, seed, W)
        if kind == "mlp":
            s.calibrate(N, n_points=1 << 18)
        sdbs.append(s)
        Ns.append(N)
    bt = gh.polygonize_batch(sdbs, Ns, precision=precision, keys=True, cells=True)
    # a fixed number of launches, whatever the number of items: counters, one
    # hopping launch per evaluator family (analytic, neural widths 64/128/256),
    # lists (8), vertex values (1 + 3), refinement (3 + 3), Marching Cubes,
    # status words
    launches, _ = gh.last_profile()
    assert launches == 1 + 4 + 8 + 4 + 6 + 1 + 1
    fam = {}
    for b, (kind, _, _, W) in enumerate(items):
        fam.setdefault((kind, W if kind == "mlp" else 0), b)
    pick = sorted(fam.values())  # one item of each family: the same launches as 64
    small = gh.polygonize_batch([sdbs[b] for b in pick], [Ns[b] for b in pick], precision=precision)
    assert gh.last_profile()[0] == launches and small.mesh(0).n_tris > 0
    checked = 0
    for b, (kind, seed, N, W) in enumerate(items):
        m = bt.mesh(b)
        single = gh.polygonize(sdbs[b], N, precision=precision if kind == "mlp" else "fp32",
                               eps=sdbs[b].eps if kind == "mlp" else None, keys=True)
        _same(m, single, N)
        assert m.stats["surface_cells"] == single.stats["surface_cells"], (b, kind, N)
        if N > 256:
            continue
        if kind == "csg":
            o = oracle.csg(synth.csg_prims(seed))
        else:
            o = oracle.mlp(W, synth.MLP_NMID, synth.mlp_params(seed, W).astype(np.float64))
        gprec = precision if kind == "mlp" else "fp32"
        if kind == "csg" or N == 128:
            _, ref = oracle.polygonize(o, N)
            st = parity.compare(m, o, N, ref=ref, gsdb=sdbs[b], gprec=gprec, min_bare=0.995)
        else:
            cols = np.random.default_rng(seed).choice(N * N, 256, replace=False)
            _, ref = oracle.polygonize(o, N, cols=cols)
            st = parity.compare(m, o, N, ref=ref, restrict_cells=lambda c: np.isin(c // N, cols), gsdb=sdbs[b],
                                gprec=gprec, min_bare=0.995)
        assert st["sign_flip_outside_band"] <= 8
        checked += 1
    assert checked == 26
