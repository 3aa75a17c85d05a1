"""Runtime around the kernels: the scratch pool that hands a destroyed SDB's
polygonization buffers to the next SDB, and the device-side derivation of the
network's weight layouts (its results must not depend on which SDB object
ran before)."""
import numpy as np
import pytest

import meshutil
import oracle
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth  # noqa: E402


def _canon(m):
    return meshutil.canonical_tris(m.tri_keys.cpu().numpy())


def test_pooled_scratch_gives_identical_meshes():
    gh.release_cache()
    p = synth.mlp_params(2, 128)
    a = gh.MlpSdb(p, 128)
    ref = gh.polygonize(a, 160, keys=True)
    ref_t = _canon(ref)
    a.close()  # its scratch goes to the pool
    b = gh.MlpSdb(p, 128)  # takes it
    m = gh.polygonize(b, 160, keys=True)
    assert (_canon(m) == ref_t).all()
    # every count but row_slots (tile steps: depends on the dynamic column claims)
    strip = lambda st: {k: v for k, v in st.items() if k != "row_slots"}
    assert strip(m.stats) == strip(ref.stats)
    b.close()
    # an analytic SDB on a smaller grid reuses the same buffers
    prims = synth.csg_prims(4)
    c = gh.CsgSdb(prims)
    mc = gh.polygonize(c, 96, keys=True, cells=True)
    o = oracle.csg(prims)
    parity.compare(mc, o, 96, ref=oracle.enum(o, 96), gsdb=c)
    c.close()
    gh.release_cache()
    d = gh.MlpSdb(p, 128)
    assert (_canon(gh.polygonize(d, 160, keys=True)) == ref_t).all()


def test_device_weight_layouts_match_oracle_in_both_engines():
    p = synth.mlp_params(6, 64)
    sdb = gh.MlpSdb(p, 64)
    o = oracle.mlp(64, synth.MLP_NMID, p.astype(np.float64))
    P = torch.from_numpy(synth.uniform_points(17, 30001)).cuda()
    ref = o.eval(P.cpu().numpy().astype(np.float64))
    f32 = gh.eval_points(sdb, P, "fp32").cpu().numpy().astype(np.float64)
    f16 = gh.eval_points(sdb, P, "bf16").cpu().numpy().astype(np.float64)
    assert np.abs(f32 - ref).max() < parity.EVAL32
    assert np.abs(f16 - ref).max() < 2e-4
