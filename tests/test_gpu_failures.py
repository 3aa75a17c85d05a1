"""Failures injected from the host (no GPU fault is ever provoked): SDBs whose
evaluation is not finite, parameters that are not finite, and grids outside
the accepted range -- each must come back as its status code, and the
context must stay usable for the next correct call."""
import numpy as np
import pytest

import meshutil

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth  # noqa: E402


def _overflowing_params(width, seed=3):
    """Finite weights whose activations overflow float32: layer 0 and every
    hidden layer scaled by 1e30, so f is inf or NaN at every point."""
    layers = synth.mlp_layers(seed, width)
    out = []
    for li, (Wm, b) in enumerate(layers):
        s = 1e30 if li < len(layers) - 1 else 1.0
        out.append((Wm * s, b))
    return synth.pack_layers(out).astype(np.float32)


def test_nonfinite_parameters_rejected_at_creation():
    p = synth.mlp_params(1, 64).copy()
    p[100] = np.nan
    with pytest.raises(gh.GhError) as e:
        gh.MlpSdb(p, 64)
    assert e.value.code == gh.GH_ERR_NONFINITE
    p[100] = np.inf
    with pytest.raises(gh.GhError) as e:
        gh.MlpSdb(p, 64)
    assert e.value.code == gh.GH_ERR_NONFINITE
    prims = synth.sphere_prims(0.5).copy()
    prims[0, 2] = np.nan
    with pytest.raises(gh.GhError) as e:
        gh.CsgSdb(prims)
    assert e.value.code == gh.GH_ERR_ARG


@pytest.mark.parametrize("width", [64, 256])
def test_nonfinite_evaluation_fp32_and_bf16(width):
    bad = gh.MlpSdb(_overflowing_params(width), width)
    for precision, eps in (("fp32", None), ("bf16", 1e-3)):
        with pytest.raises(gh.GhError) as e:
            gh.polygonize(bad, 32, precision=precision, eps=eps)
        assert e.value.code == gh.GH_ERR_NONFINITE, precision
        # asynchronous: the status word carries it
        bufs = gh.Buffers(200000)
        rc = gh.polygonize_into(bad, 32, bufs, precision=precision, eps=eps, sync=False)
        assert rc == gh.GH_OK
        torch.cuda.synchronize()
        assert bufs.stats_dict()["status"] == gh.GH_ERR_NONFINITE
    # the calibration meets the same values
    with pytest.raises(gh.GhError) as e:
        bad.calibrate(32, n_points=4096)
    assert e.value.code == gh.GH_ERR_NONFINITE
    # the context is intact: a correct SDB still gives its mesh
    good = gh.MlpSdb(synth.mlp_params(1, width), width)
    a = gh.polygonize(good, 48, keys=True)
    b = gh.polygonize(good, 48, keys=True)
    assert a.n_tris > 1000
    assert np.array_equal(meshutil.canonical_tris(a.tri_keys.cpu().numpy()),
                          meshutil.canonical_tris(b.tri_keys.cpu().numpy()))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_nonfinite_item_in_a_batch(precision):
    sdbs = [gh.CsgSdb(synth.csg_prims(0)), gh.MlpSdb(_overflowing_params(128), 128),
            gh.MlpSdb(synth.mlp_params(5, 128), 128)]
    with pytest.raises(gh.GhError) as e:
        gh.polygonize_batch(sdbs, [64, 48, 40], precision=precision, eps=1e-3)
    assert e.value.code == gh.GH_ERR_NONFINITE
    assert "item 1" in str(e.value)


def test_batch_rejects_grids_outside_the_range():
    sdbs = [gh.CsgSdb(synth.csg_prims(0)), gh.CsgSdb(synth.sphere_prims(0.5))]
    for bad_n in (1, 0, -3, 2049, 4096):
        with pytest.raises(gh.GhError) as e:
            gh.polygonize_batch(sdbs, [64, bad_n])
        assert e.value.code == gh.GH_ERR_ARG, bad_n
    # and the same SDBs still run
    bt = gh.polygonize_batch(sdbs, [64, 2])
    assert bt.mesh(0).n_tris > 0


@pytest.mark.parametrize("precision", ["fp32", "bf16", "bf16x6"])
def test_bounded_wait_runs_out_then_recovers(precision):
    """Every wait of the neural engines is bounded: with the limit at 0 every
    wait on the engines' own work runs out at once, the kernel records it and
    leaves (tensor-core engines: every role, after its copies land and its
    MMAs complete; FP32 engine: it keeps waiting for its own copy), the call
    reports GH_ERR_CUDA, and the next call with the normal limit on the same
    SDB gives the same mesh as before."""
    sdb = gh.MlpSdb(synth.mlp_params(1, 128), 128)
    eps = sdb.calibrate(96) if precision != "fp32" else None
    ref = gh.polygonize(sdb, 96, precision=precision, eps=eps, keys=True)
    gh.set_wait_limit_ns(0)
    try:
        with pytest.raises(gh.GhError) as e:
            gh.polygonize(sdb, 96, precision=precision, eps=eps, keys=True)
        assert e.value.code == gh.GH_ERR_CUDA and "timed out" in str(e.value)
    finally:
        gh.set_wait_limit_ns(2_000_000_000)
    m = gh.polygonize(sdb, 96, precision=precision, eps=eps, keys=True)
    assert np.array_equal(meshutil.canonical_tris(m.tri_keys.cpu().numpy()),
                          meshutil.canonical_tris(ref.tri_keys.cpu().numpy()))
    with pytest.raises(gh.GhError) as e:
        gh.set_wait_limit_ns(3_000_000_000)
    assert e.value.code == gh.GH_ERR_ARG
