"""The no-allocation entry point gh_polygonize_csg_noalloc, for callers that
cannot allocate device memory while they polygonize (for example a plug-in in
a host application that owns the device-memory budget, or a loop that must not
call cudaMalloc / cudaFree).  Its output must equal that of gh_polygonize on
the same scene, on two calls in a row through the same static scratch.

Kept in a file that pytest collects last, so that a run stopping at the first
failure has run every other test before it."""
import numpy as np
import pytest

import meshutil

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth  # noqa: E402


def _check_same(bufs, ref, N, lo, hi):
    T = int(bufs.counts[0].item())
    assert T == ref.n_tris
    keys = bufs.tri_keys[:T].cpu().numpy()
    pos = bufs.tri_xyz[:T].cpu().numpy().astype(np.float64)
    rk = ref.tri_keys.cpu().numpy()
    rp = ref.tri_xyz.cpu().numpy().astype(np.float64)
    assert (meshutil.canonical_tris(keys) == meshutil.canonical_tris(rk)).all()
    uk, up = meshutil.vertex_table(keys, pos)
    rk2, rp2 = meshutil.vertex_table(rk, rp)
    assert (uk == rk2).all()
    h = (hi - lo) / N
    assert np.abs(up - rp2).max() <= 1e-4 * h  # the tolerance of the parity tests


def test_noalloc_matches_polygonize_on_two_calls():
    cases = [(synth.csg_prims(0), 128, -1.0, 1.0), (synth.sphere_prims(0.5), 200, -0.8, 0.8),
             (synth.mixed_prims(7), 150, -1.0, 1.0)]
    for prims, N, lo, hi in cases:
        ref = gh.polygonize(gh.CsgSdb(prims), N, lo=lo, hi=hi, keys=True)
        bufs = gh.Buffers(ref.n_tris + 100, keys=True)
        pd = gh.csg_prims_device(prims)
        assert gh.polygonize_csg_noalloc(pd, prims.shape[0], N, bufs, lo=lo, hi=hi) == gh.GH_OK
        _check_same(bufs, ref, N, lo, hi)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    prims = synth.sphere_prims(0.5)
    pd = gh.csg_prims_device(prims)
    bufs = gh.Buffers(1000, keys=True)
    with pytest.raises(gh.GhError) as e:
        gh.polygonize_csg_noalloc(pd, 1, gh.NOALLOC_MAX_N + 1, bufs)
    assert e.value.code == gh.GH_ERR_ARG
