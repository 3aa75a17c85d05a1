"""The no-allocation entry point gh_polygonize_csg_noalloc, for callers that
cannot allocate device memory while they polygonize: a plug-in inside a host
application that owns the whole device-memory budget, or a loop that must not
call cudaMalloc / cudaFree because those calls can block on, or synchronise
with, work already running on the device.  Through the C ABI, on two calls in
a row through the same static scratch, its output must equal that of
gh_polygonize on the same scene: both run the same kernels on the same
inputs, so the meshes are the same triangles with bit-identical vertex
positions.

Kept in a file that pytest collects last, so that a run stopping at the first
failure has run every other test before it."""
import numpy as np
import pytest

import meshutil

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth  # noqa: E402


def _check_same(bufs, ref):
    T = int(bufs.counts[0].item())
    assert T == ref.n_tris
    keys = bufs.tri_keys[:T].cpu().numpy()
    pos = bufs.tri_xyz[:T].cpu().numpy()
    rk = ref.tri_keys.cpu().numpy()
    rp = ref.tri_xyz.cpu().numpy()
    assert np.array_equal(meshutil.canonical_tris(keys), meshutil.canonical_tris(rk))
    uk, up = meshutil.vertex_table(keys, pos)
    rk2, rp2 = meshutil.vertex_table(rk, rp)
    assert np.array_equal(uk, rk2)
    assert np.array_equal(up.view(np.uint32), rp2.view(np.uint32))


CASES = [(synth.csg_prims(0), 128, -1.0, 1.0), (synth.sphere_prims(0.5), 200, -0.8, 0.8),
         (synth.mixed_prims(7), 150, -1.0, 1.0)]


def test_noalloc_matches_polygonize_on_two_calls():
    for prims, N, lo, hi in CASES:
        ref = gh.polygonize(gh.CsgSdb(prims), N, lo=lo, hi=hi, keys=True)
        bufs = gh.Buffers(ref.n_tris + 100, keys=True)
        pd = gh.csg_prims_device(prims)
        for _ in range(2):
            assert gh.polygonize_csg_noalloc(pd, prims.shape[0], N, bufs, lo=lo, hi=hi) == gh.GH_OK
            _check_same(bufs, ref)


def test_noalloc_allocates_no_device_memory():
    """After a first call (which loads the library's kernels and its static
    array), further calls on other scenes leave the device's free memory
    unchanged to the byte."""
    inputs = []
    for prims, N, lo, hi in CASES:
        ref = gh.polygonize(gh.CsgSdb(prims), N, lo=lo, hi=hi, keys=True)
        inputs.append((gh.csg_prims_device(prims), prims.shape[0], N, lo, hi, ref,
                       gh.Buffers(ref.n_tris + 100, keys=True)))
    pd, n, N, lo, hi, ref, bufs = inputs[0]
    assert gh.polygonize_csg_noalloc(pd, n, N, bufs, lo=lo, hi=hi) == gh.GH_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for pd, n, N, lo, hi, ref, bufs in inputs[1:] + inputs[:1]:
        assert gh.polygonize_csg_noalloc(pd, n, N, bufs, lo=lo, hi=hi) == gh.GH_OK
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    for pd, n, N, lo, hi, ref, bufs in inputs:
        _check_same(bufs, ref)


def test_noalloc_capacity_overflow_then_clean_call():
    """A scene that marks more cells than the static array holds (eight thin
    slabs across the domain at N = 256, about 2 M marked cells) gets
    GH_ERR_CAPACITY with both numbers in the message; the next call, on a
    small scene through the same array, is correct."""
    slabs = np.stack([synth.prim_row(synth.BOX, synth.UNION, [0.0, 0.0, z], [0.8, 0.8, 0.02])
                      for z in np.linspace(-0.7, 0.7, 8)])
    pd = gh.csg_prims_device(slabs)
    bufs = gh.Buffers(1000, keys=True)
    assert gh.polygonize_csg_noalloc(pd, slabs.shape[0], 256, bufs) == gh.GH_ERR_CAPACITY
    msg = gh.lib().gh_last_error().decode()
    assert "marks" in msg and "holds" in msg, msg
    prims, N, lo, hi = CASES[1]
    ref = gh.polygonize(gh.CsgSdb(prims), N, lo=lo, hi=hi, keys=True)
    bufs = gh.Buffers(ref.n_tris + 100, keys=True)
    pd = gh.csg_prims_device(prims)
    assert gh.polygonize_csg_noalloc(pd, prims.shape[0], N, bufs, lo=lo, hi=hi) == gh.GH_OK
    _check_same(bufs, ref)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    prims = synth.sphere_prims(0.5)
    pd = gh.csg_prims_device(prims)
    bufs = gh.Buffers(1000, keys=True)
    with pytest.raises(gh.GhError) as e:
        gh.polygonize_csg_noalloc(pd, 1, gh.NOALLOC_MAX_N + 1, bufs)
    assert e.value.code == gh.GH_ERR_ARG
