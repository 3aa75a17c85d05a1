"""GPU parity of the BF16 tensor-core path (tcgen05 hopper with the eps
shrink, FP32 re-evaluation of the corners of candidate cells) against the
FP32 path and the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import meshutil
import oracle
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth  # noqa: E402


def _pair(seed, width):
    p = synth.mlp_params(seed, width)
    return gh.MlpSdb(p, width), oracle.mlp(width, synth.MLP_NMID, p.astype(np.float64))


@pytest.mark.parametrize("width", [64, 128, 256])
def test_bf16_eval_close_to_fp32(width):
    sdb, o = _pair(1, width)
    n = 70001  # several tiles of 256 rows and a ragged tail
    P = torch.from_numpy(synth.uniform_points(9, n)).cuda()
    f32 = gh.eval_points(sdb, P, "fp32").cpu().numpy().astype(np.float64)
    f16 = gh.eval_points(sdb, P, "bf16").cpu().numpy().astype(np.float64)
    ref = o.eval(P.cpu().numpy().astype(np.float64))
    assert np.abs(f32 - ref).max() < 1e-6
    gap = np.abs(f16 - f32)
    # BF16 activations: a relative error of a few 2^-9 of g's scale, far below a cell
    assert gap.max() < 2e-4, gap.max()
    assert gap.mean() < 2e-5


@pytest.mark.parametrize("width", [64, 256])
def test_calibration_bounds_the_bf16_error(width):
    sdb, _ = _pair(3, width)
    eps = sdb.calibrate(256, n_points=1 << 18, seed=5)
    assert 0 < eps < 1e-3
    P = torch.from_numpy(synth.uniform_points(11, 100000)).cuda()
    gap = (gh.eval_points(sdb, P, "bf16") - gh.eval_points(sdb, P, "fp32")).abs().max().item()
    assert gap <= eps / 2


@pytest.mark.parametrize("width,N", [(64, 40), (128, 48), (256, 64)])
def test_bf16_refine_full(width, N):
    sdb, o = _pair(1 + width, width)
    eps = sdb.calibrate(N)
    m = gh.polygonize(sdb, N, precision="bf16", eps=eps, keys=True, cells=True)
    ref = oracle.enum(o, N)
    st = parity.compare(m, o, N, ref=ref, gsdb=sdb)
    assert st["cells"] > 1000
    assert st["sign_flip_outside_band"] <= 8
    assert m.stats["refined_vertices"] > 0
    # identical mesh to the FP32 path: the surface cells' corners are FP32 values
    m32 = gh.polygonize(sdb, N, precision="fp32", keys=True)
    assert (meshutil.canonical_tris(m.tri_keys.cpu().numpy()) ==
            meshutil.canonical_tris(m32.tri_keys.cpu().numpy())).all()
    ua, pa = meshutil.vertex_table(m.tri_keys.cpu().numpy(), m.tri_xyz.cpu().numpy())
    ub, pb = meshutil.vertex_table(m32.tri_keys.cpu().numpy(), m32.tri_xyz.cpu().numpy())
    assert np.array_equal(ua, ub) and np.array_equal(pa.view(np.uint32), pb.view(np.uint32))


def test_bf16_needs_eps():
    sdb, _ = _pair(1, 64)
    with pytest.raises(gh.GhError) as e:
        gh.polygonize(sdb, 32, precision="bf16")
    assert e.value.code == gh.GH_ERR_ARG
