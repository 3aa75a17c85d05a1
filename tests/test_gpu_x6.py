"""The split-BF16 tensor-core evaluator ("x6": each FP32 operand split into
three BF16 parts, six part products accumulated in FP32) against the FP64
oracle and against plain FP32, and the BF16 path refined with it
(GH_BF16_REFINE_X6) against the oracle.  It may replace FP32 refinement
only with an error against FP64 no larger than plain FP32's."""
import numpy as np
import pytest

import oracle
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth  # noqa: E402


def _edge_endpoints(mesh, N, lo=-1.0, hi=1.0):
    """float32 positions of both end points of every crossing lattice edge of a
    mesh (the vertices refinement re-evaluates), from its edge keys."""
    k = np.unique(mesh.tri_keys.cpu().numpy().astype(np.int64))
    N1 = N + 1
    ax, r = k // N1**3, k % N1**3
    A = np.stack([r % N1, (r // N1) % N1, r // N1**2], 1)
    B = A.copy()
    B[np.arange(B.shape[0]), ax] += 1
    return parity.lattice32(np.unique(np.concatenate([A, B]), axis=0), N, lo, hi)


def _pair(seed, width):
    p = synth.mlp_params(seed, width)
    return gh.MlpSdb(p, width), oracle.mlp(width, synth.MLP_NMID, p.astype(np.float64))


def _errors(sdb, o, P):
    ref = o.eval_many(P.cpu().numpy().astype(np.float64))
    f32 = gh.eval_points(sdb, P, "fp32").cpu().numpy().astype(np.float64)
    fx6 = gh.eval_points(sdb, P, "bf16x6").cpu().numpy().astype(np.float64)
    return np.abs(f32 - ref), np.abs(fx6 - ref)


@pytest.mark.parametrize("width", [64, 128, 256])
def test_x6_error_no_larger_than_fp32(width):
    """f of the workloads' form (|p| - 0.6 + 0.1 g) / 1.1, where the FP32
    radial term shares the error, and the network alone (f = g), where all of
    the error is the hidden layers' arithmetic."""
    p = synth.mlp_params(1, width)
    n = (1 << 20) + 77  # 2^20 uniform points and a ragged tail
    P = torch.from_numpy(synth.uniform_points(12, n)).cuda()
    out = {}
    for form, kw in (("radial", {}), ("network", dict(r0=0.0, alpha=1.0, beta=1.0, radial=False))):
        sdb = gh.MlpSdb(p, width, **kw)
        o = oracle.mlp(width, synth.MLP_NMID, p.astype(np.float64), **kw)
        Q = P
        if form == "radial":  # plus the end points of the crossing edges of an N = 256 mesh
            ends = _edge_endpoints(gh.polygonize(sdb, 256, keys=True), 256)
            Q = torch.cat([P, torch.from_numpy(ends).cuda()])
        e32, ex6 = _errors(sdb, o, Q)
        out[form] = (e32.max(), e32.mean(), ex6.max(), ex6.mean())
        print("width %d %s: max |f32 - f64| %.4g (mean %.4g), max |x6 - f64| %.4g (mean %.4g)" % (
            (width, form) + out[form]))
    # the workloads' f: x6's error is FP32's (the FP32 radial term dominates
    # both; the hidden layers add below 1e-9)
    e32max, e32mean, ex6max, ex6mean = out["radial"]
    assert ex6max <= e32max * 1.001
    assert ex6mean <= e32mean * 1.01
    # the network alone: the tensor core's FP32 accumulation over 6 x W/16
    # updates per output gives up to 3x FP32's error at width 256 (below 1e-8)
    e32max, e32mean, ex6max, ex6mean = out["network"]
    assert ex6max <= 2.0 * e32max and ex6max < 1e-8
    assert ex6mean <= 3.0 * e32mean


@pytest.mark.parametrize("width,N", [(64, 40), (128, 48), (256, 64)])
def test_bf16_x6_refine_full(width, N):
    sdb, o = _pair(1 + width, width)
    eps = sdb.calibrate(N)
    m = gh.polygonize(sdb, N, precision="bf16x6", eps=eps, keys=True, cells=True)
    st = parity.compare(m, o, N, ref=oracle.enum(o, N), gsdb=sdb, gprec="bf16x6")
    print("x6 refine width %d N %d: %s" % (width, N, st))
    assert st["cells"] > 1000
    assert m.stats["refined_vertices"] > 0
    assert st["sign_flip_outside_band"] <= 8
