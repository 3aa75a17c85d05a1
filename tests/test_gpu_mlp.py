"""GPU parity of the neural-SDB path (FP32 on the FFMA pipe) against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth  # noqa: E402


def _pair(seed, width):
    p = synth.mlp_params(seed, width)
    return gh.MlpSdb(p, width), oracle.mlp(width, synth.MLP_NMID, p.astype(np.float64))


@pytest.mark.parametrize("width", [64, 128, 256])
def test_eval_fp32_pointwise(width):
    sdb, o = _pair(1, width)
    P = synth.uniform_points(5, 20000)
    f = gh.eval_points(sdb, torch.from_numpy(P).cuda()).cpu().numpy()
    assert np.abs(f - o.eval(P.astype(np.float64))).max() < 1e-6


@pytest.mark.parametrize("width,N", [(64, 40), (128, 48), (256, 56)])
def test_mlp_fp32_full(width, N):
    sdb, o = _pair(1 + width, width)
    m = gh.polygonize(sdb, N, keys=True, cells=True)
    ref = oracle.enum(o, N)
    st = parity.compare(m, o, N, ref=ref, gsdb=sdb)
    assert st["cells"] > 1000
    assert st["sign_flip_outside_band"] <= 8


def test_enumeration_equals_hopping_mlp():
    import meshutil
    sdb, o = _pair(4, 64)
    N = 48
    e = gh.polygonize(sdb, N, keys=True, cells=True, method="enum")
    hp = gh.polygonize(sdb, N, keys=True, cells=True)
    ke, pe = meshutil.vertex_table(e.tri_keys.cpu().numpy(), e.tri_xyz.cpu().numpy())
    kh, ph = meshutil.vertex_table(hp.tri_keys.cpu().numpy(), hp.tri_xyz.cpu().numpy())
    assert (ke == kh).all() and np.array_equal(pe, ph)
    parity.compare(e, o, N, ref=oracle.enum(o, N), gsdb=sdb)
    with pytest.raises(gh.GhError):
        gh.polygonize(sdb, N, method="enum", precision="bf16", eps=1e-5)
