"""The paper's network form on the GPU (Sec. 5.2): 8 layers of width 64 with
batch normalisation folded in, SDB = network / 1.5, no radial term.  FP32
and BF16+refine meshes against the FP64 oracle's enumeration, the GPU
enumeration against the GPU hopper, and the implicit adjoint of the
radial-free form against the oracle."""
import numpy as np
import pytest

import meshutil
import oracle
import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2111_05778_gb300 import gh, synth  # noqa: E402


@pytest.fixture(scope="module")
def net():
    params, W, L, lam, _ = synth.paper_network(0)
    sdb = gh.paper_mlp(params, W, L, lam)
    o = oracle.mlp(W, L, params.astype(np.float64), r0=0.0, alpha=1.0, beta=1.0, lam=lam, radial=False)
    return params, W, L, lam, sdb, o


def test_paper_network_eval_matches_oracle(net):
    params, W, L, lam, sdb, o = net
    P = torch.from_numpy(synth.uniform_points(21, 50001)).cuda()
    f = gh.eval_points(sdb, P, "fp32").cpu().numpy().astype(np.float64)
    ref = o.eval(P.cpu().numpy().astype(np.float64))
    assert np.abs(f - ref).max() < parity.EVAL32


@pytest.mark.parametrize("N,lo,hi", [(100, -1.0, 1.0), (77, -0.9, 0.85)])
def test_paper_network_fp32_matches_oracle(net, N, lo, hi):
    params, W, L, lam, sdb, o = net
    m = gh.polygonize(sdb, N, lo=lo, hi=hi, keys=True, cells=True)
    ref = oracle.enum(o, N, lo, hi)
    st = parity.compare(m, o, N, lo, hi, ref=ref, gsdb=sdb)
    assert st["cells"] > 3000


def test_paper_network_bf16_refine(net):
    params, W, L, lam, sdb, o = net
    N = 128
    eps = sdb.calibrate(N)
    m = gh.polygonize(sdb, N, precision="bf16", eps=eps, keys=True, cells=True)
    parity.compare(m, o, N, ref=oracle.enum(o, N), gsdb=sdb)
    m32 = gh.polygonize(sdb, N, precision="fp32", keys=True)
    assert (meshutil.canonical_tris(m.tri_keys.cpu().numpy()) ==
            meshutil.canonical_tris(m32.tri_keys.cpu().numpy())).all()


def test_paper_network_hop_equals_gpu_enumeration(net):
    """Sec. 5.2: with lambda = 1.5 the methods give identical meshes."""
    params, W, L, lam, sdb, o = net
    N = 160
    a = gh.polygonize(sdb, N, keys=True)
    b = gh.polygonize(sdb, N, keys=True, method="enum")
    assert a.n_tris == b.n_tris > 10000
    assert (meshutil.canonical_tris(a.tri_keys.cpu().numpy()) ==
            meshutil.canonical_tris(b.tri_keys.cpu().numpy())).all()
    assert a.stats["hop_evals"] < b.stats["hop_evals"] / 4


def test_paper_network_adjoint(net):
    params, W, L, lam, sdb, o = net
    m = gh.polygonize(sdb, 96, indexed=True)
    V = m.verts
    c = torch.tensor([0.02, -0.01, 0.03], device="cuda")
    r = (V - c).norm(dim=1, keepdim=True)
    G = (2 * (r - 0.45) / r) * (V - c) / V.shape[0]
    g = gh.backward(sdb, V, G).cpu().numpy().astype(np.float64)
    Vn, Gn = V.cpu().numpy().astype(np.float64), G.cpu().numpy().astype(np.float64)
    ref = oracle.np_adjoint(params.astype(np.float64), W, L, Vn, Gn, r0=0.0, alpha=1.0, beta=1.0, lam=lam,
                            radial=False)
    scale = np.maximum(np.abs(ref), 1e-2 * np.abs(ref).max())
    assert (np.abs(g - ref) <= 1e-3 * scale).mean() > 0.995
