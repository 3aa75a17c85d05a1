"""The paper's own network form (Sec. 5.2): eight ReLU layers of width 64
with batch normalisation in all but the last, folded into the weights for
inference, SDB = network / lambda with lambda = 1.5, no radial term.

CPU pins: the folding against an explicit FP64 forward pass with the
normalisation applied as its definition states; the architecture's size;
the oracle's radial-free form against a closed form; and the paper's
observation that with lambda = 1.5 hopping yields exactly the enumeration
mesh, checked with the FP64 oracle on the trained stand-in network."""
import numpy as np
import pytest

import oracle
from paper_2111_05778_gb300 import synth
from paper_2111_05778_gb300.bn import fold_batchnorm


def _bn_forward(linears, norms, P, eps=1e-5):
    a = P
    for i, ((W, b), bn) in enumerate(zip(linears, norms)):
        z = a @ np.asarray(W, np.float64).T + b
        if bn is not None:
            g, be, m, v = (np.asarray(x, np.float64) for x in bn)
            z = (z - m) / np.sqrt(v + eps) * g + be
        a = np.maximum(z, 0.0) if i + 1 < len(linears) else z
    return a[:, 0]


def test_fold_batchnorm_hand_case():
    W = np.array([[1.0, -2.0, 0.5]])
    b = np.array([0.25])
    bn = (np.array([2.0]), np.array([1.0]), np.array([0.5]), np.array([3.0]))
    (Wf, bf), = fold_batchnorm([(W, b)], [bn], eps=1.0)
    # y = 2 (W p + 0.25 - 0.5) / sqrt(3 + 1) + 1 = W p - 0.25 + 1
    np.testing.assert_allclose(Wf, W, atol=1e-15)
    np.testing.assert_allclose(bf, [0.75], atol=1e-15)


def test_fold_batchnorm_matches_unfolded_forward():
    rng = np.random.default_rng(0)
    dims = [3, 16, 16, 1]
    linears = [(rng.standard_normal((dims[i + 1], dims[i])), rng.standard_normal(dims[i + 1])) for i in range(3)]
    norms = [(rng.uniform(0.5, 2, 16), rng.normal(0, 0.3, 16), rng.normal(0, 0.3, 16), rng.uniform(0.2, 3, 16))
             for _ in range(2)] + [None]
    P = rng.uniform(-1, 1, (500, 3))
    folded = fold_batchnorm(linears, norms)
    a = P
    for i, (W, b) in enumerate(folded):
        a = a @ W.T + b
        if i + 1 < len(folded):
            a = np.maximum(a, 0.0)
    np.testing.assert_allclose(a[:, 0], _bn_forward(linears, norms, P), rtol=1e-12, atol=1e-12)


def test_radial_free_closed_form():
    """Width 3, identity layers: g(p) = sum relu(p_i) + 0.25 and, without the
    radial term, f = (alpha g - r0) / beta / lambda."""
    I = np.eye(3, dtype=np.float32)
    layers = [(I, np.zeros(3, np.float32))] * 3 + [(np.ones((1, 3), np.float32), np.array([0.25], np.float32))]
    s = oracle.mlp(3, 2, synth.pack_layers(layers).astype(np.float64), r0=0.1, alpha=2.0, beta=1.25, lam=1.5,
                   radial=False)
    P = np.random.default_rng(1).uniform(-1, 1, (100, 3))
    ref = (2.0 * (np.maximum(P, 0).sum(1) + 0.25) - 0.1) / 1.25 / 1.5
    np.testing.assert_allclose(s.eval(P), ref, atol=1e-15)
    # its x-gradient has no p/|p| part
    gx = s.grad_x(P)
    np.testing.assert_allclose(gx, 2.0 * (P > 0) / 1.25 / 1.5, atol=1e-12)


@pytest.fixture(scope="module")
def paper_net():
    return synth.paper_network(0)


def test_paper_network_architecture(paper_net):
    params, W, L, lam, (linears, norms) = paper_net
    assert (W, L, lam) == (64, 6, 1.5)
    assert len(linears) == 8 and sum(bn is not None for bn in norms) == 7 and norms[-1] is None
    assert [l[0].shape for l in linears] == [(64, 3)] + [(64, 64)] * 6 + [(1, 64)]
    # weights and biases 25,281 plus 2 x 448 normalisation parameters, near
    # the network size Sec. 5.2 gives
    assert params.size == 25281 == synth.mlp_param_count(64, 6)
    # the packed parameters are the fold of the trained layers
    P = np.random.default_rng(2).uniform(-1, 1, (300, 3))
    s = oracle.mlp(W, L, params.astype(np.float64), r0=0.0, alpha=1.0, beta=1.0, lam=1.0, radial=False)
    np.testing.assert_allclose(s.eval(P), _bn_forward(linears, norms, P), rtol=0, atol=2e-5)


def test_paper_network_is_a_working_sdb_at_lambda_15(paper_net):
    """Sec. 5.2: with the network divided by lambda = 1.5 the hopper's surface
    equals the enumeration's (the oracle, FP64, N = 48)."""
    params, W, L, lam, _ = paper_net
    s = oracle.mlp(W, L, params.astype(np.float64), r0=0.0, alpha=1.0, beta=1.0, lam=lam, radial=False)
    N = 48
    _, mr = oracle.polygonize(s, N)
    er = oracle.enum(s, N)
    surf = lambda r: np.sort(r.cells[(r.cases > 0) & (r.cases < 255)])
    assert np.array_equal(surf(mr), surf(er))
    assert surf(er).size > 1000
