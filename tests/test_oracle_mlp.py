"""Pins for the oracle's neural SDB (Sec. 5.2) and its gradients.

Closed forms with hand-made weights, finite differences of the oracle's own
evaluator (central, FP64), the Lipschitz bound that makes the network a
signed distance bound (Sec. 1), and the implicit-surface adjoint against
finite differences of the loss it differentiates."""
import numpy as np
import pytest

import oracle
from paper_2111_05778_gb300 import synth


def _packed(layers):
    return synth.pack_layers(layers).astype(np.float64)


def test_identity_network_closed_form():
    """Width 3 with identity matrices and zero biases: g(p) = sum relu(p_i)
    summed by an all-ones output row, so f = (|p| - r0 + alpha g) / beta."""
    I = np.eye(3, dtype=np.float32)
    layers = [(I, np.zeros(3, np.float32))] + [(I, np.zeros(3, np.float32))] * 2 + [
        (np.ones((1, 3), np.float32), np.array([0.25], np.float32))]
    s = oracle.mlp(3, 2, _packed(layers), r0=0.6, alpha=0.1, beta=1.1, lam=1.5)
    rng = np.random.default_rng(0)
    P = rng.uniform(-1, 1, (200, 3))
    g = np.maximum(P, 0).sum(1) + 0.25
    ref = (np.linalg.norm(P, axis=1) - 0.6 + 0.1 * g) / 1.1 / 1.5
    np.testing.assert_allclose(s.eval(P), ref, rtol=0, atol=1e-15)


def test_layer_order_and_bias_placement():
    """Non-commuting layers: a permutation then a scaling; biases after each
    matrix and before the ReLU."""
    A = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], np.float32)
    B = np.diag([0.5, 0.25, 0.125]).astype(np.float32)
    b1 = np.array([0.1, -0.2, 0.3], np.float32)
    layers = [(A, b1), (B, np.zeros(3, np.float32)), (np.array([[1, 2, 3]], np.float32), np.zeros(1, np.float32))]
    s = oracle.mlp(3, 1, _packed(layers), r0=0.0, alpha=1.0, beta=1.0)
    P = np.array([[0.3, -0.4, 0.5], [-0.9, 0.8, 0.1]])
    h = np.maximum(P @ A.T.astype(np.float64) + b1, 0)
    h = np.maximum(h @ B.T.astype(np.float64), 0)
    g = h @ np.array([1, 2, 3.0])
    np.testing.assert_allclose(s.eval(P), np.linalg.norm(P, axis=1) + g, atol=1e-15)


@pytest.mark.parametrize("width", [64, 128, 256])
def test_generator_spectral_norms(width):
    for W, b in synth.mlp_layers(1, width):
        assert np.linalg.svd(W.astype(np.float64), compute_uv=False)[0] <= 1 + 1e-6


def test_c2_network_is_a_distance_bound():
    s = oracle.mlp(256, synth.MLP_NMID, synth.mlp_params(1, 256).astype(np.float64))
    rng = np.random.default_rng(5)
    A = rng.uniform(-1, 1, (2000, 3))
    B = A + rng.normal(0, 0.05, A.shape)
    lip = np.abs(s.eval(A) - s.eval(B)) / np.linalg.norm(A - B, axis=1)
    assert lip.max() <= 1 + 1e-6
    # a closed surface inside the unit ball: f < 0 at the origin, f > 0 on the domain's corners
    f0 = s.eval(np.zeros((1, 3)))[0]
    g0 = (f0 * 1.1 + 0.6) / 0.1
    assert abs(g0) < 3 and f0 < 0
    corners = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], np.float64)
    assert (s.eval(corners) > 0).all()


def test_grad_x_matches_central_differences():
    w = 48
    s = oracle.mlp(w, synth.MLP_NMID, synth.mlp_params(2, w).astype(np.float64), lam=1.3)
    rng = np.random.default_rng(1)
    P = rng.uniform(-0.9, 0.9, (50, 3))
    G = s.grad_x(P)
    d = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = d
        fd = (s.eval(P + e) - s.eval(P - e)) / (2 * d)
        np.testing.assert_allclose(G[:, a], fd, rtol=1e-6, atol=1e-8)


def test_grad_theta_matches_central_differences():
    w = 16
    nmid = 3
    base = synth.mlp_params(3, w, nmid).astype(np.float64)
    s = oracle.mlp(w, nmid, base)
    p = np.array([0.31, -0.42, 0.27])
    g = s.grad_theta_point(p)
    rng = np.random.default_rng(2)
    idx = rng.choice(base.size, 40, replace=False)
    d = 1e-6
    for i in idx:
        hi = base.copy()
        lo = base.copy()
        hi[i] += d
        lo[i] -= d
        fd = (oracle.mlp(w, nmid, hi).eval(p[None])[0] - oracle.mlp(w, nmid, lo).eval(p[None])[0]) / (2 * d)
        assert abs(g[i] - fd) <= 1e-7 + 1e-5 * abs(fd)


def test_adjoint_matches_implicit_fd_target():
    """dL/dtheta of the implicit rule equals the derivative of
    L(v - (f(v;theta') - f(v;theta)) grad_x f / |grad_x f|^2) at theta' = theta."""
    w = 24
    nmid = 3
    base = synth.mlp_params(4, w, nmid).astype(np.float64)
    s = oracle.mlp(w, nmid, base)
    hr, mr = oracle.polygonize(s, 24)
    keys, pos = mr.tri_keys.ravel(), mr.tri_pos.reshape(-1, 3)
    _, first = np.unique(keys, return_index=True)
    V = pos[first]
    c = np.array([0.02, -0.01, 0.03])

    def loss(v):
        r = np.linalg.norm(v - c, axis=1)
        return np.mean((r - 0.55) ** 2)

    r = np.linalg.norm(V - c, axis=1)
    dldv = (2 * (r - 0.55) / r)[:, None] * (V - c) / V.shape[0]
    g = s.adjoint(V, dldv)
    gx = s.grad_x(V)
    f0 = s.eval(V)
    n2 = (gx * gx).sum(1)

    def implicit_loss(params):
        f1 = oracle.mlp(w, nmid, params).eval(V)
        return loss(V - ((f1 - f0) / n2)[:, None] * gx)

    rng = np.random.default_rng(3)
    # a small step keeps the perturbation from crossing a ReLU kink of the
    # piecewise-smooth loss at any of the ~10^3 vertices
    d = 1e-7
    for i in rng.choice(base.size, 24, replace=False):
        hi = base.copy()
        lo = base.copy()
        hi[i] += d
        lo[i] -= d
        fd = (implicit_loss(hi) - implicit_loss(lo)) / (2 * d)
        # relative error, floored at 1e-6 of the largest component (the FD
        # round-off is about 1e-19 / (2 d) in absolute terms)
        assert abs(g[i] - fd) <= 1e-5 * abs(fd) + 1e-6 * np.abs(g).max(), (i, g[i], fd)


def test_numpy_helpers_match_the_c_oracle():
    """The matmul-based FP64 helpers restate the C oracle's definitions; they
    must agree with it (values, input gradient, adjoint)."""
    w, nmid = 32, 3
    params = synth.mlp_params(6, w, nmid).astype(np.float64)
    s = oracle.mlp(w, nmid, params, lam=1.2)
    rng = np.random.default_rng(4)
    P = rng.uniform(-0.9, 0.9, (300, 3))
    np.testing.assert_allclose(oracle.np_eval(params, w, nmid, P, lam=1.2), s.eval(P), rtol=0, atol=1e-14)
    np.testing.assert_allclose(oracle.np_grad_x(params, w, nmid, P, lam=1.2), s.grad_x(P), rtol=1e-12, atol=1e-14)
    G = rng.normal(size=P.shape)
    np.testing.assert_allclose(oracle.np_adjoint(params, w, nmid, P, G, lam=1.2), s.adjoint(P, G), rtol=1e-10,
                               atol=1e-14)
