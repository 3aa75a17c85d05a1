"""Pins for the oracle's serial grid hopper (Sec. 3, Algorithm 1) against
what the paper fixes: the hopper finds exactly the cells enumeration finds
(Sec. 5: all methods give the same mesh), the plane analyses of Sec. 4.1
(Case 1 escape by doubling, Case 2 the harmonic bound) and the
O(N^2 log N) growth."""
import math

import numpy as np
import pytest

import oracle
from paper_2111_05778_gb300 import synth


def _surface(res):
    c, k = res.cells, res.cases
    return set(c[(k > 0) & (k < 255)].tolist())


@pytest.mark.parametrize("N", [16, 32, 64, 128])
def test_sphere_hop_equals_enumeration(N):
    s = oracle.csg(synth.sphere_prims(0.5))
    hr, mr = oracle.polygonize(s, N)
    er = oracle.enum(s, N)
    assert _surface(mr) == set(er.cells.tolist())
    assert set(er.cells.tolist()) <= set(hr.marks.tolist())
    # identical meshes (Sec. 5): same triangle multiset
    a = np.sort(np.sort(mr.tri_keys, axis=1), axis=0)
    b = np.sort(np.sort(er.tri_keys, axis=1), axis=0)
    assert a.shape == b.shape and (np.sort(a.view("i8,i8,i8"), axis=0) == np.sort(b.view("i8,i8,i8"), axis=0)).all()


@pytest.mark.parametrize("tau_mode", [oracle.TAU_DIAGONAL, oracle.TAU_HALF_DIAGONAL])
def test_csg_hop_equals_enumeration(tau_mode):
    s = oracle.csg(synth.csg_prims(0))
    N = 96
    hr, mr = oracle.polygonize(s, N, tau_mode=tau_mode)
    er = oracle.enum(s, N)
    assert _surface(mr) == set(er.cells.tolist())
    assert mr.tri_keys.shape == er.tri_keys.shape


def test_mlp_hop_equals_enumeration():
    w = 32
    s = oracle.mlp(w, synth.MLP_NMID, synth.mlp_params(1, w).astype(np.float64))
    N = 48
    hr, mr = oracle.polygonize(s, N)
    er = oracle.enum(s, N)
    assert len(er.cells) > 1000
    assert _surface(mr) == set(er.cells.tolist())


def test_eps_shrink_keeps_surface():
    s = oracle.csg(synth.csg_prims(3))
    N = 64
    base = oracle.hop(s, N)
    shr = oracle.hop(s, N, eps=0.3 * 2.0 / N)
    er = oracle.enum(s, N)
    assert set(er.cells.tolist()) <= set(shr.marks.tolist())
    assert shr.col_evals.sum() >= base.col_evals.sum()


def _parallel_plane_expected(N, C, tau_mode):
    """Case 2 of Sec. 4.1: the plane x = C is parallel to the rays, so every
    evaluation along column i returns the same distance D_i = |x_i - C| and
    the ray advances by a constant s_i cells: ceil(N / s_i) evaluations."""
    h = 2.0 / N
    tau = math.sqrt(3.0) * h * (1.0 if tau_mode == 0 else 0.5)
    per_i = []
    for i in range(N):
        D = abs(-1.0 + (i + 0.5) * h - C)
        if D <= tau:
            per_i.append(N)
        else:
            s = max(1, math.floor(D / h))
            per_i.append(-(-N // s))
    return np.repeat(np.array(per_i, np.int64), N)


@pytest.mark.parametrize("N", [32, 64, 128])
@pytest.mark.parametrize("tau_mode", [0, 1])
def test_parallel_plane_closed_form(N, tau_mode):
    prims = synth.half_space_prims([1.0, 0.0, 0.0], 0.1234)
    C = prims[0, 2] + prims[0, 5]  # effective plane position after float32 rounding
    s = oracle.csg(prims)
    hr = oracle.hop(s, N, tau_mode=tau_mode)
    np.testing.assert_array_equal(hr.col_evals, _parallel_plane_expected(N, C, tau_mode))
    # the paper's bound S <= N^2 (1 + 2 H_N), up to the fully marked columns
    H = sum(1.0 / n for n in range(1, N + 1))
    assert hr.col_evals.sum() <= N * N * (1 + 2 * H) + 3 * N * N


@pytest.mark.parametrize("N", [32, 64, 128, 256, 512])
def test_perpendicular_plane_escape_doubles(N):
    """Case 1 of Sec. 4.1: one approach step, a couple of polygonized cells,
    then the distance doubles each step: about log2 N steps per ray."""
    s = oracle.csg(synth.half_space_prims([0.0, 0.0, 1.0], -0.3127))
    hr = oracle.hop(s, N, cols=np.arange(0, N * N, max(1, N * N // 257)))
    ev = hr.col_evals
    assert (ev == ev[0]).all()
    assert math.log2(N) - 1 <= ev[0] <= math.log2(N) + 6


def test_general_plane_logarithmic():
    """Case 3 of Sec. 4.1: geometric approach and escape, O(log N) per ray."""
    per = []
    for N in (32, 64, 128, 256, 512):
        s = oracle.csg(synth.half_space_prims([0.3, -0.5, 0.81], 0.05))
        hr = oracle.hop(s, N)
        per.append(hr.col_evals.mean())
    per = np.array(per)
    inc = np.diff(per)
    # grows by a bounded amount per doubling of N (log N), not by a factor 2 (N)
    assert (inc > 0).all() and (inc < 0.6 * per[:-1]).all()


def test_sphere_n2logn_growth():
    """Sec. 4: evaluations grow like N^2 log N: evals/N^2 is affine in log2 N
    and evals/N^3 falls."""
    s = oracle.csg(synth.sphere_prims(0.5))
    Ns = np.array([32, 64, 128, 256, 512])
    ev = np.array([oracle.hop(s, int(N)).col_evals.sum() for N in Ns], np.float64)
    y = ev / Ns**2
    x = np.log2(Ns)
    a, b = np.polyfit(x, y, 1)
    assert a > 0
    assert np.max(np.abs(y - (a * x + b)) / y) < 0.10
    assert (np.diff(ev / Ns**3) < 0).all()
