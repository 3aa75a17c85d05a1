"""Randomised pins of the oracle's serial hopper (Sec. 3, Algorithm 1): on
random scenes of all seven primitives under union, subtraction and a final
intersection, over random grid sizes and offset domains, the hopper's
surface cells and mesh equal enumeration's (the Sec. 5 invariant).  Drawn by
hypothesis where it is installed."""
import numpy as np
import pytest

import oracle
from paper_2111_05778_gb300 import synth

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")


def _surface(res):
    c, k = res.cells, res.cases
    return set(c[(k > 0) & (k < 255)].tolist())


def _tris(res):
    t = np.sort(res.tri_keys, axis=1)
    return sorted(map(tuple, t.tolist()))


@hyp.settings(max_examples=60, deadline=None, derandomize=True)
@hyp.given(seed=st.integers(0, 10_000), n=st.integers(3, 16), N=st.integers(4, 40),
           lo=st.floats(-1.2, -0.6), span=st.floats(1.2, 2.4),
           tau_mode=st.sampled_from([oracle.TAU_DIAGONAL, oracle.TAU_HALF_DIAGONAL]))
def test_random_scene_hop_equals_enumeration(seed, n, N, lo, span, tau_mode):
    s = oracle.csg(synth.mixed_prims(seed, n))
    hr, mr = oracle.polygonize(s, N, lo, lo + span, tau_mode=tau_mode)
    er = oracle.enum(s, N, lo, lo + span)
    assert _surface(mr) == set(er.cells.tolist())
    assert set(er.cells.tolist()) <= set(hr.marks.tolist())
    assert _tris(mr) == _tris(er)


@hyp.settings(max_examples=20, deadline=None, derandomize=True)
@hyp.given(seed=st.integers(0, 10_000), width=st.sampled_from([16, 32]), N=st.integers(6, 28),
           tau_mode=st.sampled_from([oracle.TAU_DIAGONAL, oracle.TAU_HALF_DIAGONAL]))
def test_random_network_hop_equals_enumeration(seed, width, N, tau_mode):
    s = oracle.mlp(width, synth.MLP_NMID, synth.mlp_params(seed, width).astype(np.float64))
    hr, mr = oracle.polygonize(s, N, tau_mode=tau_mode)
    er = oracle.enum(s, N)
    assert len(er.cells) > 0
    assert _surface(mr) == set(er.cells.tolist())
    assert _tris(mr) == _tris(er)
