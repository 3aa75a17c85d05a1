"""The GPU-vs-oracle comparator itself, on the CPU: an oracle mesh compared
with itself passes with nothing excluded, and each planted mistake (a
dropped triangle, a changed case index, a moved vertex, a missing surface
cell) is reported and makes the checking form fail."""
import numpy as np
import pytest

import oracle
import parity
from paper_2111_05778_gb300 import synth

torch = pytest.importorskip("torch")


class _Mesh:
    def __init__(self, cells, cases, keys, pos):
        self.cell_ids = torch.from_numpy(np.asarray(cells, np.int64))
        self.cell_cases = torch.from_numpy(np.asarray(cases, np.uint8))
        self.tri_keys = torch.from_numpy(np.asarray(keys, np.int64))
        self.tri_xyz = torch.from_numpy(np.asarray(pos, np.float32))


def _setup(N=24):
    prims = synth.csg_prims(3)
    o = oracle.csg(prims)
    ref = oracle.enum(o, N)
    sel = (ref.cases > 0) & (ref.cases < 255)
    mesh = dict(cells=ref.cells[sel], cases=ref.cases[sel], keys=ref.tri_keys, pos=ref.tri_pos)
    f32 = lambda p: o.eval(np.asarray(p, np.float64))  # FP64 values at the float32 points
    return o, ref, mesh, f32


def test_self_comparison_is_exact():
    o, ref, m, f32 = _setup()
    st = parity.compare(_Mesh(**m), o, 24, ref=ref, f32=f32)
    assert st["mismatched_cells"] == st["mismatched_tris"] == st["vertices_over_tol"] == 0
    assert st["cells"] > 500 and st["bare_frac"] == 1.0


@pytest.mark.parametrize("plant", ["drop_tri", "case", "vertex", "drop_cell"])
def test_planted_mistakes_are_caught(plant):
    o, ref, m, f32 = _setup()
    m = {k: np.array(v) for k, v in m.items()}
    h = 2.0 / 24
    if plant == "drop_tri":
        m["keys"], m["pos"] = m["keys"][1:], m["pos"][1:]
    elif plant == "case":
        m["cases"][5] ^= 1 if m["cases"][5] not in (1, 254) else 3
    elif plant == "vertex":
        hit = m["keys"] == m["keys"][7, 1]  # every copy of that vertex
        m["pos"][hit, 2] += np.float32(1e-3 * h)
    else:
        m["cells"], m["cases"] = m["cells"][1:], m["cases"][1:]
    st = parity.compare(_Mesh(**m), o, 24, ref=ref, f32=f32, check=False)
    assert st["mismatched_cells"] + st["mismatched_tris"] + st["vertices_over_tol"] > 0
    with pytest.raises(AssertionError):
        parity.compare(_Mesh(**m), o, 24, ref=ref, f32=f32)
